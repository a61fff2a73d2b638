"""The reference arm of the benchmark (the FP64 oracle on the host cores):
one JSON line with the keys the contract asks for, on rank 0 only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--workload", "building", "--steps", "1", "--warmup", "0"],
                          capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)


def test_reference_line_on_rank0():
    r = _run({})
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "Mpoints/s"
    assert line["steps"] == 1 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_reference_other_ranks_print_nothing():
    r = _run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_reference_arm_loads_no_cuda_library():
    # the oracle arm runs the oracle alone: neither the ctypes binding nor
    # libtct.so may be loaded into its process
    code = (
        "import sys, runpy\n"
        "sys.argv = ['bench.py', '--impl', 'reference', '--workload', 'building', "
        "'--steps', '1', '--warmup', '0']\n"
        "runpy.run_path('bench.py', run_name='__main__')\n"
        "maps = open('/proc/self/maps').read()\n"
        "assert 'libtct' not in maps, 'libtct.so mapped'\n"
        "assert 'paper_2403_07631_gb300.tct' not in sys.modules, 'binding imported'\n"
        "print('clean')\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().splitlines()[-1] == "clean"


def test_bench_robot_is_the_library_robot():
    # the parameters written out in bench.py equal the binding's robot_params()
    sys.path.insert(0, ROOT)
    import bench
    from paper_2403_07631_gb300 import tct
    lib = tct.robot_params()
    for k, v in bench.ROBOT_PARAMS.items():
        if k == "flags":
            continue
        assert abs(float(lib[k]) - float(v)) <= 1e-7 * max(1.0, abs(float(v))), k
