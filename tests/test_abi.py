"""The C ABI: libtct.so builds for sm_103a, loads without a GPU and exports
every entry point include/tct.h declares; host-only calls behave as the
header documents (no kernel is launched here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tct.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[a-z_ ]*?[a-z_0-9]+\s*\*?\s*(tct_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_07631_gb300 import build, tct
    build.build()
    return tct.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("tct_build", "tct_evaluate", "tct_build_evaluate", "tct_bounds",
              "tct_workspace_bytes", "tct_plan_grid", "tct_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), f"libtct.so does not export {n}"


def test_binding_covers_every_declared_symbol():
    from paper_2403_07631_gb300 import tct
    for n in declared_functions():
        assert n in tct._SIGNATURES, f"binding lacks {n}"


def test_struct_layouts_match_header(lib):
    from paper_2403_07631_gb300 import tct
    assert ctypes.sizeof(tct.TctGrid) == 36
    assert ctypes.sizeof(tct.TctParams) == 52
    assert ctypes.sizeof(tct.TctStats) == 48 + 2 * 8 * 128


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every struct of the header, compiled by the host C compiler: the same
    size and the same offset of every field as the binding's ctypes types."""
    import shutil
    import subprocess
    from paper_2403_07631_gb300 import tct
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    types = {"tct_grid": tct.TctGrid, "tct_params": tct.TctParams, "tct_stats": tct.TctStats,
             "tct_map": tct.TctMap, "tct_tuning": tct.TctTuning, "tct_host_io": tct.TctHostIO}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tct.h"', 'int main(void) {']
    for cname, ct in types.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in ct._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['    return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        cname, what, value = line.split()
        ct = types[cname]
        got = ctypes.sizeof(ct) if what == "size" else getattr(ct, what).offset
        assert got == int(value), f"{cname}.{what}: binding {got}, C {value}"


def test_host_only_calls(lib):
    from paper_2403_07631_gb300 import tct
    assert tct.tct_status_string(0) == "ok"
    assert "workspace" in tct.tct_status_string(-2)
    p = tct.params_default()
    assert p["c_b"] == 50.0 and p["patch_radius"] == 2
    g = tct.tct_plan_grid([0.0, 0.0, -0.0499, 19.99, 19.95, 5.84], 0.1, 0.5)
    assert (g.W, g.H, g.n_slices) == (200, 200, 12)
    # the hand-worked cell edges of the oracle's pin (r_g = 0.25, exact): a
    # maximum on the left edge of cell 8 opens it, one just inside does not
    for (xmax, ymax, W, H) in ((2.0, 0.75, 9, 4), (1.99, 0.7499, 8, 3), (0.25, 0.0, 2, 1)):
        g = tct.tct_plan_grid([0.0, 0.0, 0.0, xmax, ymax, 0.3], 0.25, 0.5)
        assert (g.x0, g.y0, g.W, g.H, g.n_slices) == (0.0, 0.0, W, H, 1)
    with pytest.raises(tct.TctError):
        tct.tct_plan_grid([0.0, 0.0, 0.0, 1.0, 1.0, 1000.0], 0.1, 0.5)   # N > 127
    n = tct.tct_workspace_bytes(tct.Grid(0.0, 0.0, 0.1, 1000, 1000, 0.5, 40), 5_000_000)
    assert n >= 4 * 5_000_000 + 8 * 1_000_000
    with pytest.raises(tct.TctError):
        tct.tct_workspace_bytes(tct.Grid(0.0, 0.0, -0.1, 10, 10, 0.5, 4), 10)


def test_argument_errors_need_no_gpu(lib):
    from paper_2403_07631_gb300 import tct
    g = tct.Grid(0.0, 0.0, 0.1, 10, 10, 0.5, 4).c()
    P = tct.TctParams(**{k: v for k, v in tct.params_default().items()})
    # NULL buffers and a too-small workspace are refused before any launch
    rc = lib.tct_build_evaluate(None, 10, 3, ctypes.byref(g), ctypes.byref(P), None, 0,
                                None, None, None, None, None, None, None)
    assert rc == -1
    fake = ctypes.c_void_p(256)
    rc = lib.tct_build_evaluate(fake, 10, 3, ctypes.byref(g), ctypes.byref(P), fake, 16,
                                fake, fake, fake, fake, fake, None, None)
    assert rc == -2
    rc = lib.tct_build_evaluate(fake, 10, 5, ctypes.byref(g), ctypes.byref(P), fake, 1 << 30,
                                fake, fake, fake, fake, fake, None, None)
    assert rc == -1
    g.n_slices = 200
    rc = lib.tct_evaluate(ctypes.byref(g), ctypes.byref(P), fake, fake, fake, 1 << 30,
                          fake, fake, fake, None, None, None)
    assert rc == -4


def test_constants_match_the_header(tmp_path):
    """Every constant the binding mirrors has the header's value."""
    import shutil
    import subprocess
    from paper_2403_07631_gb300 import tct
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = {"TCT_OK": tct.OK, "TCT_MAX_SLICES": tct.MAX_SLICES,
             "TCT_GRID_ZMIN_FROM_DATA": tct.GRID_ZMIN_FROM_DATA, "TCT_KEEP_ENDS": tct.KEEP_ENDS,
             "TCT_ALLOW_COARSE": tct.ALLOW_COARSE, "TCT_DEV_NONFINITE": tct.DEV_NONFINITE,
             "TCT_DEV_BAD_QUERY": tct.DEV_BAD_QUERY, "TCT_MAX_PATH_LEN": tct.MAX_PATH_LEN,
             "TCT_NOALLOC_SCRATCH_BYTES": tct.NOALLOC_SCRATCH_BYTES,
             "TCT_MAX_BATCH": tct.MAX_BATCH, "TCT_TILE_AUTO": tct.TILE_AUTO,
             "TCT_TILE_64": tct.TILE_64, "TCT_TILE_32": tct.TILE_32,
             "TCT_TILE_64x56": tct.TILE_64x56, "TCT_TILE_64x40": tct.TILE_64x40,
             "TCT_TILE_128x56": tct.TILE_128x56,
             "TCT_HOST_KEPT_ONLY": tct.HOST_KEPT_ONLY}
    lines = ['#include <stdio.h>', '#include "tct.h"', 'int main(void) {']
    lines += [f'    printf("{k} %lld\\n", (long long)({k}));' for k in pairs]
    lines += ['    return 0;', '}']
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in filter(None, out.split("\n")):
        name, value = line.split()
        assert pairs[name] == int(value), f"{name}: binding {pairs[name]}, header {value}"
