"""GPU parity at the full sizes the benchmark times for the batched and the
query workloads, against the FP64 oracle.

- 64 batched maps (the benchmark's seeds 3000-3063: 50.6M points, grids of
  128-1024 cells a side, 4-48 slices): one autotuned batched call captured in
  a CUDA graph and replayed, as the benchmark times it; every map's layers,
  masks, keep flags and statistics against the oracle run on that map alone
  (Sec. III-A/B/C per map).
- the parking structure built, then evaluated on its layers: bit-identical
  to the fused call.
- 256 paths x 512 waypoints on the evaluated 5M-point parking structure: the
  cost / elevation queries and their adjoint (the C(q), e^G(q) of Eq. 10)
  against the oracle's values and analytic gradients, and the 50-step
  refinement: each of the 50 steps against one oracle step from the same
  float32 waypoints, and the fused 50-step launch against the 50 single steps.
Tolerances as in _parity.py (layers) and test_sample_gpu.py (queries).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from conftest import PARAMS_ROBOT  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import _parity as P  # noqa: E402
import oracle  # noqa: E402
from paper_2403_07631_gb300 import build, scenes, tct  # noqa: E402

RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.compile_library()


def _grid(sc):
    return tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, sc.n_slices, 0.0, True)


def test_batched_64_maps_full_size_graph_replay():
    scs = scenes.batched_maps()
    assert len(scs) == 64
    maps = [tct.MapBuffers.allocate(torch.from_numpy(sc.points).cuda(), _grid(sc)) for sc in scs]
    ws = torch.empty(tct.tct_workspace_bytes_batched(maps, PARAMS_ROBOT), dtype=torch.uint8,
                     device="cuda")
    tuning = tct.tct_autotune_batched(maps, PARAMS_ROBOT, ws)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        tct.tct_build_evaluate_batched(maps, PARAMS_ROBOT, ws, tuning)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        tct.tct_build_evaluate_batched(maps, PARAMS_ROBOT, ws, tuning)
    for m in maps:                       # the replay must write every output
        m.ground.fill_(float("nan"))
        m.ceil.fill_(float("nan"))
        m.cost.fill_(float("nan"))
        m.mask.fill_(7)
        m.keep.fill_(7)
        m.stats.zero_()
    graph.replay()
    torch.cuda.synchronize()
    n_cells = 0
    for sc, m in zip(scs, maps):
        got = {k: getattr(m, k).cpu().numpy() for k in ("ground", "ceil", "cost", "mask", "keep")}
        ref = P.oracle_all(sc.points, _grid(sc), PARAMS_ROBOT)
        where = f" ({sc.name}: {len(sc.points)} points, {sc.H} x {sc.W} x {sc.n_slices})"
        P.assert_equal_layers(got["ground"], ref["ground"], "ground" + where)
        P.assert_equal_layers(got["ceil"], ref["ceil"], "ceiling" + where)
        P.assert_costs(got["cost"], ref["cost"], ref["fragile"])
        P.assert_masks(got["mask"], ref["mask"], ref["fragile"])
        P.assert_keep(got["keep"], got["ground"], got["cost"], ref, PARAMS_ROBOT)
        st = tct.stats_from(m.stats)
        assert st.n_points == len(sc.points) and st.n_dropped == ref["dropped"]
        assert st.n_kept == int(got["keep"].sum())
        N = sc.n_slices
        np.testing.assert_array_equal(np.array(st.valid_cells[:N]),
                                      (ref["ground"] > -np.inf).reshape(N, -1).sum(1))
        np.testing.assert_array_equal(np.array(st.trav_cells[:N]),
                                      got["mask"].reshape(N, -1).sum(1))
        n_cells += got["cost"].size
    assert n_cells > 400_000_000          # the whole batch was compared


@pytest.fixture(scope="module")
def parking():
    sc = scenes.parking_structure()
    g = P.gpu_build_evaluate(sc.points, _grid(sc), PARAMS_ROBOT)
    st = g["stats"]
    k = int(max(range(sc.n_slices), key=lambda i: st.trav_cells[i]))
    z_min = float(st.z_min)
    grid = tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, sc.n_slices, z_min, True)
    og = oracle.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, z_min, sc.n_slices)
    xy = scenes.straight_paths(g["mask"][k] != 0, sc.x0, sc.y0, sc.res, 256, 512)
    sl = np.full(xy.shape[:2], k, np.int32)
    return dict(grid=grid, og=og, cost=g["cost"], ground=g["ground"], mask=g["mask"],
                keep=g["keep"], stats=st, xy=xy, sl=sl)


def _close(a, b, scale, what):
    err = np.abs(a.astype(np.float64) - b)
    lim = RTOL * np.maximum(np.abs(b), scale)
    bad = ~(err <= lim)
    assert not bad.any(), f"{what}: {int(bad.sum())} out of tolerance, max err {err[bad].max()}"


def test_paths_queries_and_adjoint_full_size(parking):
    p = parking
    grid, og, cost, ground = p["grid"], p["og"], p["cost"], p["ground"]
    xy, sl = p["xy"].reshape(-1, 2), p["sl"].reshape(-1)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (xy, sl, cost, ground)]
    c_out = torch.empty(len(xy), device="cuda")
    e_out = torch.empty(len(xy), device="cuda")
    tct.tct_sample_cost(grid, d[2], d[3], d[0], d[1], c_out, e_out)
    rng = np.random.default_rng(9)
    wc = rng.normal(size=len(xy)).astype(np.float32)
    we = rng.normal(size=len(xy)).astype(np.float32)
    gxy = torch.empty_like(d[0])
    tct.tct_sample_cost_backward(grid, d[2], d[3], d[0], d[1], torch.from_numpy(wc).cuda(),
                                 torch.from_numpy(we).cuda(), gxy)
    torch.cuda.synchronize()
    rc, gc = oracle.sample(og, cost, xy, sl)
    re, ge = oracle.sample(og, ground, xy, sl, is_ground=True)
    zmax = float(np.abs(ground[np.isfinite(ground)]).max())
    _close(c_out.cpu().numpy(), rc, PARAMS_ROBOT["c_b"], "cost")
    _close(e_out.cpu().numpy(), re, zmax, "elevation")
    ref = wc[:, None].astype(np.float64) * gc + we[:, None].astype(np.float64) * ge
    scale = (np.abs(wc) * PARAMS_ROBOT["c_b"] + np.abs(we) * zmax)[:, None] / grid.res
    _close(gxy.cpu().numpy(), ref, scale, "gradient")


def test_paths_refinement_50_steps_full_size(parking):
    p = parking
    grid, og, cost = p["grid"], p["og"], p["cost"]
    eta, lam, steps = 1e-3, 1.0, 50
    d_c = torch.from_numpy(cost).cuda()
    d_sl = torch.from_numpy(p["sl"]).cuda()
    fused = torch.from_numpy(p["xy"]).cuda()
    tct.tct_refine_paths(grid, d_c, d_sl, fused, steps, eta, lam)
    stepped = torch.from_numpy(p["xy"]).cuda()
    for s in range(steps):
        before = stepped.cpu().numpy()
        tct.tct_refine_paths(grid, d_c, d_sl, stepped, 1, eta, lam)
        after = stepped.cpu().numpy()
        # one oracle step (FP64 update, queries at the same float32 waypoints)
        ref = oracle.refine(og, cost, p["sl"], before, steps=1, eta=eta, lam=lam)
        # the waypoint moves by eta * gradient; the gradient's tolerance is
        # 1e-5 c^B / r_g, and the float32 waypoint carries half an ulp of ~100 m
        lim = eta * RTOL * PARAMS_ROBOT["c_b"] / grid.res + 8e-6
        err = np.abs(after.astype(np.float64) - ref)
        assert err.max() <= lim, f"step {s}: max error {err.max()} above {lim}"
    torch.cuda.synchronize()
    np.testing.assert_array_equal(fused.cpu().numpy(), stepped.cpu().numpy())


def test_parking_build_then_evaluate_equals_fused(parking):
    """The paper times construction and evaluation separately (Sec. IV-A):
    tct_build then tct_evaluate on its layers (the incremental kernel in the
    tile shape the benchmark's workload takes, with the given layers in place
    of the pointer advance) give the fused call's costs, masks, keep flags
    and per-slice counts bit for bit at full size (the fused outputs are
    compared with the oracle in test_parity_gpu)."""
    sc = scenes.parking_structure()
    g_b, c_b, st_b = P.gpu_build(sc.points, _grid(sc))
    z_min = float(st_b.z_min)
    egrid = tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, sc.n_slices, z_min, False)
    ev = P.gpu_evaluate(g_b, c_b, egrid, PARAMS_ROBOT, aux=False)
    np.testing.assert_array_equal(g_b, parking["ground"])
    np.testing.assert_array_equal(ev["cost"], parking["cost"])
    np.testing.assert_array_equal(ev["mask"], parking["mask"])
    np.testing.assert_array_equal(ev["keep"], parking["keep"])
    assert ev["stats"].trav_cells[:sc.n_slices] == parking["stats"].trav_cells[:sc.n_slices]
