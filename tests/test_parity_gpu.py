"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on
the same seeded inputs, element by element (tolerances in tests/_parity.py).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from conftest import PARAMS_ROBOT, PARAMS_TABLE1  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import _parity as P  # noqa: E402
from paper_2403_07631_gb300 import scenes, tct  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_07631_gb300 import build
    build.build()
    import oracle
    oracle.compile_library()


def _grid_of(sc, n_slices=None, zmin_from_data=True, z_min=0.0):
    return tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s,
                    n_slices if n_slices else sc.n_slices, z_min, zmin_from_data)


def _full_check(points, grid, params, stride=3, misalign=False):
    g = P.gpu_build_evaluate(points, grid, params, stride=stride, misalign=misalign)
    r = P.oracle_all(points, grid, params)
    P.assert_equal_layers(g["ground"], r["ground"], "ground")
    P.assert_equal_layers(g["ceil"], r["ceil"], "ceiling")
    P.assert_costs(g["cost"], r["cost"], r["fragile"])
    P.assert_masks(g["mask"], r["mask"], r["fragile"])
    P.assert_keep(g["keep"], g["ground"], g["cost"], r, params)
    st = g["stats"]
    assert st.status == 0 or st.n_nonfinite > 0
    assert st.n_dropped == r["dropped"]
    assert st.n_nonfinite == r["nonfinite"]
    assert st.n_points == len(points)
    assert st.n_kept == int(g["keep"].sum())
    N = grid.n_slices
    np.testing.assert_array_equal(np.array(st.valid_cells[:N]),
                                  (r["ground"] > -np.inf).reshape(N, -1).sum(1))
    np.testing.assert_array_equal(np.array(st.trav_cells[:N]), g["mask"].reshape(N, -1).sum(1))
    return g, r


# ---------------------------------------------------------------- construction

@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("stride", [3, 4])
def test_build_random_cloud(seed, stride):
    rng = np.random.default_rng(seed)
    n = 50_003                                   # ragged: not a multiple of 4
    pts = np.stack([rng.uniform(-0.5, 7.3, n), rng.uniform(-0.2, 5.1, n),
                    rng.choice([0.0, 0.3, 1.2, 2.5], n) + rng.normal(0, 0.2, n)], 1).astype(np.float32)
    grid = tct.Grid(0.0, 0.0, 0.1, 71, 49, 0.5, 6, 0.0, True)
    ground, ceil, st = P.gpu_build(pts, grid, stride=stride)
    eG, eC, og, dropped, bad = P.oracle.build(pts, P.oracle_grid(grid), True)
    P.assert_equal_layers(ground, eG, "ground")
    P.assert_equal_layers(ceil, eC, "ceiling")
    assert st.n_dropped == dropped and st.n_nonfinite == 0
    assert st.z_min == pts[:, 2].min() and st.z_max == pts[:, 2].max()


def test_build_given_zmin_and_overflow_bin():
    # explicit z_min and too few planes: points above the last plane only
    # ever appear as ceilings
    sc = scenes.building(5, 30_000, side_cells=60, floors=[0.0, 3.0], ceilings=[2.8, 5.8])
    grid = _grid_of(sc, n_slices=5, zmin_from_data=False, z_min=-0.25)
    ground, ceil, st = P.gpu_build(sc.points, grid)
    eG, eC, _, _, _ = P.oracle.build(sc.points, P.oracle_grid(grid), False)
    P.assert_equal_layers(ground, eG, "ground")
    P.assert_equal_layers(ceil, eC, "ceiling")


def test_build_nonfinite_and_offgrid_points():
    rng = np.random.default_rng(9)
    pts = rng.uniform(0, 3, (1000, 3)).astype(np.float32)
    pts[::17, 0] = np.nan
    pts[5::23, 2] = np.inf
    pts[7::31, 1] = -np.inf
    pts[3::11, 0] = 50.0                         # far off the grid
    pts[4::13, 2] = -0.0
    grid = tct.Grid(0.0, 0.0, 0.1, 30, 30, 0.5, 7, 0.0, True)
    ground, ceil, st = P.gpu_build(pts, grid)
    eG, eC, _, dropped, bad = P.oracle.build(pts, P.oracle_grid(grid), True)
    P.assert_equal_layers(ground, eG, "ground")
    P.assert_equal_layers(ceil, eC, "ceiling")
    assert st.n_nonfinite == bad > 0 and st.n_dropped == dropped > 0
    assert st.status & tct.DEV_NONFINITE
    assert not np.any((ground == 0) & np.signbit(ground))     # -0 is stored as +0


def test_get_status_reads_the_device_word():
    pts = np.zeros((64, 3), np.float32)
    pts[:, :2] = 0.5
    grid = tct.Grid(0.0, 0.0, 0.1, 20, 20, 0.5, 4, 0.0, True)
    d = torch.from_numpy(pts).cuda()
    ws = torch.empty(tct.tct_workspace_bytes(grid, len(pts)), dtype=torch.uint8, device="cuda")
    g = torch.empty(grid.shape, device="cuda")
    c = torch.empty(grid.shape, device="cuda")
    stats = torch.zeros(tct.STATS_BYTES, dtype=torch.uint8, device="cuda")
    tct.tct_build(d, grid, ws, g, c, stats)
    assert tct.tct_get_status(stats) == 0
    d[3, 1] = float("nan")
    tct.tct_build(d, grid, ws, g, c, stats)
    assert tct.tct_get_status(stats) & tct.DEV_NONFINITE


def test_build_empty_cloud():
    pts = np.zeros((0, 3), np.float32)
    grid = tct.Grid(0.0, 0.0, 0.1, 20, 10, 0.5, 3, 0.0, False)
    ground, ceil, st = P.gpu_build(pts, grid)
    assert np.all(ground == -np.inf) and np.all(ceil == np.inf)


# ------------------------------------------------------------------ evaluation

def _evaluate_check(eG, eC, params, res=0.1):
    N, H, W = eG.shape
    grid = tct.Grid(0.0, 0.0, res, W, H, 0.5, N, 0.0, False)
    g = P.gpu_evaluate(eG, eC, grid, params)
    og = P.oracle.Grid(0.0, 0.0, res, W, H, 0.5, 0.0, N)
    op = P.oracle_params(params)
    cT, mask, frag, aux = P.oracle.evaluate(og, op, eG, eC, want_aux=True)
    P.assert_costs(g["cost"], cT, frag)
    P.assert_masks(g["mask"], mask, frag)
    ok = np.broadcast_to((frag & 1) == 0, aux.shape)
    ga = g["aux"].astype(np.float64)
    fin = np.isfinite(aux)
    assert np.array_equal(np.isfinite(ga), fin), "aux infinities differ"
    with np.errstate(invalid="ignore"):      # inf - inf on cells the check leaves out
        err = np.abs(ga - aux)
    lim = P.COST_RTOL * np.maximum(1.0, np.abs(aux))
    assert np.all((err <= lim)[ok & fin]), "intermediate values out of tolerance"
    keep_ref, robust = P.oracle.simplify(eG, cT, op["c_b"], frag)
    P.assert_keep(g["keep"], eG, g["cost"], dict(keep=keep_ref, robust=robust), params)
    # without the aux export the call runs the incremental slice stack (for
    # its window radii) on the given layers: the same checks
    gi = P.gpu_evaluate(eG, eC, grid, params, aux=False)
    P.assert_costs(gi["cost"], cT, frag)
    P.assert_masks(gi["mask"], mask, frag)
    P.assert_keep(gi["keep"], eG, gi["cost"], dict(keep=keep_ref, robust=robust), params)
    st = gi["stats"]
    np.testing.assert_array_equal(np.array(st.valid_cells[:N]), (eG > -np.inf).reshape(N, -1).sum(1))
    np.testing.assert_array_equal(np.array(st.trav_cells[:N]), gi["mask"].reshape(N, -1).sum(1))
    return g, cT, frag


@pytest.mark.parametrize("deg", [15.0, 25.0, 40.0])
def test_evaluate_tilted_plane(deg):
    t = math.tan(math.radians(deg))
    H, W = 37, 45
    j = np.arange(W)[None, :]
    i = np.arange(H)[:, None]
    eG = np.stack([((t * (j + 0.5) + 0.3 * t * (i + 0.5)) * 0.1).astype(np.float32)] * 2)
    eC = np.full_like(eG, np.inf)
    eC[1] = eG[1] + np.float32(0.55)
    g, cT, frag = _evaluate_check(eG, eC, PARAMS_ROBOT)


@pytest.mark.parametrize("params", [PARAMS_ROBOT, PARAMS_TABLE1,
                                    dict(PARAMS_ROBOT, theta_p=1.0),
                                    dict(PARAMS_ROBOT, patch_radius=0),
                                    dict(PARAMS_ROBOT, patch_radius=4)])
def test_evaluate_random_layers(params):
    rng = np.random.default_rng(4)
    N, H, W = 5, 83, 67                          # ragged against 16- and 32-cell tiles
    base = (rng.normal(0, 0.04, (H, W)).cumsum(1) * 0.3).astype(np.float32)
    eG = np.stack([base + 0.4 * k for k in range(N)]).astype(np.float32)
    eG[rng.random(eG.shape) < 0.03] = -np.inf
    eC = (eG + rng.uniform(0.3, 1.5, eG.shape)).astype(np.float32)
    eC[rng.random(eG.shape) < 0.3] = np.inf
    _evaluate_check(eG, eC, params)


@pytest.mark.parametrize("theta_p", [0.37, 0.45])
def test_evaluate_step_patch_at_the_map_border(theta_p):
    # the oracle's border pin of the p_s patch (off-map neighbours count as
    # not gentle and stay in the denominator): a staircase whose step edges
    # run into the top and bottom borders (slice 0) and, transposed, into the
    # left and right borders (slice 1)
    j = np.arange(32)[None, :]
    st = np.broadcast_to((0.17 * (j // 4)).astype(np.float32), (32, 32))
    eG = np.ascontiguousarray(np.stack([st, st.T])).astype(np.float32)
    _evaluate_check(eG, np.full_like(eG, np.inf), dict(PARAMS_ROBOT, theta_p=theta_p))


def test_evaluate_fine_resolution_radius_12():
    # r_g = 0.05 m: D_inf = 6, D_sm = 7, a 25 x 25 window
    rng = np.random.default_rng(12)
    N, H, W = 3, 70, 90
    eG = np.zeros((N, H, W), np.float32) + (rng.normal(0, 0.003, (N, H, W))).astype(np.float32)
    eG[:, 30:33, 40:44] = 1.0                     # a block: barrier edges
    eC = np.full((N, H, W), np.inf, np.float32)
    _evaluate_check(eG, eC, PARAMS_ROBOT, res=0.05)


def test_evaluate_nonmonotone_layers_simplification():
    # layers that do not come from a build (ground not monotone in k)
    rng = np.random.default_rng(2)
    N, H, W = 6, 40, 40
    eG = rng.choice([0.0, 0.5, 1.0], (N, 1, 1)).astype(np.float32) + np.zeros((N, H, W), np.float32)
    eC = np.full((N, H, W), np.inf, np.float32)
    eC[:, 10:20, 10:20] = eG[:, 10:20, 10:20] + rng.uniform(0.5, 0.7, (N, 1, 1)).astype(np.float32)
    _evaluate_check(eG, eC, PARAMS_ROBOT)


# --------------------------------------------------------- fused build + evaluate

def test_evaluate_built_layers_equals_fused():
    # tct_evaluate on the layers tct_build_evaluate wrote gives exactly its
    # costs, masks and kept slices (one kernel, given layers for segments)
    sc = scenes.building(16, 90_000, side_cells=110, floors=[0.0, 2.4], ceilings=[2.2, 4.6])
    grid = _grid_of(sc, n_slices=11)
    f = P.gpu_build_evaluate(sc.points, grid, PARAMS_ROBOT)
    eg = tct.Grid(grid.x0, grid.y0, grid.res, grid.W, grid.H, grid.d_s, grid.n_slices, 0.0, False)
    g = P.gpu_evaluate(f["ground"], f["ceil"], eg, PARAMS_ROBOT, aux=False)
    for key in ("cost", "mask", "keep"):
        np.testing.assert_array_equal(g[key], f[key], err_msg=key)


def test_two_storey_building_full():
    sc = scenes.two_storey_building()
    g, r = _full_check(sc.points, _grid_of(sc, n_slices=12), PARAMS_ROBOT)
    assert r["robust"]
    assert g["keep"].sum() >= 2


@pytest.mark.parametrize("stride,misalign", [(4, False), (3, True)])
def test_building_point_layouts(stride, misalign):
    sc = scenes.building(8, 60_001, side_cells=90, floors=[0.0, 2.5], ceilings=[2.3, 4.9])
    _full_check(sc.points, _grid_of(sc, n_slices=11), PARAMS_ROBOT, stride=stride,
                misalign=misalign)


def test_keep_ends_and_table1():
    sc = scenes.building(10, 50_000, side_cells=70, floors=[0.0, 1.2, 2.9],
                         ceilings=[1.0, 2.7, 4.0])
    p = dict(PARAMS_TABLE1, flags=tct.KEEP_ENDS)
    g, r = _full_check(sc.points, _grid_of(sc, n_slices=10), p)
    assert g["keep"][0] == 1 and g["keep"][-1] == 1


def test_single_slice_and_tiny_grid():
    rng = np.random.default_rng(1)
    pts = np.stack([rng.uniform(0, 0.5, 400), rng.uniform(0, 0.3, 400),
                    rng.normal(0, 0.01, 400)], 1).astype(np.float32)
    _full_check(pts, tct.Grid(0.0, 0.0, 0.1, 5, 3, 0.5, 1, 0.0, True), PARAMS_ROBOT)


def test_parking_structure_full_size():
    # the 5M-point, 1000 x 1000 x 40 workload in the launch configuration the
    # benchmark times, every output compared with the oracle
    sc = scenes.parking_structure()
    g, r = _full_check(sc.points, _grid_of(sc), PARAMS_ROBOT)
    assert r["robust"]


def test_coverage_rule_rejected():
    grid = tct.Grid(0.0, 0.0, 0.1, 8, 8, 0.6, 2, 0.0, False)
    eG = np.zeros(grid.shape, np.float32)
    with pytest.raises(tct.TctError, match="exceeds d_min"):
        P.gpu_evaluate(eG, eG, grid, PARAMS_ROBOT)
    g = P.gpu_evaluate(eG, np.full_like(eG, np.inf), grid, dict(PARAMS_ROBOT, flags=tct.ALLOW_COARSE))
    assert g["cost"].shape == grid.shape


def test_fine_resolution_build_radius_12():
    # r_g = 0.05 m: the 25 x 25 inflation window of the build path
    sc = scenes.building(14, 120_000, side_cells=150, res=0.05, floors=[0.0, 1.1, 2.3],
                         ceilings=[0.9, 2.0, 3.6])
    _full_check(sc.points, _grid_of(sc, n_slices=9), PARAMS_ROBOT)


def test_generic_window_fallback():
    # a patch radius without a specialised instance takes the generic kernel
    sc = scenes.building(15, 40_000, side_cells=70, floors=[0.0, 2.0], ceilings=[1.8, 3.9])
    _full_check(sc.points, _grid_of(sc, n_slices=9), dict(PARAMS_ROBOT, patch_radius=3))


@pytest.mark.parametrize("seed", [21, 22])
def test_many_slices_dense_changes(seed):
    # noisy multi-level clutter: grounds and ceilings change in most slices
    rng = np.random.default_rng(seed)
    n = 200_000
    xy = rng.uniform(0, 13.0, (n, 2))
    z = rng.choice(np.arange(0, 12, 0.7), n) + rng.normal(0, 0.08, n)
    pts = np.concatenate([xy, z[:, None]], 1).astype(np.float32)
    grid = tct.Grid(0.0, 0.0, 0.1, 130, 130, 0.25, 48, 0.0, True)
    _full_check(pts, grid, dict(PARAMS_ROBOT, d_min=0.3, d_ref=0.45))


def test_long_cell_segments():
    # cells holding 20, 50, 100, 200, 300, 3000 and 9000 points (vertical
    # scan lines): the per-thread networks, the warp register sorts of 32, 64,
    # 128 and 256 heights, the block sort in shared memory and the chunked
    # block sort with merge passes all run
    rng = np.random.default_rng(31)
    base = np.stack([rng.uniform(0, 4.0, 30_000), rng.uniform(0, 4.0, 30_000),
                     rng.normal(0, 0.01, 30_000)], 1)
    cols = []
    for (x, y, m) in ((1.05, 1.05, 20), (1.55, 3.05, 50), (2.55, 3.55, 100), (3.55, 0.55, 200),
                      (2.05, 1.55, 300), (3.05, 2.55, 3000), (0.55, 3.55, 9000)):
        z = rng.uniform(0.0, 6.0, m)
        z[: m // 10] = np.round(z[: m // 10], 1)          # repeated heights
        cols.append(np.stack([np.full(m, x), np.full(m, y), z], 1))
    pts = np.concatenate([base] + cols).astype(np.float32)
    grid = tct.Grid(0.0, 0.0, 0.1, 40, 40, 0.5, 13, 0.0, True)
    _full_check(pts, grid, PARAMS_ROBOT)


def test_huge_cell_segment_time_bound():
    # one cell holding a million points (a LiDAR's invalid returns written as
    # one position, a dense pole) and one holding 20 001: the chunked block
    # sort with merge passes, O(n log^2 n), must finish well inside a second
    import time
    rng = np.random.default_rng(33)
    base = np.stack([rng.uniform(0, 2.4, 20_000), rng.uniform(0, 2.4, 20_000),
                     rng.normal(0, 0.01, 20_000)], 1)
    cols = []
    for (x, y, m) in ((1.05, 1.05, 1_000_000), (0.35, 2.05, 20_001)):
        z = rng.uniform(0.0, 6.0, m)
        z[: m // 4] = np.round(z[: m // 4], 2)           # many repeated heights
        cols.append(np.stack([np.full(m, x), np.full(m, y), z], 1))
    pts = np.concatenate([base] + cols).astype(np.float32)
    grid = tct.Grid(0.0, 0.0, 0.1, 24, 24, 0.5, 13, 0.0, True)
    g, r = _full_check(pts, grid, PARAMS_ROBOT)
    dev = torch.device("cuda")
    d = torch.from_numpy(pts).to(dev)
    ws, ground, ceil, cost, mask, keep, stats = tct.alloc_outputs(grid, len(pts), dev,
                                                                  PARAMS_ROBOT)
    tct.tct_build_evaluate(d, grid, PARAMS_ROBOT, ws, ground, ceil, cost, mask, keep, stats)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tct.tct_build_evaluate(d, grid, PARAMS_ROBOT, ws, ground, ceil, cost, mask, keep, stats)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 1.0
    np.testing.assert_array_equal(ground.cpu().numpy(), r["ground"])


@pytest.mark.parametrize("kept_only", [False, True])
def test_host_buffers_entry_point(kept_only):
    sc = scenes.building(41, 60_000, 90, 0.1, [0.0, 1.6], [1.4, 3.2], 6.0, 0.01)
    grid = tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, 9, 0.0, True)
    ref = P.gpu_build_evaluate(sc.points, grid, PARAMS_ROBOT)
    h_xyz = torch.from_numpy(sc.points).pin_memory()
    d_xyz = torch.empty_like(h_xyz, device="cuda")
    ws, g, c, cost, mask, keep, stats = tct.alloc_outputs(grid, len(sc.points), "cuda",
                                                          PARAMS_ROBOT)
    hs = [torch.full(grid.shape, -7.0).pin_memory() for _ in range(3)]
    hm = torch.full(grid.shape, 9, dtype=torch.uint8).pin_memory()
    hk = torch.zeros(grid.n_slices, dtype=torch.uint8).pin_memory()
    m = tct.tct_build_evaluate_host(h_xyz, grid, PARAMS_ROBOT, ws, d_xyz, g, c, cost, mask, keep,
                                    stats, hs[0], hs[1], hs[2], hm, hk, kept_only=kept_only)
    torch.cuda.synchronize()
    k = np.flatnonzero(ref["keep"]) if kept_only else np.arange(grid.n_slices)
    assert m == len(k) and np.array_equal(hk.numpy(), ref["keep"])
    for h, key in zip(hs + [hm], ("ground", "ceil", "cost", "mask")):
        np.testing.assert_array_equal(h.numpy()[:m], ref[key][k], err_msg=key)
    if kept_only:   # beyond the kept slices the host arrays are untouched
        assert (hs[2].numpy()[m:] == -7.0).all() and (hm.numpy()[m:] == 9).all()


def test_maximum_slice_count():
    """N = TCT_MAX_SLICES (127): the uniqueness matrix uses all four words of
    a row; clutter at many heights makes most slices differ."""
    # 36 flat 10 x 10-cell patches 0.33 m apart in height, each under a slab
    # (underside 0.6 m, top 0.7 m above its floor): every floor is the ground
    # of a few slices only, so slices up to ~123 are kept
    rng = np.random.default_rng(31)
    jj, ii = np.meshgrid(np.arange(60), np.arange(60))
    jj, ii = np.repeat(jj.ravel(), 3), np.repeat(ii.ravel(), 3)
    z = 0.33 * ((ii // 10) * 6 + jj // 10) + np.tile([0.0, 0.6, 0.7], 3600)
    z = z + rng.normal(0, 0.003, ii.size)
    pts = np.stack([(jj + rng.random(jj.size)) * 0.1, (ii + rng.random(ii.size)) * 0.1, z],
                   1).astype(np.float32)
    grid = tct.Grid(0.0, 0.0, 0.1, 60, 60, 0.1, tct.MAX_SLICES, 0.0, True)
    params = dict(PARAMS_ROBOT, d_min=0.1, d_ref=0.2, flags=tct.ALLOW_COARSE)
    g, _ = _full_check(pts, grid, params)
    kept = np.flatnonzero(g["keep"])
    assert len(kept) > 20 and kept[-2] > 96      # the fourth word of a uniqueness row in use
    with pytest.raises(tct.TctError):
        bad = tct.Grid(0.0, 0.0, 0.1, 60, 60, 0.1, tct.MAX_SLICES + 1, 0.0, True)
        P.gpu_build_evaluate(pts, bad, params)


def test_maximum_window_and_patch_radius():
    """Inflation radius 15 cells (d_inf 0.4 m, d_sm 0.45 m at 0.05 m) and p_s
    patch radius 4, the largest the ABI takes (the generic kernel); one more
    cell of either is refused."""
    sc = scenes.building(32, 50_000, side_cells=90, res=0.05, floors=[0.0, 1.2],
                         ceilings=[1.0, 2.6])
    params = dict(PARAMS_ROBOT, d_inf=0.4, d_sm=0.45, patch_radius=4)
    _full_check(sc.points, _grid_of(sc, n_slices=6), params)
    with pytest.raises(tct.TctError, match="limit"):
        P.gpu_build_evaluate(sc.points, _grid_of(sc, n_slices=6), dict(params, d_sm=0.5))
    with pytest.raises(tct.TctError):
        P.gpu_build_evaluate(sc.points, _grid_of(sc, n_slices=6), dict(params, patch_radius=5))


@pytest.mark.parametrize("stride", [3, 4])
def test_bounds_and_planned_grid(stride):
    """tct_bounds against the oracle's bounds (finite points only, the others
    counted), and the grid tct_plan_grid derives from them against the
    oracle's (Sec. III-A: footprint, z_min, plane count)."""
    sc = scenes.two_storey_building()
    pts = sc.points.copy()
    pts[::501, 0] = np.nan
    pts[7::613, 2] = np.inf
    d = torch.from_numpy(pts)
    if stride == 4:
        d = torch.cat([d, torch.zeros(len(d), 1)], 1).contiguous()
    d = d.cuda()
    out6 = torch.empty(6, device="cuda")
    stats = torch.zeros(tct.STATS_BYTES, dtype=torch.uint8, device="cuda")
    tct.tct_bounds(d, out6, stats)
    torch.cuda.synchronize()
    ref, bad = P.oracle.bounds(pts)
    got = out6.cpu().numpy()
    np.testing.assert_array_equal(got.astype(np.float64), ref)
    st = tct.stats_from(stats)
    assert st.n_nonfinite == bad > 0 and st.status & tct.DEV_NONFINITE
    g = tct.tct_plan_grid(got, 0.1, 0.5)
    og = P.oracle.derive_grid(pts, 0.1, 0.5)
    assert (g.W, g.H, g.n_slices) == (og.W, og.H, og.N)
    assert (g.x0, g.y0, g.z_min) == (og.x0, og.y0, og.z_min)
