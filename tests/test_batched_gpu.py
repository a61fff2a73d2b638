"""Batched maps (tct_build_evaluate_batched): every map of a batch must give
what the FP64 oracle gives for it alone, and exactly what the single-map
path gives; the batch must survive capture into a CUDA graph and replay."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from conftest import PARAMS_ROBOT, PARAMS_TABLE1  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import _parity as P  # noqa: E402
from paper_2403_07631_gb300 import build, scenes, tct  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    import oracle
    oracle.compile_library()


def _uneven_batch(seed=0, count=6):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(rng.integers(40, 170))
        n_fl = int(rng.integers(1, 4))
        floors, ceilings, z = [], [], 0.0
        for _ in range(n_fl):
            floors.append(round(z, 3))
            gap = float(rng.uniform(0.4, 2.5))
            ceilings.append(round(z + gap, 3))
            z += gap + 0.2
        n_pts = int(rng.integers(8_000, 60_000))
        sc = scenes.building(100 + i, n_pts, side, 0.1, floors, ceilings,
                             float(rng.uniform(5, 25)), 0.01)
        sc.n_slices = int(rng.integers(2, 16))
        out.append(sc)
    # a map without points and a single-slice map
    empty = scenes.building(200, 1000, 30, 0.1, [0.0], [2.0], 10.0, 0.01)
    empty.points = empty.points[:0]
    empty.n_slices = 3
    single = scenes.building(201, 5000, 50, 0.1, [0.0], [1.5], 10.0, 0.01)
    single.n_slices = 1
    return out + [empty, single]


def _grid(sc):
    return tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, sc.n_slices, 0.0, True)


def _maps(scs, dev="cuda"):
    return [tct.MapBuffers.allocate(torch.from_numpy(sc.points).to(dev), _grid(sc)) for sc in scs]


def _host(m):
    return {k: getattr(m, k).cpu().numpy() for k in ("ground", "ceil", "cost", "mask", "keep")}


def _single(sc, params):
    return P.gpu_build_evaluate(sc.points, _grid(sc), params)


@pytest.mark.parametrize("tuning", [None, (tct.TILE_64, 0, 4096), (tct.TILE_32, 1, 2048),
                                    (tct.TILE_64, 1, 8192), (tct.TILE_64x56, 0, 4096),
                                    (tct.TILE_64x40, 0, 4096), (tct.TILE_128x56, 0, 4096)])
def test_batch_matches_oracle_and_single_path(tuning):
    scs = _uneven_batch()
    maps = _maps(scs)
    ws = torch.empty(tct.tct_workspace_bytes_batched(maps, PARAMS_ROBOT), dtype=torch.uint8,
                     device="cuda")
    t = None if tuning is None else tct.TctTuning(*tuning, 0)
    tct.tct_build_evaluate_batched(maps, PARAMS_ROBOT, ws, t)
    torch.cuda.synchronize()
    for sc, m in zip(scs, maps):
        got = _host(m)
        one = _single(sc, PARAMS_ROBOT)
        for key in ("ground", "ceil", "cost", "mask", "keep"):
            np.testing.assert_array_equal(got[key], one[key], err_msg=key)
        ref = P.oracle_all(sc.points, _grid(sc), PARAMS_ROBOT)
        P.assert_equal_layers(got["ground"], ref["ground"], "ground")
        P.assert_equal_layers(got["ceil"], ref["ceil"], "ceiling")
        P.assert_costs(got["cost"], ref["cost"], ref["fragile"])
        P.assert_masks(got["mask"], ref["mask"], ref["fragile"])
        P.assert_keep(got["keep"], got["ground"], got["cost"], ref, PARAMS_ROBOT)
        st = tct.stats_from(m.stats)
        assert st.n_points == len(sc.points) and st.n_dropped == ref["dropped"]
        assert st.n_kept == int(got["keep"].sum())


def test_batch_graph_capture_and_replay_with_new_points():
    scs = _uneven_batch(seed=3, count=4)
    maps = _maps(scs)
    params = dict(PARAMS_TABLE1, flags=tct.KEEP_ENDS)
    ws = torch.empty(tct.tct_workspace_bytes_batched(maps, params), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        tct.tct_build_evaluate_batched(maps, params, ws)          # first call before capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        tct.tct_build_evaluate_batched(maps, params, ws)
    # new clouds of the same sizes into the captured buffers, then replay
    new = []
    for i, (sc, m) in enumerate(zip(scs, maps)):
        sc2 = scenes.building(900 + i, len(sc.points), sc.W, 0.1, [0.0, 1.0], [0.8, 2.3], 12.0,
                              0.01)
        sc2.n_slices = sc.n_slices
        m.xyz.copy_(torch.from_numpy(sc2.points[: len(sc.points)]))
        new.append(sc2)
    g.replay()
    torch.cuda.synchronize()
    for sc2, sc, m in zip(new, scs, maps):
        pts = sc2.points[: len(sc.points)]
        one = P.gpu_build_evaluate(pts, _grid(sc), params)
        got = _host(m)
        for key in ("ground", "ceil", "cost", "mask", "keep"):
            np.testing.assert_array_equal(got[key], one[key], err_msg=key)


def test_autotune_then_run():
    scs = _uneven_batch(seed=5, count=5)
    maps = _maps(scs)
    ws = torch.empty(tct.tct_workspace_bytes_batched(maps, PARAMS_ROBOT), dtype=torch.uint8,
                     device="cuda")
    t = tct.tct_autotune_batched(maps, PARAMS_ROBOT, ws)
    assert t.tile in (tct.TILE_64, tct.TILE_32, tct.TILE_64x56, tct.TILE_64x40, tct.TILE_128x56)
    assert t.points_per_block % 4 == 0
    tct.tct_build_evaluate_batched(maps, PARAMS_ROBOT, ws, t)
    torch.cuda.synchronize()
    for sc, m in zip(scs, maps):
        one = _single(sc, PARAMS_ROBOT)
        np.testing.assert_array_equal(m.cost.cpu().numpy(), one["cost"])
        np.testing.assert_array_equal(m.keep.cpu().numpy(), one["keep"])


def test_batch_refusals():
    scs = _uneven_batch(seed=7, count=2)
    maps = _maps(scs)
    ws = torch.empty(tct.tct_workspace_bytes_batched(maps, PARAMS_ROBOT), dtype=torch.uint8,
                     device="cuda")
    with pytest.raises(tct.TctError, match="workspace"):
        tct.tct_build_evaluate_batched(maps, PARAMS_ROBOT, ws[:1024])
    with pytest.raises(tct.TctError, match="limit"):
        tct.tct_build_evaluate_batched(maps * 33, PARAMS_ROBOT, ws)      # 66 maps


@pytest.mark.parametrize("params", [PARAMS_ROBOT, dict(PARAMS_ROBOT, patch_radius=3)])
def test_batch_mixed_resolutions_and_generic_radii(params):
    """Maps at 0.1 m and 0.05 m in one batch (a window each), and a patch
    radius without a specialised kernel: the batch runs map after map and
    every map equals the single-map call and the oracle."""
    scs = _uneven_batch(seed=9, count=2)
    fine = scenes.building(310, 30_000, 80, 0.05, [0.0, 1.1], [0.9, 2.4], 8.0, 0.01)
    fine.n_slices = 5
    scs.append(fine)
    maps = _maps(scs)
    ws = torch.empty(tct.tct_workspace_bytes_batched(maps, params), dtype=torch.uint8,
                     device="cuda")
    tct.tct_build_evaluate_batched(maps, params, ws)
    torch.cuda.synchronize()
    for sc, m in zip(scs, maps):
        got = _host(m)
        one = _single(sc, params)
        for key in ("ground", "ceil", "cost", "mask", "keep"):
            np.testing.assert_array_equal(got[key], one[key], err_msg=key)
        ref = P.oracle_all(sc.points, _grid(sc), params)
        P.assert_costs(got["cost"], ref["cost"], ref["fragile"])
        P.assert_masks(got["mask"], ref["mask"], ref["fragile"])
        P.assert_keep(got["keep"], got["ground"], got["cost"], ref, params)


@pytest.mark.parametrize("res,params", [(0.1, PARAMS_TABLE1), (0.05, PARAMS_ROBOT)])
@pytest.mark.parametrize("tile", [tct.TILE_64x56, tct.TILE_64x40, tct.TILE_64, tct.TILE_32,
                                  tct.TILE_128x56])
def test_batch_other_window_radii(res, params, tile):
    """The radius-4 (Table I, 0.1 m) and radius-12 (0.05 m) instances in every
    tile shape, on maps with ragged last tiles."""
    rng = np.random.default_rng(11)
    scs = []
    for i, side in enumerate((70, 131, 97)):
        sc = scenes.building(300 + i, int(rng.integers(20_000, 60_000)), side, res, [0.0, 1.1],
                             [0.9, 2.4], 8.0, 0.01)
        sc.n_slices = int(rng.integers(3, 9))
        scs.append(sc)
    maps = _maps(scs)
    ws = torch.empty(tct.tct_workspace_bytes_batched(maps, params), dtype=torch.uint8,
                     device="cuda")
    tct.tct_build_evaluate_batched(maps, params, ws, tct.TctTuning(tile, 0, 4096, 0))
    torch.cuda.synchronize()
    for sc, m in zip(scs, maps):
        got = _host(m)
        ref = P.oracle_all(sc.points, _grid(sc), params)
        P.assert_equal_layers(got["ground"], ref["ground"], "ground")
        P.assert_costs(got["cost"], ref["cost"], ref["fragile"])
        P.assert_masks(got["mask"], ref["mask"], ref["fragile"])
        P.assert_keep(got["keep"], got["ground"], got["cost"], ref, params)


def test_build_then_evaluate_batched_equal_single_calls():
    """The construction-only and evaluation-only batched calls give, map by
    map, exactly what tct_build and tct_evaluate give on each map alone."""
    scs = _uneven_batch(seed=13, count=5)
    maps = _maps(scs)
    ws = torch.empty(tct.tct_workspace_bytes_batched(maps, PARAMS_ROBOT), dtype=torch.uint8,
                     device="cuda")
    tct.tct_build_batched(maps, ws, tct.TctTuning(tct.TILE_AUTO, 0, 2048, 0))
    torch.cuda.synchronize()
    for sc, m in zip(scs, maps):
        g, c, st = P.gpu_build(sc.points, _grid(sc))
        np.testing.assert_array_equal(m.ground.cpu().numpy(), g)
        np.testing.assert_array_equal(m.ceil.cpu().numpy(), c)
        mst = tct.stats_from(m.stats)
        assert (mst.n_points, mst.n_dropped, mst.z_min, mst.z_max) == \
               (st.n_points, st.n_dropped, st.z_min, st.z_max)
    # the evaluation reads no plane heights: a map without points (z_min = inf) gets 0
    z_mins = [float(np.nan_to_num(tct.stats_from(m.stats).z_min, posinf=0.0)) for m in maps]
    ws2 = torch.empty(tct.tct_workspace_bytes_evaluate_batched(maps, PARAMS_ROBOT),
                      dtype=torch.uint8, device="cuda")
    tct.tct_evaluate_batched(maps, PARAMS_ROBOT, ws2)
    torch.cuda.synchronize()
    for sc, m, z_min in zip(scs, maps, z_mins):
        g = m.ground.cpu().numpy()
        grid = tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, sc.n_slices, z_min, False)
        one = P.gpu_evaluate(g, m.ceil.cpu().numpy(), grid, PARAMS_ROBOT, aux=False)
        np.testing.assert_array_equal(m.cost.cpu().numpy(), one["cost"])
        np.testing.assert_array_equal(m.mask.cpu().numpy(), one["mask"])
        np.testing.assert_array_equal(m.keep.cpu().numpy(), one["keep"])


def _scan_lines(seed, lines):
    """A 40 x 40 cloud with vertical scan lines: cells holding the given numbers of points."""
    rng = np.random.default_rng(seed)
    base = np.stack([rng.uniform(0, 4.0, 20_000), rng.uniform(0, 4.0, 20_000),
                     rng.normal(0, 0.01, 20_000)], 1)
    cols = []
    for (x, y, m) in lines:
        z = rng.uniform(0.0, 6.0, m)
        z[: m // 10] = np.round(z[: m // 10], 1)          # repeated heights
        cols.append(np.stack([np.full(m, x), np.full(m, y), z], 1))
    return np.concatenate([base] + cols).astype(np.float32)


def test_batch_long_segments_in_every_sort_class():
    """Cells of 20 to 9000 points in two maps of one batch go through the warp
    sorts (queued from the front of the shared list) and the block and rank
    sorts (queued from its back): every map's layers equal the single-map
    path's and the oracle's."""
    pts = [_scan_lines(41, ((1.05, 1.05, 20), (1.55, 3.05, 50), (2.55, 3.55, 100),
                            (3.55, 0.55, 200), (2.05, 1.55, 300), (3.05, 2.55, 3000))),
           _scan_lines(42, ((0.55, 3.55, 9000), (1.25, 0.35, 700), (3.35, 1.85, 130)))]
    grids = [tct.Grid(0.0, 0.0, 0.1, 40, 40, 0.5, 13, 0.0, True) for _ in pts]
    maps = [tct.MapBuffers.allocate(torch.from_numpy(p).cuda(), g) for p, g in zip(pts, grids)]
    ws = torch.empty(tct.tct_workspace_bytes_batched(maps, PARAMS_ROBOT), dtype=torch.uint8,
                     device="cuda")
    tct.tct_build_evaluate_batched(maps, PARAMS_ROBOT, ws, None)
    torch.cuda.synchronize()
    for p, g, m in zip(pts, grids, maps):
        got = _host(m)
        one = P.gpu_build_evaluate(p, g, PARAMS_ROBOT)
        for key in ("ground", "ceil", "cost", "mask", "keep"):
            np.testing.assert_array_equal(got[key], one[key], err_msg=key)
        ref = P.oracle_all(p, g, PARAMS_ROBOT)
        P.assert_equal_layers(got["ground"], ref["ground"], "ground")
        P.assert_equal_layers(got["ceil"], ref["ceil"], "ceiling")
