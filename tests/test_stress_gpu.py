"""Stress workload at full size: 60M points of cave terrain, a 4000 x 4000
grid at 0.05 m, 80 slices (inflation radius 12 cells), built and evaluated
in one call, then a batch of 4096 paths x 512 waypoints queried forward and
backward through the sampler.

The FP64 oracle cannot evaluate 1.28G slice-cells in a test, so parity is
checked on seeded windows of the map, each cut out with every point that
falls into it and a halo of 1 + R_p + R_K cells (the reach of one cost
through Eq. 2-6: gradient stencil, p_s patch, inflation window).  Points are
rasterized on the full grid and moved to the centres of the same cells of
the window's own grid, which changes no elevation (Sec. III-A bins by cell
and z only).  Elevations are compared bit-exact over window and halo, costs
and masks on the window's core, with the tolerances of the other parity
tests.  The keep flags are a decision over the whole map: they are checked
against the oracle's chain (Sec. III-C, Eq. 7-9) on the GPU's own layers,
and the per-slice statistics against the layers.  Query values and
gradients are compared with the oracle on a seeded subset of waypoints.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from conftest import PARAMS_ROBOT  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import _parity as P  # noqa: E402
import _windows as W  # noqa: E402
import oracle  # noqa: E402
from paper_2403_07631_gb300 import build, scenes, tct  # noqa: E402

N_WINDOWS = 64
CORE = 64


@pytest.fixture(scope="module")
def stress():
    build.build()
    oracle.compile_library()
    sc = scenes.cave_terrain()
    grid = tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, sc.n_slices, 0.0, True)
    pts = torch.from_numpy(sc.points).cuda()
    ws, ground, ceil, cost, mask, keep, stats = tct.alloc_outputs(grid, len(sc.points), "cuda",
                                                                  PARAMS_ROBOT)
    tct.tct_build_evaluate(pts, grid, PARAMS_ROBOT, ws, ground, ceil, cost, mask, keep, stats)
    torch.cuda.synchronize()
    del ws, pts
    bounds, _ = oracle.bounds(sc.points)
    z_min = float(np.float32(bounds[2]))
    return dict(sc=sc, grid=grid, z_min=z_min, ground=ground, ceil=ceil, cost=cost, mask=mask,
                keep=keep.cpu().numpy(), stats=tct.stats_from(stats))


def _windows(sc, seed=11):
    """Core windows: seeded random ones, one over each grid corner (the ragged
    last tile included) and some centred on cave tunnels (several layers)."""
    rng = np.random.default_rng(seed)
    out = [(0, 0), (sc.H - CORE, sc.W - CORE), (0, sc.W - CORE), (sc.H - CORE, 0)]
    for cx, cy in sc.meta["tunnel_points"][:20]:
        i = int(cy / sc.res) - CORE // 2
        j = int(cx / sc.res) - CORE // 2
        out.append((min(max(i, 0), sc.H - CORE), min(max(j, 0), sc.W - CORE)))
    while len(out) < N_WINDOWS:
        out.append((int(rng.integers(0, sc.H - CORE)), int(rng.integers(0, sc.W - CORE))))
    return out


def test_stress_windows_match_oracle(stress):
    sc = stress["sc"]
    hal = W.halo(PARAMS_ROBOT, sc.res)
    ij = W.cells(sc.points, sc.x0, sc.y0, sc.res)
    n_cells = n_fragile = n_multi = 0
    for (ci, cj) in _windows(sc):
        box, core = W.window_bounds(ci, cj, CORE, hal, sc.H, sc.W)
        eG, eC, cT, mask, frag = W.oracle_window(sc.points, ij, box, sc.res, sc.d_s,
                                                 stress["z_min"], sc.n_slices, PARAMS_ROBOT)
        i_lo, i_hi, j_lo, j_hi = box
        win = (slice(None), slice(i_lo, i_hi), slice(j_lo, j_hi))
        where = f"window rows {i_lo}:{i_hi} cols {j_lo}:{j_hi}"
        P.assert_equal_layers(stress["ground"][win].cpu().numpy(), eG, "ground, " + where)
        P.assert_equal_layers(stress["ceil"][win].cpu().numpy(), eC, "ceiling, " + where)
        P.assert_costs(stress["cost"][win].cpu().numpy()[core], cT[core], frag[core],
                         max_fragile=None)
        P.assert_masks(stress["mask"][win].cpu().numpy()[core], mask[core], frag[core])
        n_cells += frag[core].size
        n_fragile += int((frag[core] != 0).sum())
        g = eG[core]
        fin = np.isfinite(g)
        with np.errstate(invalid="ignore"):  # -inf - -inf where both slices lack ground
            rises = (np.diff(g, axis=0) > 0) & fin[1:] & fin[:-1]
        n_multi += int(rises.any(0).sum())
    assert n_fragile <= 1e-3 * n_cells
    assert n_multi > 0, "no window saw more than one ground layer"


def test_stress_keep_flags_and_stats(stress):
    sc = stress["sc"]
    eG = stress["ground"].cpu().numpy()
    cT = stress["cost"].cpu().numpy().astype(np.float64)
    c_b = float(np.float32(PARAMS_ROBOT["c_b"]))
    keep, _ = oracle.simplify(eG, cT, c_b, None)
    np.testing.assert_array_equal(stress["keep"], keep)
    st = stress["stats"]
    assert st.n_points == len(sc.points)
    assert st.n_kept == int(keep.sum())
    i, j = W.cells(sc.points, sc.x0, sc.y0, sc.res)
    inside = (i >= 0) & (i < sc.H) & (j >= 0) & (j < sc.W)
    assert st.n_dropped == int((~inside).sum())
    valid = np.isfinite(eG).reshape(sc.n_slices, -1).sum(1)
    trav = (cT < c_b).reshape(sc.n_slices, -1).sum(1)
    np.testing.assert_array_equal(np.array(st.valid_cells[: sc.n_slices]), valid)
    np.testing.assert_array_equal(np.array(st.trav_cells[: sc.n_slices]), trav)
    assert keep.sum() >= 2 and trav.max() > 0


def _paths(sc, trav, n_paths, length, seed=4):
    """Straight lines between random traversable cells of one slice with
    N(0, 0.2 m) noise on the inner waypoints; the slice is the start's."""
    rng = np.random.default_rng(seed)
    k_of = np.flatnonzero(trav.reshape(sc.n_slices, -1).any(1))
    ks = rng.choice(k_of, n_paths)
    ends = np.empty((n_paths, 2), np.int64)
    for k in np.unique(ks):
        cells = np.flatnonzero(trav[k].reshape(-1))
        ends[ks == k] = rng.choice(cells, (int((ks == k).sum()), 2))
    centre = lambda c: np.stack([(c % sc.W + 0.5) * sc.res, (c // sc.W + 0.5) * sc.res], -1)
    t = np.linspace(0.0, 1.0, length)[None, :, None]
    xy = centre(ends[:, :1]) * (1 - t) + centre(ends[:, 1:]) * t
    xy[:, 1:-1] += rng.normal(0.0, 0.2, (n_paths, length - 2, 2))
    xy = xy.astype(np.float32)
    sl = np.broadcast_to(ks[:, None], (n_paths, length)).astype(np.int32)
    return xy, sl


def test_stress_path_queries(stress):
    sc, grid = stress["sc"], stress["grid"]
    c_b = float(np.float32(PARAMS_ROBOT["c_b"]))
    cost = stress["cost"].cpu().numpy()
    ground = stress["ground"].cpu().numpy()
    xy, sl = _paths(sc, cost < c_b, 4096, 512)
    gridz = tct.Grid(grid.x0, grid.y0, grid.res, grid.W, grid.H, grid.d_s, grid.n_slices,
                     stress["z_min"], False)
    d_xy = torch.from_numpy(xy.reshape(-1, 2)).cuda().requires_grad_(True)
    d_sl = torch.from_numpy(sl.reshape(-1).copy()).cuda()
    c, e = tct.sample_cost(d_xy, d_sl, stress["cost"], stress["ground"], gridz)
    (c.sum() + e.sum()).backward()
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    pick = rng.choice(len(d_sl), 50_000, replace=False)
    q, s = xy.reshape(-1, 2)[pick], sl.reshape(-1)[pick]
    og = oracle.Grid(grid.x0, grid.y0, grid.res, grid.W, grid.H, grid.d_s, stress["z_min"],
                     grid.n_slices)
    rc, gc = oracle.sample(og, cost, q, s)
    re, ge = oracle.sample(og, ground, q, s, is_ground=True)
    zmax = float(np.abs(ground[np.isfinite(ground)]).max())
    rt = 1e-5
    for got, ref, scale, what in ((c.detach().cpu().numpy()[pick], rc, c_b, "cost"),
                                  (e.detach().cpu().numpy()[pick], re, zmax, "elevation"),
                                  (d_xy.grad.cpu().numpy()[pick], gc + ge,
                                   (c_b + zmax) / grid.res, "gradient")):
        err = np.abs(got.astype(np.float64) - ref)
        lim = rt * np.maximum(np.abs(ref), scale)
        bad = ~(err <= lim)
        assert not bad.any(), f"{what}: {int(bad.sum())} out of tolerance, max err {err[bad].max()}"
