"""Pins of the oracle's tomogram construction (Sec. III-A, the construction part of Alg. 1).

Nothing here re-types the oracle's loops: expected values are enumerated by
hand, follow from closed forms, are checked as invariants, or come from an
independent numpy formulation (sort by cell + binary search) on tiny inputs.
"""
import numpy as np
import pytest

from paper_2403_07631_gb300 import scenes

INF = np.inf


def test_hand_enumerated_cloud(oracle_mod):
    # 3x3 grid of 1 m cells, planes at z_min + (k+1) d_s = 1, 2, 3, 4.
    pts = np.array([
        [0.5, 0.5, 0.2],    # cell (0,0)
        [0.5, 0.5, 2.5],    # cell (0,0)
        [0.5, 0.5, 1.0],    # cell (0,0), exactly on plane 0: lower group
        [2.5, 0.5, 3.7],    # row 0, column 2 (x selects the column)
        [0.5, 2.5, -0.0],   # row 2, column 0; -0 is stored as +0
        [1.5, 1.5, 5.0],    # cell (1,1), above every plane: ceiling only
        [3.5, 0.5, 1.0],    # x beyond the last column: dropped
        [-0.25, 0.5, 1.0],  # x before the first column: dropped
    ], np.float32)
    g = oracle_mod.Grid(0.0, 0.0, 1.0, 3, 3, 1.0, 0.0, 4)
    eG, eC, g2, dropped, bad = oracle_mod.build(pts, g, zmin_from_data=False)
    assert dropped == 2 and bad == 0
    expG = np.full((4, 3, 3), -INF, np.float32)
    expC = np.full((4, 3, 3), INF, np.float32)
    expG[:, 0, 0] = [1.0, 1.0, 2.5, 2.5]
    expC[:, 0, 0] = [2.5, 2.5, INF, INF]
    expG[:, 0, 2] = [-INF, -INF, -INF, 3.7]
    expC[:, 0, 2] = [3.7, 3.7, 3.7, INF]
    expG[:, 2, 0] = 0.0
    expC[:, 1, 1] = 5.0
    np.testing.assert_array_equal(eG, expG)
    np.testing.assert_array_equal(eC, expC)
    assert not np.signbit(eG[0, 2, 0])


def test_plane_heights_first_plane_above_lowest_point(oracle_mod):
    # Sec. III-A: the first plane is d_s above the lowest point; equidistant.
    g = oracle_mod.Grid(0.0, 0.0, 0.1, 4, 4, 0.5, -0.0372, 12)
    h = oracle_mod.plane_heights(g).astype(np.float64)
    exact = -0.0372 + 0.5 * np.arange(1, 13)
    assert np.all(np.abs(h - np.float32(-0.0372).astype(np.float64) - 0.5 * np.arange(1, 13)) <=
                  np.spacing(np.abs(h).astype(np.float32)) * 0.5 + 1e-12)
    assert np.allclose(h, exact, atol=1e-6)


def test_rasterize_matches_ieee_float32(oracle_mod):
    # j = floor(fl32(fl32(x - x0) / r_g)); numpy float32 arithmetic is IEEE
    # single precision, an independent check of the oracle's double route.
    rng = np.random.default_rng(11)
    W = H = 50
    x0, y0, res = np.float32(-1.37), np.float32(2.11), np.float32(0.1)
    xy = rng.uniform(-1.5, 4.0, (4000, 2)).astype(np.float32)
    xy[:, 1] += np.float32(3.5)
    # points placed exactly on cell boundaries
    xy[:200, 0] = x0 + np.float32(0.1) * rng.integers(0, 50, 200).astype(np.float32)
    pts = np.concatenate([xy, np.full((len(xy), 1), 0.25, np.float32)], 1)
    g = oracle_mod.Grid(float(x0), float(y0), float(res), W, H, 0.5, 0.0, 2)
    eG, _, _, dropped, _ = oracle_mod.build(pts, g, zmin_from_data=False)
    u = np.floor((xy[:, 0] - x0) / res)
    v = np.floor((xy[:, 1] - y0) / res)
    on = (u >= 0) & (u < W) & (v >= 0) & (v < H)
    occupied = np.zeros((H, W), bool)
    occupied[v[on].astype(int), u[on].astype(int)] = True
    assert dropped == int((~on).sum())
    np.testing.assert_array_equal(eG[0] == np.float32(0.25), occupied)


def _numpy_sorted_reference(pts, x0, y0, res, W, H, h):
    """Independent formulation: sort each cell's z, binary-search every plane."""
    u = np.floor((pts[:, 0] - np.float32(x0)) / np.float32(res))
    v = np.floor((pts[:, 1] - np.float32(y0)) / np.float32(res))
    on = (u >= 0) & (u < W) & (v >= 0) & (v < H)
    cell = (v[on] * W + u[on]).astype(np.int64)
    z = pts[on, 2]
    order = np.lexsort((z, cell))
    cell, z = cell[order], z[order]
    G = np.full((len(h), H * W), -np.inf, np.float32)
    C = np.full((len(h), H * W), np.inf, np.float32)
    starts = np.searchsorted(cell, np.arange(H * W))
    ends = np.searchsorted(cell, np.arange(H * W), side="right")
    for c in np.nonzero(ends > starts)[0]:
        zc = z[starts[c]:ends[c]]
        n_low = np.searchsorted(zc, h, side="right")   # count of z <= h_k
        for k, m in enumerate(n_low):
            if m > 0:
                G[k, c] = zc[m - 1]
            if m < len(zc):
                C[k, c] = zc[m]
    return G.reshape(len(h), H, W), C.reshape(len(h), H, W)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_clouds_against_sorted_reference(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = 300
    pts = np.stack([rng.uniform(0, 0.6, n), rng.uniform(0, 0.5, n),
                    rng.choice([0.0, 0.25, 0.5, 1.0], n) + rng.normal(0, 0.1, n)], 1).astype(np.float32)
    g = oracle_mod.Grid(0.0, 0.0, 0.1, 6, 5, 0.25, 0.0, 8)
    eG, eC, g2, dropped, _ = oracle_mod.build(pts, g, zmin_from_data=True)
    h = oracle_mod.plane_heights(g2)
    assert g2.z_min == pts[:, 2].min()
    G, C = _numpy_sorted_reference(pts, 0.0, 0.0, 0.1, 6, 5, h)
    np.testing.assert_array_equal(eG, G)
    np.testing.assert_array_equal(eC, C)


def test_invariants_on_building(oracle_mod):
    sc = scenes.building(7, 20_000, side_cells=40, floors=[0.0, 1.5], ceilings=[1.3, 2.9])
    g = oracle_mod.derive_grid(sc.points, 0.1, 0.5)
    eG, eC, g2, _, _ = oracle_mod.build(sc.points, g, zmin_from_data=True)
    h = oracle_mod.plane_heights(g2)[:, None, None]
    vg = eG > -np.inf
    vc = eC < np.inf
    # ground at or below its plane, ceiling strictly above it
    assert np.all(eG[vg] <= np.broadcast_to(h, eG.shape)[vg])
    assert np.all(eC[vc] > np.broadcast_to(h, eC.shape)[vc])
    # both layers are non-decreasing from slice to slice
    assert np.all(eG[1:] >= eG[:-1])
    assert np.all(eC[1:] >= eC[:-1])
    # every valid elevation is one of the input heights
    zs = set(np.unique(sc.points[:, 2]).tolist())
    assert set(np.unique(eG[vg]).tolist()) <= zs
    assert set(np.unique(eC[vc]).tolist()) <= zs


def test_flat_floor_under_ceiling(oracle_mod):
    # floor a under ceiling b: every plane h_k in [a, b) sees ground a, ceiling b
    a, b = 0.25, 1.75
    xs = (np.arange(8) + 0.5) * 0.1
    X, Y = np.meshgrid(xs, xs)
    fl = np.stack([X.ravel(), Y.ravel(), np.full(64, a)], 1)
    ce = np.stack([X.ravel(), Y.ravel(), np.full(64, b)], 1)
    pts = np.concatenate([fl, ce]).astype(np.float32)
    g = oracle_mod.Grid(0.0, 0.0, 0.1, 8, 8, 0.5, 0.0, 4)       # planes 0.5, 1, 1.5, 2
    eG, eC, _, _, _ = oracle_mod.build(pts, g, zmin_from_data=False)
    for k, hk in enumerate([0.5, 1.0, 1.5]):
        assert a <= hk < b
        assert np.all(eG[k] == np.float32(a)) and np.all(eC[k] == np.float32(b))
    assert np.all(eG[3] == np.float32(b)) and np.all(eC[3] == np.inf)


def test_coverage_rule_ds_le_dmin(oracle_mod):
    # Sec. III-A: with d_s <= d_min every floor/ceiling gap of at least d_min
    # is cut by some plane, so some slice shows both surfaces together.
    rng = np.random.default_rng(5)
    d_s = 0.5
    for _ in range(200):
        a = rng.uniform(0, 3)
        b = a + rng.uniform(0.5, 1.5)
        pts = np.array([[0.05, 0.05, 0.0], [0.05, 0.05, a], [0.05, 0.05, b]], np.float32)
        g = oracle_mod.Grid(0.0, 0.0, 0.1, 1, 1, d_s, 0.0, 12)
        eG, eC, _, _, _ = oracle_mod.build(pts, g, zmin_from_data=False)
        seen = (eG[:, 0, 0] == np.float32(a)) & (eC[:, 0, 0] == np.float32(b))
        assert seen.any()


def test_derive_grid_two_storey_building(oracle_mod):
    sc = scenes.two_storey_building()
    g = oracle_mod.derive_grid(sc.points, 0.1, 0.5)
    zmin, zmax = sc.points[:, 2].min(), sc.points[:, 2].max()
    assert g.z_min == zmin
    assert g.N == 12
    h = oracle_mod.plane_heights(g)
    assert h[-1] >= zmax > h[-2]
    assert g.x0 == sc.points[:, 0].min() and g.y0 == sc.points[:, 1].min()


@pytest.mark.parametrize("xmax,ymax,W,H", [
    (2.0, 0.75, 9, 4),          # maxima exactly on a cell edge: they open cells 8 and 3
    (1.99, 0.7499, 8, 3),       # just inside: the last cells are 7 and 2
    (0.25, 0.0, 2, 1),          # one edge past the origin; a line of points along x
])
def test_derive_grid_width_height_at_cell_edges(oracle_mod, xmax, ymax, W, H):
    """Sec. III-A: the grid starts at the cloud's minimum and its last column
    and row hold the maximum.  With r_g = 0.25 (exact in binary) the cell of
    a coordinate is floor(x / 0.25) by hand: x = 2.0 lies on the left edge of
    cell 8, so W = 9; x = 1.99 lies in cell 7, so W = 8."""
    pts = np.array([[0.0, 0.0, 0.0], [xmax, ymax, 0.3], [xmax / 2, ymax / 3, 0.1]], np.float32)
    g = oracle_mod.derive_grid(pts, 0.25, 0.5)
    assert (g.x0, g.y0) == (0.0, 0.0)
    assert (g.W, g.H) == (W, H)
    # every point of the cloud lands on the grid, the maximum in the last cell
    eG, _, _, dropped, _ = oracle_mod.build(pts, g, zmin_from_data=True)
    assert dropped == 0
    assert eG[0, H - 1, W - 1] == np.float32(0.3)
    # shifted origin: the same widths with the cloud moved by (-1.5, +2.25)
    g2 = oracle_mod.derive_grid(pts + np.array([-1.5, 2.25, 0.0], np.float32), 0.25, 0.5)
    assert (g2.x0, g2.y0, g2.W, g2.H) == (-1.5, 2.25, W, H)


def test_nonfinite_points_are_rejected(oracle_mod):
    pts = np.array([[0.05, 0.05, 0.0], [np.nan, 0.05, 1.0], [0.05, np.inf, 1.0],
                    [0.05, 0.05, -np.inf]], np.float32)
    g = oracle_mod.Grid(0.0, 0.0, 0.1, 2, 2, 0.5, 0.0, 2)
    eG, eC, _, dropped, bad = oracle_mod.build(pts, g, zmin_from_data=False)
    assert bad == 3 and dropped == 0
    assert eG[0, 0, 0] == 0.0 and np.all(eC == np.inf)


def test_bounds_against_numpy(oracle_mod):
    """The cloud bounds are numpy's min / max over the finite points, with the
    non-finite ones counted (and -0 read as +0, which compares equal)."""
    rng = np.random.default_rng(12)
    pts = rng.normal(0, 5, (5000, 3)).astype(np.float32)
    pts[::97, 1] = np.nan
    pts[3::101, 2] = np.inf
    pts[5::89, 0] = -np.inf
    b, bad = oracle_mod.bounds(pts)
    ok = np.isfinite(pts).all(1)
    assert bad == int((~ok).sum())
    np.testing.assert_array_equal(b[:3], pts[ok].min(0).astype(np.float64))
    np.testing.assert_array_equal(b[3:], pts[ok].max(0).astype(np.float64))
