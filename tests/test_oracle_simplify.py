"""Pins of the oracle's tomogram simplification (Sec. III-C, Eq. 7-9).

Expected keep flags are worked out by hand on constructed scenes (the
three-slice ramp-and-overhang scene of Fig. 2, identical neighbouring
slices), and the chain is checked against the invariant it guarantees:
every traversable cell of a removed slice is represented by a kept slice
with the same ground elevation and no higher cost.
"""
import numpy as np
import pytest

from conftest import PARAMS_ROBOT
from paper_2403_07631_gb300 import scenes


def _surface(x0, x1, y0, y1, z, res=0.1):
    """One point at the centre of every cell of [x0,x1) x [y0,y1)."""
    xs = np.arange(round(x0 / res), round(x1 / res)) * res + res / 2
    ys = np.arange(round(y0 / res), round(y1 / res)) * res + res / 2
    X, Y = np.meshgrid(xs, ys)
    Z = z(X, Y) if callable(z) else np.full_like(X, z)
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)


def fig2_scene():
    """Regions along x, 4 m wide in y:
    A [0,4): floor 0 under a slab (underside 1.1, top 1.2)
    B [4,8): ramp from 0 up to 1.2 (0.3 m/m, gentle), open above
    C [8,10): upper floor 1.2
    D [10,14): floor 0 with a table (underside 0.75, top 0.8) on [11,13)x[1,3)
    Planes at 0.5, 1.0, 1.5.  Slice 0 sees the floor under the table (unique
    against slice 1, where the table top is the ground); slice 1 adds only the
    middle of the ramp and the table top, both identical in slice 2; slice 2
    sees the slab top over A.  The middle slice is therefore redundant, as in
    the caption of Fig. 2."""
    parts = [
        _surface(0, 4, 0, 4, 0.0), _surface(0, 4, 0, 4, 1.1), _surface(0, 4, 0, 4, 1.2),
        _surface(4, 8, 0, 4, lambda x, y: 0.3 * (x - 4.0)),
        _surface(8, 10, 0, 4, 1.2),
        _surface(10, 14, 0, 4, 0.0),
        _surface(11, 13, 1, 3, 0.75), _surface(11, 13, 1, 3, 0.8),
    ]
    return np.concatenate(parts).astype(np.float32)


def test_fig2_middle_slice_removed(oracle_mod):
    pts = fig2_scene()
    g = oracle_mod.Grid(0.0, 0.0, 0.1, 140, 40, 0.5, 0.0, 3)
    eG, eC, g, _, _ = oracle_mod.build(pts, g, zmin_from_data=False)
    cT, mask, frag, = oracle_mod.evaluate(g, PARAMS_ROBOT, eG, eC)
    keep, robust = oracle_mod.simplify(eG, cT, 50.0, frag)
    assert robust
    assert keep.tolist() == [1, 0, 1]
    # the removed slice's traversable cells all reappear in the kept ones
    _assert_coverage(eG, cT, keep)


def _assert_coverage(eG, cT, keep, c_b=50.0):
    kept = np.nonzero(keep)[0]
    N = len(keep)
    for k in range(N):
        trav = cT[k] < c_b
        covered = np.zeros_like(trav)
        for q in kept:
            covered |= (eG[q] == eG[k]) & (cT[q] <= cT[k])
        assert np.all(covered[trav]), f"slice {k} has unrepresented traversable cells"


def test_identical_slices_keep_one(oracle_mod):
    # Two identical floors in slices 0 and 1 and an upper floor in slice 2.
    # Testing every slice against its original neighbours (the literal reading
    # of the removal loop of Alg. 1) would drop both floor slices; the sequential chain
    # of Sec. III-C keeps exactly one of them.
    N, H, W = 3, 6, 6
    eG = np.zeros((N, H, W), np.float32)
    eG[2] = 3.0
    cT = np.ones((N, H, W))
    keep, robust = oracle_mod.simplify(eG, cT, 50.0)
    assert keep.tolist() == [0, 1, 1] and robust
    _assert_coverage(eG, cT, keep)


def test_lower_cost_makes_cell_unique(oracle_mod):
    # Same ground in all slices; slice 1 is cheaper at one cell (its ceiling
    # rose), slice 2 dearer again.  Slice 0 has nothing unique (Eq. 9 fails
    # everywhere: c_0 >= c_1); slice 1 passes Eq. 8 vacuously and Eq. 9 at
    # that cell (c_1 < c_2); slice 2 is no cheaper than the kept slice 1
    # anywhere, so Eq. 8 fails and slice 1 represents it.
    N, H, W = 3, 5, 5
    eG = np.zeros((N, H, W), np.float32)
    cT = np.full((N, H, W), 2.0)
    cT[1, 2, 2] = 1.0
    keep, robust = oracle_mod.simplify(eG, cT, 50.0)
    assert keep.tolist() == [0, 1, 0]
    _assert_coverage(eG, cT, keep)
    # if slice 2 is cheaper than slice 1 somewhere, it is kept as well
    cT[2, 0, 0] = 1.5
    keep, robust = oracle_mod.simplify(eG, cT, 50.0)
    assert keep.tolist() == [0, 1, 1]


def test_untraversable_slice_removed_and_keep_ends(oracle_mod):
    N, H, W = 4, 5, 5
    eG = np.zeros((N, H, W), np.float32)
    eG[2:] = 2.0
    cT = np.full((N, H, W), 50.0)       # nothing traversable anywhere
    keep, _ = oracle_mod.simplify(eG, cT, 50.0)
    assert keep.tolist() == [0, 0, 0, 0]
    keep, _ = oracle_mod.simplify(eG, cT, 50.0, keep_ends=True)
    assert keep.tolist() == [1, 0, 0, 1]


def test_near_equal_costs_are_not_robust(oracle_mod):
    N, H, W = 2, 4, 4
    eG = np.zeros((N, H, W), np.float32)
    cT = np.full((N, H, W), 1.0)
    cT[1] += 1e-9                       # Eq. 9 for slice 0 hinges on 1e-9
    keep, robust = oracle_mod.simplify(eG, cT, 50.0)
    assert keep.tolist() == [1, 0]
    assert not robust


def test_two_storey_building_chain(oracle_mod):
    sc = scenes.building(21, 60_000, side_cells=80, floors=[0.0, 3.0], ceilings=[2.8, 5.8])
    g = oracle_mod.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, 0.5, 0.0, 12)
    eG, eC, g, _, _ = oracle_mod.build(sc.points, g, zmin_from_data=True)
    cT, mask, frag = oracle_mod.evaluate(g, PARAMS_ROBOT, eG, eC)
    keep, robust = oracle_mod.simplify(eG, cT, 50.0, frag)
    assert robust
    _assert_coverage(eG, cT, keep)
    kept = np.nonzero(keep)[0]
    # both storeys are represented by kept slices with wide traversable floors
    for z in (0.0, 3.0):
        best = max(((np.abs(eG[k] - z) < 0.05) & (cT[k] < 50.0)).mean() for k in kept)
        assert best > 0.3
    assert len(kept) < g.N
