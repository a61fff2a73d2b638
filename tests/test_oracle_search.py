"""Pins of the search oracle (Sec. III-D) to closed forms and hand-counted
cases: octile distances on a free floor, uniform node costs, a slope, a wall
with a gap, node merging across slices (c^N = min c^T) and gateways, which
only open towards the slice with the lower c^T."""
import math

import numpy as np
import pytest

from oracle import search

C_B = 50.0
RES = 0.1


def flat(H, W, N=1, cost=0.0, z=0.0):
    eG = np.full((N, H, W), z, np.float32)
    cT = np.full((N, H, W), cost, np.float32)
    return eG, cT


@pytest.mark.parametrize("a,b", [(0, 7), (5, 5), (3, 8), (9, 2)])
def test_free_floor_is_octile_distance(a, b):
    eG, cT = flat(12, 12)
    cost, path = search.plan(eG, cT, None, C_B, RES, (0, 0, 0), (a, b, 0))
    assert cost == pytest.approx(abs(a - b) + math.sqrt(2) * min(a, b), rel=1e-12)
    assert path[0] == (0, 0, 0) and path[-1] == (a, b, 0)
    assert len(path) == max(a, b) + 1


def test_uniform_cost_counts_entered_nodes():
    c = 3.5
    eG, cT = flat(10, 10, cost=c)
    cost, path = search.plan(eG, cT, None, C_B, RES, (1, 1, 0), (4, 9, 0))
    # 8 nodes entered, 3 of them diagonally
    assert cost == pytest.approx(8 * c + 5 + 3 * math.sqrt(2), rel=1e-12)
    assert search.path_cost(eG, cT, None, C_B, RES, path) == pytest.approx(cost, rel=1e-12)


def test_slope_adds_the_elevation_change():
    s = 0.25   # rise per metre
    eG, cT = flat(3, 20)
    eG[0] = (np.arange(20) * RES * s).astype(np.float32)[None, :]
    cost, _ = search.plan(eG, cT, None, C_B, RES, (1, 0, 0), (1, 19, 0))
    steps = np.diff(eG[0, 1].astype(np.float64)) / RES
    assert cost == pytest.approx(np.sum(np.sqrt(1.0 + steps ** 2)), rel=1e-12)
    assert cost > 19.0


def test_wall_with_a_gap():
    eG, cT = flat(9, 9)
    cT[0, :, 4] = C_B          # a wall along column 4 ...
    cT[0, 8, 4] = 0.0          # ... open at the last row
    cost, path = search.plan(eG, cT, None, C_B, RES, (0, 0, 0), (0, 8, 0))
    assert (8, 4, 0) in path
    # through the gap cell: (0, 0) -> (8, 4) is 8 rows and 4 columns, octile
    # 4 + 4 sqrt 2, and (8, 4) -> (0, 8) the same
    leg = (8 - 4) + math.sqrt(2) * 4
    assert cost == pytest.approx(2 * leg, rel=1e-12)


def test_barrier_everywhere_is_unreachable():
    eG, cT = flat(5, 5)
    cT[0, :, 2] = C_B
    cost, path = search.plan(eG, cT, None, C_B, RES, (2, 0, 0), (2, 4, 0))
    assert cost == math.inf and path == []


def test_invalid_ground_cannot_be_entered():
    eG, cT = flat(5, 5)
    eG[0, :, 2] = -np.inf
    cost, _ = search.plan(eG, cT, None, C_B, RES, (2, 0, 0), (2, 4, 0))
    assert cost == math.inf


def two_levels():
    """Two kept slices over a 3 x 12 strip.  Slice 0 sees the lower floor
    (z = 0) everywhere, open on columns 0-4 (c^T 0), costlier on column 5
    (c^T 2) and blocked under the upper structure on columns 6-11 (c^B).
    Slice 1 sees the upper structure (z = 3, c^B) over columns 0-4, the lower
    floor on column 5 (c^T 1: cheaper than slice 0, a gateway up), a ramp
    cell at 0.05 m on column 6 and the upper floor (z = 3) on columns 7-11,
    all at c^T 0.5.  Only column 5 has the same ground on both slices."""
    H, W = 3, 12
    eG = np.zeros((2, H, W), np.float32)
    cT = np.zeros((2, H, W), np.float32)
    cT[0, :, 5] = 2.0
    cT[0, :, 6:] = C_B
    eG[1, :, :5] = 3.0
    cT[1, :, :5] = C_B
    cT[1, :, 5] = 1.0
    eG[1, :, 6] = 0.05
    eG[1, :, 7:] = 3.0
    cT[1, :, 6:] = 0.5
    return eG, cT


RAMP = float(np.float32(0.05))


def upper_leg():
    """Cost from column 5 (z = 0) to column 11 on slice 1: the ramp cell, the
    climb onto the upper floor and 4 cells on it."""
    return (0.5 + math.sqrt(1 + (RAMP / RES) ** 2)
            + 0.5 + math.sqrt(1 + ((3.0 - RAMP) / RES) ** 2) + 4 * (0.5 + 1.0))


def test_gateway_up_and_node_merge():
    eG, cT = two_levels()
    cost, path = search.plan(eG, cT, None, C_B, RES, (1, 0, 0), (1, 11, 1))
    # slice 0: 4 free cells, then column 5 whose c^N is min(2, 1) = 1 (the
    # same node on both slices); the gateway to slice 1; the upper leg
    assert cost == pytest.approx(4 * 1.0 + (1.0 + 1.0) + upper_leg(), rel=1e-12)
    ks = [k for (_, _, k) in path]
    assert ks[0] == 0 and ks[-1] == 1 and ks == sorted(ks)
    gate = [p for p, q in zip(path[:-1], path[1:]) if p[:2] == q[:2]]
    assert len(gate) == 1 and gate[0][1] == 5
    assert search.path_cost(eG, cT, None, C_B, RES, path) == pytest.approx(cost, rel=1e-12)


def test_no_gateway_towards_the_costlier_slice():
    eG, cT = two_levels()
    cT[1, :, 5] = 3.0           # now slice 1 is costlier at the shared column
    cost, _ = search.plan(eG, cT, None, C_B, RES, (1, 0, 0), (1, 11, 1))
    assert cost == math.inf


def test_gateway_down_and_goal_on_the_merged_node():
    eG, cT = two_levels()
    cT[1, :, 5] = 3.0           # slice 0 cheaper at column 5: a gateway down
    cost, path = search.plan(eG, cT, None, C_B, RES, (1, 11, 1), (1, 0, 0))
    # the upper leg backwards (column 5 entered at c^N = min(2, 3) = 2 instead
    # of the ramp cell's 0.5 on the way up), the gateway, 5 free cells
    back = (4 * (0.5 + 1.0) + 0.5 + math.sqrt(1 + ((3.0 - RAMP) / RES) ** 2)
            + 2.0 + math.sqrt(1 + (RAMP / RES) ** 2) + 5 * 1.0)
    assert cost == pytest.approx(back, rel=1e-12)
    assert path[-1] == (1, 0, 0)
    assert search.path_cost(eG, cT, None, C_B, RES, path) == pytest.approx(cost, rel=1e-12)
    # the goal is the node, not the slice: a goal given on slice 1 at column 5
    # is reached on slice 0 already
    c2, p2 = search.plan(eG, cT, None, C_B, RES, (1, 0, 0), (1, 5, 1))
    assert c2 == pytest.approx(4 * 1.0 + 2.0 + 1.0, rel=1e-12)
    assert p2[-1] == (1, 5, 0)


def test_dropped_slices_are_skipped():
    eG, cT = two_levels()
    eG3 = np.stack([eG[0], eG[0], eG[1]])
    cT3 = np.stack([cT[0], cT[0], cT[1]])
    a, _ = search.plan(eG, cT, None, C_B, RES, (1, 0, 0), (1, 11, 1))
    b, _ = search.plan(eG3, cT3, [1, 0, 1], C_B, RES, (1, 0, 0), (1, 11, 2))
    assert a == pytest.approx(b, rel=1e-15)
