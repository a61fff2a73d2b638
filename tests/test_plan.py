"""The library's path search across slices (tct_planner_*, Sec. III-D; host
code, so these run on the CPU) against the search oracle: optimal costs
equal up to summation order, every returned path a valid walk of the graph
whose cost is the reported one, unreachable goals reported as such."""
import math

import numpy as np
import pytest

from conftest import PARAMS_TABLE1

from oracle import search

C_B = 50.0


@pytest.fixture(scope="module")
def tct():
    from paper_2403_07631_gb300 import build, tct
    build.build()
    return tct


def random_tomogram(seed, N=5, H=22, W=26):
    """Ground stacks non-decreasing in the slice index drawn from a few levels
    (so that equal ground across slices, i.e. merged nodes and gateways, are
    common), invalid ground at the bottom of some cells, costs in [0, 20)
    with a fifth of the cells at c^B."""
    rng = np.random.default_rng(seed)
    levels = np.array([-np.inf, 0.0, 0.02, 0.1, 0.4, 1.5, 3.0], np.float32)
    steps = rng.integers(0, 3, (N, H, W))
    steps[0] = rng.integers(0, 4, (H, W))
    idx = np.minimum(np.cumsum(steps, 0), len(levels) - 1)
    eG = levels[idx]
    cT = rng.uniform(0.0, 20.0, (N, H, W)).astype(np.float32)
    cT[rng.random((N, H, W)) < 0.2] = C_B
    cT[~np.isfinite(eG)] = C_B
    keep = (rng.random(N) < 0.8).astype(np.uint8)
    keep[rng.integers(0, N)] = 1
    return eG, cT, keep


def traversable_endpoints(eG, cT, keep, count, seed):
    rng = np.random.default_rng(seed)
    kept = np.flatnonzero(keep)
    cand = [(i, j, int(k)) for k in kept for i, j in zip(*np.nonzero(cT[k] < C_B))]
    pick = rng.choice(len(cand), (count, 2))
    return [cand[a] for a in pick[:, 0]], [cand[b] for b in pick[:, 1]]


def grid_of(tct, eG, res):
    N, H, W = eG.shape
    return tct.Grid(0.0, 0.0, res, W, H, 0.5, N, 0.0, False)


def check(tct, eG, cT, keep, res, starts, goals, n_threads=0):
    pl = tct.Planner(grid_of(tct, eG, res), eG, cT, keep, C_B)
    paths, costs, expanded = pl.plan(starts, goals, n_threads=n_threads)
    res64 = float(np.float32(res))
    n_reach = 0
    for s, g, path, c in zip(starts, goals, paths, costs):
        ref, _ = search.plan(eG, cT, keep, C_B, res64, s, g)
        if math.isinf(ref):
            assert math.isinf(c) and len(path) == 0, (s, g)
            continue
        n_reach += 1
        assert c == pytest.approx(ref, rel=1e-12, abs=1e-12), (s, g)
        walk = [tuple(int(v) for v in p) for p in path]
        assert walk[0] == tuple(s)
        assert walk[-1][:2] == tuple(g[:2]) and eG[walk[-1][2]][g[0], g[1]] == eG[g[2]][g[0], g[1]]
        assert search.path_cost(eG, cT, keep, C_B, res64, walk) == pytest.approx(c, rel=1e-12,
                                                                                abs=1e-12)
    return paths, costs, expanded, n_reach


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_tomograms_match_oracle(tct, seed):
    eG, cT, keep = random_tomogram(seed)
    starts, goals = traversable_endpoints(eG, cT, keep, 40, seed + 100)
    _, _, expanded, n_reach = check(tct, eG, cT, keep, 0.1, starts, goals)
    assert n_reach >= 5
    assert (expanded > 0).all()


def test_building_tomogram_matches_oracle(tct, oracle_mod):
    """A two-storey building with a ramp evaluated by the oracle itself: real
    gateways between the floors' slices."""
    from paper_2403_07631_gb300 import scenes
    sc = scenes.building(7, 60_000, side_cells=60, res=0.1, floors=[0.0, 2.0],
                         ceilings=[1.8, 3.8])
    g = oracle_mod.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, 0.0, 10)
    eG, eC, g, _, _ = oracle_mod.build(sc.points, g, True)
    op = {k: PARAMS_TABLE1[k] for k in oracle_mod.PARAM_FIELDS}
    cT, _, frag = oracle_mod.evaluate(g, op, eG, eC)
    keep, _ = oracle_mod.simplify(eG, cT, op["c_b"], frag)
    cT = cT.astype(np.float32)
    starts, goals = traversable_endpoints(eG, cT, keep, 12, 5)
    _, costs, _, n_reach = check(tct, eG, cT, keep, sc.res, starts, goals)
    assert n_reach >= 3


def test_threads_give_the_same_answers(tct):
    eG, cT, keep = random_tomogram(9)
    starts, goals = traversable_endpoints(eG, cT, keep, 64, 9)
    pl = tct.Planner(grid_of(tct, eG, 0.1), eG, cT, keep, C_B)
    p1, c1, e1 = pl.plan(starts, goals, n_threads=1)
    p4, c4, e4 = pl.plan(starts, goals, n_threads=4)
    np.testing.assert_array_equal(c1, c4)
    np.testing.assert_array_equal(e1, e4)
    for a, b in zip(p1, p4):
        np.testing.assert_array_equal(a, b)


def test_refusals_and_truncation(tct):
    eG, cT, keep = random_tomogram(4)
    pl = tct.Planner(grid_of(tct, eG, 0.1), eG, cT, keep, C_B)
    dropped = int(np.flatnonzero(keep == 0)[0]) if (keep == 0).any() else None
    with pytest.raises(tct.TctError, match="tct_plan_paths"):
        pl.plan([(0, 0, 0)], [(eG.shape[1], 0, 0)])
    if dropped is not None:
        with pytest.raises(tct.TctError):
            pl.plan([(0, 0, dropped)], [(1, 1, dropped)])
    # a free floor: the far corner takes 21 states at least; max_len 5 cuts it
    N, H, W = 1, 12, 21
    free = np.zeros((N, H, W), np.float32)
    pl2 = tct.Planner(grid_of(tct, free, 0.1), free, free, None, C_B)
    with pytest.raises(tct.TctError, match="workspace"):
        pl2.plan([(0, 0, 0)], [(H - 1, W - 1, 0)], max_len=5)
    paths, costs, _ = pl2.plan([(0, 0, 0)], [(H - 1, W - 1, 0)], max_len=64)
    assert len(paths[0]) == W and costs[0] == pytest.approx((W - H) + math.sqrt(2) * (H - 1))
    # an end point on a barrier: unreachable, not an error
    wall = free.copy()
    wall[0, 5, 5] = C_B
    pl3 = tct.Planner(grid_of(tct, free, 0.1), free, wall, None, C_B)
    paths, costs, _ = pl3.plan([(5, 5, 0)], [(0, 0, 0)])
    assert len(paths[0]) == 0 and math.isinf(costs[0])
    with pytest.raises(ValueError):
        tct.Planner(grid_of(tct, free, 0.1), free[:, :4], free, None, C_B)
