"""Pins of the oracle's scene evaluation (Sec. III-B, Eq. 1-6).

Expected values are closed forms of the equations on constructed elevation
layers (tilted planes, flat floors under known ceilings, a staircase, a
single barrier), the Fig. 3 kernel values, and invariants (m^xy <= m^grad,
c^init <= c^T <= c^B, mask = barriers dilated by the d_inf disc).
"""
import math
import os

import numpy as np
import pytest

from conftest import PARAMS_ROBOT, PARAMS_TABLE1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = np.inf


def _grid(oracle_mod, H, W, N=1, res=0.1):
    return oracle_mod.Grid(0.0, 0.0, res, W, H, 0.5, 0.0, N)


def _eval(oracle_mod, eG, eC, params, res=0.1):
    eG = np.asarray(eG, np.float32)[None] if eG.ndim == 2 else np.asarray(eG, np.float32)
    eC = np.asarray(eC, np.float32)[None] if eC.ndim == 2 else np.asarray(eC, np.float32)
    N, H, W = eG.shape
    return oracle_mod.evaluate(_grid(oracle_mod, H, W, N, res), params, eG, eC, want_aux=True)


def _plane(H, W, ax, ay, res=0.1):
    j = np.arange(W)[None, :]
    i = np.arange(H)[:, None]
    return ((ax * (j + 0.5) + ay * (i + 0.5)) * res).astype(np.float32)


INTERIOR = (slice(1, -1), slice(1, -1))


@pytest.mark.parametrize("deg", [15.0, 25.0])
@pytest.mark.parametrize("axis", ["x", "y"])
def test_tilted_plane_gradient_is_tan_theta(oracle_mod, deg, axis):
    t = math.tan(math.radians(deg))
    eG = _plane(24, 30, t, 0.0) if axis == "x" else _plane(24, 30, 0.0, t)
    eC = np.full_like(eG, INF)
    cT, mask, frag, aux = _eval(oracle_mod, eG, eC, PARAMS_ROBOT)
    mxy, mgr, cI, cG = aux[0, 0], aux[1, 0], aux[2, 0], aux[3, 0]
    np.testing.assert_allclose(mgr[INTERIOR], t, rtol=1e-5)
    np.testing.assert_allclose(mxy[INTERIOR], t, rtol=1e-5)
    # border cells have no central difference: barrier
    assert np.all(np.isinf(mgr[0])) and np.all(np.isinf(mgr[:, -1]))
    assert np.all(cG[0] == 50.0)
    # gentle (tan 15 and tan 25 are below theta_s = tan 30): Eq. 3 second case
    th_s = np.float32(PARAMS_ROBOT["theta_s"]).astype(np.float64)
    np.testing.assert_allclose(cG[INTERIOR], 15.0 * (t / th_s) ** 2, rtol=1e-5)
    assert np.all(cI == 0.0)          # no ceiling anywhere


def test_steep_plane_with_table1_theta_s_is_barrier(oracle_mod):
    # tan 25 = 0.466 exceeds Table I's theta_s = 0.36 and no neighbour is
    # gentle, so p_s = 0 and Eq. 4 gives c^B; tan 15 = 0.268 stays gentle.
    eG = _plane(20, 20, math.tan(math.radians(25.0)), 0.0)
    cT, mask, frag, aux = _eval(oracle_mod, eG, np.full_like(eG, INF), PARAMS_TABLE1)
    assert np.all(aux[3, 0][INTERIOR] == 50.0)
    assert not mask.any()
    eG = _plane(20, 20, math.tan(math.radians(15.0)), 0.0)
    cT, mask, frag, aux = _eval(oracle_mod, eG, np.full_like(eG, INF), PARAMS_TABLE1)
    np.testing.assert_allclose(aux[3, 0][INTERIOR],
                               15.0 * (math.tan(math.radians(15.0)) / np.float32(0.36)) ** 2,
                               rtol=1e-5)


def test_diagonal_plane_mxy_vs_mgrad(oracle_mod):
    a = 0.3
    eG = _plane(20, 20, a, a)
    cT, mask, frag, aux = _eval(oracle_mod, eG, np.full_like(eG, INF), PARAMS_ROBOT)
    np.testing.assert_allclose(aux[0, 0][INTERIOR], a, rtol=1e-5)
    np.testing.assert_allclose(aux[1, 0][INTERIOR], a * math.sqrt(2.0), rtol=1e-5)


@pytest.mark.parametrize("gap,expected", [(0.60, 1.0), (0.45, 50.0), (0.70, 0.0),
                                          (0.65, 0.0), (2.0, 0.0)])
def test_interval_cost_closed_form(oracle_mod, gap, expected):
    # Eq. 1 on a flat floor a = 0 under a flat ceiling b: d^I = b - a.
    H = W = 21
    eG = np.zeros((H, W), np.float32)
    eC = np.full((H, W), gap, np.float32)
    cT, mask, frag, aux = _eval(oracle_mod, eG, eC, PARAMS_ROBOT)
    cI = aux[2, 0]
    np.testing.assert_allclose(cI, expected, rtol=1e-5, atol=1e-5)
    # far from the (barrier) map border, c^T equals the uniform c^init
    R = 5
    core = (slice(R + 1, -R - 1), slice(R + 1, -R - 1))
    np.testing.assert_allclose(cT[0][core], expected, rtol=1e-5, atol=1e-5)
    assert np.all(mask[0][core] == (expected < 50.0))


def test_interval_at_dmin_fragility(oracle_mod):
    # d^I exactly d_min, as a difference float32 holds exactly: not a barrier
    # (Eq. 1 is strict) and decided the same way in any precision.
    eG = np.zeros((15, 15), np.float32)
    eC = np.full((15, 15), 0.5, np.float32)
    cT, mask, frag, aux = _eval(oracle_mod, eG, eC, PARAMS_ROBOT)
    np.testing.assert_allclose(aux[2, 0], 20.0 * (0.65 - 0.5), rtol=1e-5)
    assert frag[0][7, 7] == 0
    # ground 0.001, ceiling fl32(0.501): in FP64 d^I = 0.4999999871 < d_min,
    # but the float32 difference rounds to 0.5; the cell and its window are
    # marked fragile (cost and mask).
    eG[7, 7] = np.float32(0.001)
    eC[7, 7] = np.float32(0.501)
    assert float(eC[7, 7]) - float(eG[7, 7]) < 0.5
    assert np.float32(eC[7, 7]) - np.float32(eG[7, 7]) == np.float32(0.5)
    cT, mask, frag, aux = _eval(oracle_mod, eG, eC, PARAMS_ROBOT)
    assert aux[2, 0][7, 7] == 50.0
    assert frag[0][7, 7] == 3 and frag[0][7, 10] == 3
    assert frag[0][7, 13] == 0          # beyond the window radius of 5


def _staircase(H, W, tread=4, riser=0.17):
    j = np.arange(W)[None, :]
    return np.broadcast_to((riser * (j // tread)).astype(np.float32), (H, W)).copy()


@pytest.mark.parametrize("theta_p,edge_cost", [(0.20, 5.0), (0.60, 5.0), (0.70, 50.0), (1.0, 50.0)])
def test_staircase_step_cost(oracle_mod, theta_p, edge_cost):
    # Treads of 4 cells and 0.17 m risers: the two tread cells next to a riser
    # see a central difference of 0.17 / 0.2 = 0.85, inside (theta_s, theta_b);
    # the two middle cells see 0.  In the 5x5 patch of an edge cell the gentle
    # columns are -2, +1, +2: 15 of 24 neighbours, p_s = 0.625.  Eq. 4 then
    # gives alpha_b (0.85 / 1.7)^2 = 5.0 when p_s > theta_p, else c^B;
    # theta_p = 1 is the wheeled-robot setting that never allows it.
    eG = _staircase(16, 32)
    p = dict(PARAMS_ROBOT, theta_p=theta_p)
    cT, mask, frag, aux = _eval(oracle_mod, eG, np.full_like(eG, INF), p)
    cG = aux[3, 0]
    mxy = aux[0, 0]
    rows = slice(3, 13)
    for j in range(4, 28):
        if j % 4 in (0, 3):
            np.testing.assert_allclose(mxy[rows, j], 0.85, rtol=1e-5)
            np.testing.assert_allclose(cG[rows, j], edge_cost, rtol=1e-5)
        else:
            assert np.all(cG[rows, j] == 0.0)


@pytest.mark.parametrize("axis", ["rows", "columns"])
def test_step_cost_patch_at_the_map_border(oracle_mod, axis):
    """The p_s patch of Eq. 4 (our reading R8): the (2R_p+1)^2 - 1 = 24
    neighbours without the centre; a neighbour off the map counts as not
    gentle and stays in the denominator.  On the staircase above, a step-edge
    cell in the interior sees 15 gentle neighbours (p_s = 15/24).  One cell
    from the map border, its patch loses the off-map line (5 cells) and the
    border line (no central difference there, so not gentle): 3 gentle
    columns on 3 lines, p_s = 9/24 = 0.375.  Two cells from the border only
    the border line is lost: 12/24 = 0.5.  theta_p = 0.37 separates 9/24 from
    9/25 (a patch that counted the centre), theta_p = 0.45 separates 9/24
    from 9/19 (a patch that dropped off-map neighbours from the
    denominator)."""
    eG = _staircase(16, 32)
    if axis == "columns":
        eG = np.ascontiguousarray(eG.T)
    for theta_p, near1 in ((0.37, 5.0), (0.45, 50.0)):
        p = dict(PARAMS_ROBOT, theta_p=theta_p)
        cT, mask, frag, aux = _eval(oracle_mod, eG, np.full_like(eG, INF), p)
        cG = aux[3, 0] if axis == "rows" else aux[3, 0].T
        n = cG.shape[0]
        for j in range(4, 28):
            if j % 4 not in (0, 3):
                continue
            # one line from either border: 9/24; two lines: 12/24; interior 15/24
            np.testing.assert_allclose([cG[1, j], cG[n - 2, j]], near1, rtol=1e-6)
            np.testing.assert_allclose([cG[2, j], cG[n - 3, j], cG[7, j]], 5.0, rtol=1e-6)
        assert np.all(frag == 0)


def _golden_fig3():
    rows = []
    with open(os.path.join(GOLDEN, "fig3_inflation.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                d, v = line.split()
                rows.append((int(d), float(v)))
    return rows


def test_single_barrier_inflation_fig3(oracle_mod):
    # One barrier cell (ceiling 0.3 m above a flat floor: d^I < d_min) in an
    # otherwise free field, with the Fig. 3 kernel: c^T = c^B K(m, n).
    p = dict(PARAMS_TABLE1, d_inf=0.2, d_sm=0.4)
    H = W = 31
    c = 15
    eG = np.zeros((H, W), np.float32)
    eC = np.full((H, W), INF, np.float32)
    eC[c, c] = 0.3
    cT, mask, frag, aux = _eval(oracle_mod, eG, eC, p)
    for d, v in _golden_fig3():
        for (di, dj) in ((0, d), (0, -d), (d, 0), (-d, 0)):
            assert cT[0][c + di, c + dj] == pytest.approx(v, rel=1e-12, abs=1e-12)
    # the whole window follows Eq. 6
    K = oracle_mod.kernel(p, 0.1)
    R = K.shape[0] // 2
    assert R == 4
    np.testing.assert_allclose(cT[0][c - R:c + R + 1, c - R:c + R + 1], 50.0 * K, rtol=1e-12)
    # mask: the barrier dilated by the disc of radius d_inf / r_g = 2 cells
    ii, jj = np.mgrid[0:H, 0:W]
    disc = (ii - c) ** 2 + (jj - c) ** 2 <= 4
    core = (slice(6, -6), slice(6, -6))
    np.testing.assert_array_equal(mask[0][core], ~disc[core])


def test_kernel_weights_eq6(oracle_mod):
    # Fig. 3 parameters in cell units: D_inf = 2, D_sm = 3
    K = oracle_mod.kernel(dict(PARAMS_TABLE1, d_inf=0.2, d_sm=0.4), 0.1)
    R = 4
    assert K.shape == (9, 9)
    for n in range(-R, R + 1):
        for m in range(-R, R + 1):
            d = math.hypot(m, n)
            assert K[n + R, m + R] == pytest.approx(min(1.0, max(0.0, 1.0 - (d - 2.0) / 3.0)))
    # benchmark robot: d_inf = 0.3 -> D_inf = 3, D_sm = 3, window radius 5,
    # 109 taps with a positive weight; at 0.05 m: D_inf = 6, D_sm = 7, radius 12
    K = oracle_mod.kernel(PARAMS_ROBOT, 0.1)
    assert K.shape == (11, 11) and int((K > 0).sum()) == 109
    assert K[5, 8] == 1.0 and K[5, 9] == pytest.approx(2.0 / 3.0)
    K = oracle_mod.kernel(PARAMS_ROBOT, 0.05)
    assert K.shape == (25, 25)


def test_invariants_random_field(oracle_mod):
    rng = np.random.default_rng(3)
    H, W, N = 40, 36, 3
    base = rng.normal(0, 0.05, (H, W)).cumsum(1).astype(np.float32) * 0.2
    eG = np.stack([base + 0.5 * k for k in range(N)]).astype(np.float32)
    eG[rng.random(eG.shape) < 0.05] = -INF
    eC = (eG + rng.uniform(0.3, 1.2, eG.shape)).astype(np.float32)
    eC[rng.random(eG.shape) < 0.3] = INF
    cT, mask, frag, aux = oracle_mod.evaluate(_grid(oracle_mod, H, W, N), PARAMS_ROBOT, eG, eC,
                                              want_aux=True)
    mxy, mgr, cinit = aux[0], aux[1], aux[4]
    fin = np.isfinite(mgr)
    assert np.all(mxy[fin] <= mgr[fin] * (1 + 1e-15))
    assert np.all(np.isinf(mxy[~fin]))
    assert np.all(cinit <= cT + 1e-12) and np.all(cT <= 50.0)
    assert np.all(cinit[eG == -INF] == 50.0)        # no ground: barrier
    np.testing.assert_array_equal(mask, (cT < 50.0).astype(np.uint8))
    assert (frag > 0).mean() < 0.01


def test_invalid_neighbour_blocks_gradient(oracle_mod):
    eG = np.zeros((9, 9), np.float32)
    eG[4, 4] = -INF
    cT, mask, frag, aux = _eval(oracle_mod, eG, np.full_like(eG, INF), PARAMS_ROBOT)
    mgr = aux[1, 0]
    for (i, j) in ((3, 4), (5, 4), (4, 3), (4, 5), (4, 4)):
        assert np.isinf(mgr[i, j])
    assert mgr[3, 3] == 0.0
