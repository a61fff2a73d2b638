"""Pins of the oracle's cost/elevation queries (the C(q), e^G(q) of Eq. 10):
bilinear reproduction of linear fields with their constant gradient, a
2x2 example worked by hand, clamping at the border, the invalid-ground fill,
the analytic gradient against central differences, and the refinement:
its descent property, a straight equally spaced path as a fixed point of
the smoothness term, one step on a linear cost moving each interior
waypoint by exactly -eta * gradient, and translation invariance."""
import numpy as np
import pytest


def _grid(oracle_mod, H, W, N=1, res=0.1, z_min=0.0, d_s=0.5):
    return oracle_mod.Grid(0.0, 0.0, res, W, H, d_s, z_min, N)


def test_linear_field_reproduced_with_constant_gradient(oracle_mod):
    H, W = 9, 12
    a, b, c0 = 0.7, -1.3, 2.0
    jj, ii = np.meshgrid(np.arange(W), np.arange(H))
    # value at cell centres (x = (j+0.5) r, y = (i+0.5) r)
    layer = (c0 + a * (jj + 0.5) * 0.1 + b * (ii + 0.5) * 0.1).astype(np.float32)[None]
    rng = np.random.default_rng(0)
    xy = np.stack([rng.uniform(0.05, W * 0.1 - 0.05, 200), rng.uniform(0.05, H * 0.1 - 0.05, 200)], 1)
    val, grad = oracle_mod.sample(_grid(oracle_mod, H, W), layer, xy, np.zeros(200))
    xyf = xy.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(val, c0 + a * xyf[:, 0] + b * xyf[:, 1], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(grad[:, 0], a, rtol=1e-5)
    np.testing.assert_allclose(grad[:, 1], b, rtol=1e-5)


def test_two_by_two_by_hand(oracle_mod):
    # centres at (0.5, 0.5), (1.5, 0.5), (0.5, 1.5), (1.5, 1.5) with r = 1:
    # at (0.75, 1.25): fu = 0.25, fv = 0.75 ->
    # 0.75*0.25*1 + 0.25*0.25*3 + 0.75*0.75*5 + 0.25*0.75*7 = 4.5
    layer = np.array([[[1.0, 3.0], [5.0, 7.0]]], np.float32)
    g = _grid(oracle_mod, 2, 2, res=1.0)
    val, grad = oracle_mod.sample(g, layer, np.array([[0.75, 1.25]]), np.array([0]))
    assert val[0] == pytest.approx(4.5)
    # d/dx = (1-fv)(3-1) + fv(7-5) = 2, d/dy = (1-fu)(5-1) + fu(7-3) = 4
    assert grad[0, 0] == pytest.approx(2.0) and grad[0, 1] == pytest.approx(4.0)
    # beyond the last centre the query is clamped and its gradient is zero
    val, grad = oracle_mod.sample(g, layer, np.array([[3.0, 1.25]]), np.array([0]))
    # u clamps to the last column: fu = 1, fv = 0.75 -> 0.25*3 + 0.75*7 = 6
    assert val[0] == pytest.approx(6.0)
    assert grad[0, 0] == 0.0 and grad[0, 1] == pytest.approx(4.0)
    # out-of-range slice and non-finite query give NaN
    val, grad = oracle_mod.sample(g, layer, np.array([[0.7, 0.7], [np.nan, 0.7]]), np.array([1, 0]))
    assert np.isnan(val).all()


def test_invalid_ground_reads_plane_below(oracle_mod):
    # ground sampler: -inf reads h_k - d_s with h_k = z_min + (k+1) d_s
    layer = np.full((2, 3, 3), -np.inf, np.float32)
    g = _grid(oracle_mod, 3, 3, N=2, z_min=1.0, d_s=0.5)
    val, _ = oracle_mod.sample(g, layer, np.array([[0.15, 0.15], [0.15, 0.15]]), np.array([0, 1]),
                               is_ground=True)
    np.testing.assert_allclose(val, [1.0, 1.5])


def test_gradient_matches_central_differences(oracle_mod):
    """The analytic gradient of the interpolant against FP64 central
    differences (h = 1e-4 m) of the oracle's own values at FP64 coordinates,
    at the sampler tolerance |g - fd| <= 1e-5 max(|fd|, c^B / r_g).  Queries
    within 2h of a lattice line are skipped (the interpolant has a kink
    there); elsewhere it is linear along each axis, so the difference is
    exact up to FP64 rounding and a dropped term, a wrong corner or a wrong
    sign would show far above the tolerance."""
    rng = np.random.default_rng(3)
    H, W = 20, 25
    layer = rng.uniform(0, 50, (2, H, W)).astype(np.float32)
    g = _grid(oracle_mod, H, W, N=2)
    h = 1e-4
    xy = np.stack([rng.uniform(0.1, 2.4, 300), rng.uniform(0.1, 1.9, 300)], 1)
    u = xy / 0.1 - 0.5
    ok = (np.abs(u - np.round(u)) > 2 * h / 0.1).all(1)
    xy = xy[ok]
    sl = rng.integers(0, 2, len(xy))
    _, grad = oracle_mod.sample_f64(g, layer, xy, sl)
    fd = np.zeros_like(grad)
    for a in range(2):
        e = np.zeros(2); e[a] = h
        vp, _ = oracle_mod.sample_f64(g, layer, xy + e, sl)
        vm, _ = oracle_mod.sample_f64(g, layer, xy - e, sl)
        fd[:, a] = (vp - vm) / (2 * h)
    scale = np.maximum(np.abs(fd), 50.0 / 0.1)
    assert np.all(np.abs(grad - fd) <= 1e-5 * scale)
    assert np.abs(grad - fd).max() < 1e-8 * 500      # FP64 rounding only
    # the float32-coordinate entry reads the same values at float32 points
    x32 = xy.astype(np.float32)
    v32, g32 = oracle_mod.sample(g, layer, x32, sl)
    v64, g64 = oracle_mod.sample_f64(g, layer, x32.astype(np.float64), sl)
    np.testing.assert_array_equal(v32, v64)
    np.testing.assert_array_equal(g32, g64)


def test_refinement_descends_smooth_bowl(oracle_mod):
    # a quadratic bowl of cost: descent pulls interior waypoints to the centre line
    H = W = 40
    jj, ii = np.meshgrid(np.arange(W), np.arange(H))
    y = (ii + 0.5) * 0.1
    cost = (5.0 * (y - 2.0) ** 2).astype(np.float32)[None]
    g = _grid(oracle_mod, H, W)
    L = 30
    xs = np.linspace(0.5, 3.5, L)
    xy = np.stack([xs, np.full(L, 2.6)], 1)[None]
    xy[0, 0, 1] = xy[0, -1, 1] = 2.0
    out = oracle_mod.refine(g, cost, np.zeros((1, L)), xy, steps=200, eta=1e-2, lam=1.0)
    assert np.all(np.abs(out[0, 1:-1, 1] - 2.0) < np.abs(xy[0, 1:-1, 1] - 2.0))
    np.testing.assert_array_equal(out[0, [0, -1]], xy[0, [0, -1]])


def test_refinement_straight_path_is_a_fixed_point(oracle_mod):
    # zero cost: only the smoothness term acts, and an equally spaced straight
    # path has every second difference zero
    H = W = 30
    g = _grid(oracle_mod, H, W)
    cost = np.zeros((1, H, W), np.float32)
    L = 25
    t = np.linspace(0.0, 1.0, L)[:, None]
    xy = (np.array([0.4, 0.7]) * (1 - t) + np.array([2.6, 2.1]) * t)[None]
    out = oracle_mod.refine(g, cost, np.zeros((1, L)), xy, steps=40, eta=1e-2, lam=1.0)
    np.testing.assert_allclose(out, xy, atol=1e-12)


def test_refinement_linear_cost_moves_by_eta_times_gradient(oracle_mod):
    # lambda = 0 and a linear cost field (reproduced exactly by the bilinear
    # query, with a constant gradient): one step moves every interior
    # waypoint by exactly -eta * gradient, the ends stay
    H, W = 30, 40
    a, b = 0.8, -0.5
    jj, ii = np.meshgrid(np.arange(W), np.arange(H))
    cost = (10.0 + a * (jj + 0.5) * 0.1 + b * (ii + 0.5) * 0.1).astype(np.float32)[None]
    g = _grid(oracle_mod, H, W)
    rng = np.random.default_rng(3)
    xy = np.stack([rng.uniform(0.5, 3.5, 12), rng.uniform(0.5, 2.5, 12)], 1)[None]
    eta = 1e-2
    out = oracle_mod.refine(g, cost, np.zeros((1, 12)), xy, steps=1, eta=eta, lam=0.0)
    expect = xy.astype(np.float32).astype(np.float64).copy()
    expect[0, 1:-1] -= eta * np.array([a, b])
    np.testing.assert_allclose(out[0, 1:-1], expect[0, 1:-1], rtol=0, atol=1e-6)
    np.testing.assert_array_equal(out[0, [0, -1]], xy[0, [0, -1]])


def test_refinement_is_translation_invariant_without_cost(oracle_mod):
    H = W = 40
    g = _grid(oracle_mod, H, W)
    cost = np.zeros((1, H, W), np.float32)
    rng = np.random.default_rng(4)
    xy = np.stack([np.linspace(0.5, 2.5, 20), 1.0 + rng.normal(0, 0.1, 20)], 1)[None]
    shift = np.array([0.75, 1.25])
    a = oracle_mod.refine(g, cost, np.zeros((1, 20)), xy, steps=5, eta=1e-2, lam=1.0)
    b = oracle_mod.refine(g, cost, np.zeros((1, 20)), xy + shift, steps=5, eta=1e-2, lam=1.0)
    np.testing.assert_allclose(b - shift, a, atol=1e-9)
