"""GPU parity of the cost / elevation queries and their adjoint (the C(q),
e^G(q) of Eq. 10) and of the fused path refinement, against the FP64
oracle and FP64 central finite differences (h = 1e-4 m).

Tolerances (mixed, because a bilinear value or gradient inherits the
float32 rounding of its largest corner): values |v - v*| <= 1e-5 * max(|v*|,
S); gradients |g - g*| <= 1e-5 * max(|g*|, S / r_g), with S = c^B for costs
and the largest |z| of the map for elevations.
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


@pytest.fixture(scope="module")
def tomogram():
    build.build()
    oracle.compile_library()
    sc = scenes.building(61, 80_000, side_cells=120, floors=[0.0, 2.2], ceilings=[2.0, 4.4])
    grid = tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, 10, 0.0, True)
    g = P.gpu_build_evaluate(sc.points, grid, PARAMS_ROBOT)
    z_min = float(sc.points[:, 2].min())
    grid = tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, 10, z_min, True)
    og = oracle.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, z_min, 10)
    return grid, og, g["cost"], g["ground"]


def _queries(grid, n, seed, margin=0.3):
    rng = np.random.default_rng(seed)
    xy = np.stack([rng.uniform(grid.x0 - margin, grid.x0 + grid.W * grid.res + margin, n),
                   rng.uniform(grid.y0 - margin, grid.y0 + grid.H * grid.res + margin, n)],
                  1).astype(np.float32)
    sl = rng.integers(0, grid.n_slices, n).astype(np.int32)
    return xy, sl


def _dev(*a):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


def _close(a, b, scale, what):
    err = np.abs(a.astype(np.float64) - b)
    lim = RTOL * np.maximum(np.abs(b), scale)
    bad = ~(err <= lim)
    assert not bad.any(), f"{what}: {int(bad.sum())} out of tolerance, max err {err[bad].max()}"


def test_forward_matches_oracle(tomogram):
    grid, og, cost, ground = tomogram
    xy, sl = _queries(grid, 50_000, 1)
    d_xy, d_sl, d_c, d_g = _dev(xy, sl, cost, ground)
    c_out = torch.empty(len(xy), device="cuda")
    e_out = torch.empty(len(xy), device="cuda")
    tct.tct_sample_cost(grid, d_c, d_g, d_xy, d_sl, c_out, e_out)
    torch.cuda.synchronize()
    rc, _ = oracle.sample(og, cost, xy, sl)
    re, _ = oracle.sample(og, ground, xy, sl, is_ground=True)
    zmax = float(np.abs(ground[np.isfinite(ground)]).max())
    _close(c_out.cpu().numpy(), rc, PARAMS_ROBOT["c_b"], "cost")
    _close(e_out.cpu().numpy(), re, max(zmax, 1.0), "elevation")


def test_backward_matches_oracle_gradient(tomogram):
    grid, og, cost, ground = tomogram
    xy, sl = _queries(grid, 50_000, 2)
    rng = np.random.default_rng(3)
    wc = rng.normal(size=len(xy)).astype(np.float32)
    we = rng.normal(size=len(xy)).astype(np.float32)
    d_xy, d_sl, d_c, d_g, d_wc, d_we = _dev(xy, sl, cost, ground, wc, we)
    gxy = torch.empty_like(d_xy)
    tct.tct_sample_cost_backward(grid, d_c, d_g, d_xy, d_sl, d_wc, d_we, gxy)
    torch.cuda.synchronize()
    _, gc = oracle.sample(og, cost, xy, sl)
    _, ge = oracle.sample(og, ground, xy, sl, is_ground=True)
    ref = wc[:, None].astype(np.float64) * gc + we[:, None].astype(np.float64) * ge
    zmax = float(np.abs(ground[np.isfinite(ground)]).max())
    scale = (np.abs(wc) * PARAMS_ROBOT["c_b"] + np.abs(we) * max(zmax, 1.0))[:, None] / grid.res
    _close(gxy.cpu().numpy(), ref, scale, "gradient")


def test_gradient_against_central_differences(tomogram):
    grid, og, cost, _ = tomogram
    xy, sl = _queries(grid, 20_000, 4, margin=-0.2)
    h = 1e-4
    u = (xy.astype(np.float64) - [grid.x0, grid.y0]) / grid.res - 0.5
    ok = (np.abs(u - np.round(u)) > 2 * h / grid.res).all(1)
    xy, sl = xy[ok], sl[ok]
    d_xy, d_sl, d_c = _dev(xy, sl, cost)
    ones = torch.ones(len(xy), device="cuda")
    gxy = torch.empty_like(d_xy)
    tct.tct_sample_cost_backward(grid, d_c, None, d_xy, d_sl, ones, None, gxy)
    torch.cuda.synchronize()
    fd = np.zeros((len(xy), 2))
    x64 = xy.astype(np.float64)
    for a in range(2):
        e = np.zeros(2)
        e[a] = h
        vp, _ = oracle.sample_f64(og, cost, x64 + e, sl)
        vm, _ = oracle.sample_f64(og, cost, x64 - e, sl)
        fd[:, a] = (vp - vm) / (2 * h)
    # FP64 differences at FP64 coordinates: exact up to FP64 rounding away
    # from lattice lines, so the bound is the sampler's own 1e-5 tolerance
    _close(gxy.cpu().numpy(), fd, PARAMS_ROBOT["c_b"] / grid.res, "finite differences")


def test_autograd_function(tomogram):
    grid, og, cost, ground = tomogram
    xy, sl = _queries(grid, 4096, 5)
    d_xy, d_sl, d_c, d_g = _dev(xy, sl, cost, ground)
    d_xy.requires_grad_(True)
    c, e = tct.sample_cost(d_xy, d_sl, d_c, d_g, grid)
    (c.sum() + 2.0 * e.sum()).backward()
    _, gc = oracle.sample(og, cost, xy, sl)
    _, ge = oracle.sample(og, ground, xy, sl, is_ground=True)
    zmax = float(np.abs(ground[np.isfinite(ground)]).max())
    _close(d_xy.grad.cpu().numpy(), gc + 2.0 * ge, (PARAMS_ROBOT["c_b"] + 2 * zmax) / grid.res,
           "autograd")


def test_bad_queries_are_flagged(tomogram):
    grid, og, cost, ground = tomogram
    xy = np.array([[1.0, 1.0], [np.nan, 1.0], [1.0, 1.0]], np.float32)
    sl = np.array([0, 0, grid.n_slices], np.int32)
    d_xy, d_sl, d_c, d_g = _dev(xy, sl, cost, ground)
    out = torch.empty(3, device="cuda")
    stats = torch.zeros(tct.STATS_BYTES, dtype=torch.uint8, device="cuda")
    tct.tct_sample_cost(grid, d_c, d_g, d_xy, d_sl, out, None, stats)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.isfinite(o[0]) and np.isnan(o[1]) and np.isnan(o[2])
    assert tct.stats_from(stats).status & tct.DEV_BAD_QUERY


def test_refinement_smooth_bowl_matches_oracle():
    H = W = 60
    ii = np.arange(H)[:, None] + np.zeros((1, W))
    cost = (5.0 * ((ii + 0.5) * 0.1 - 3.0) ** 2).astype(np.float32)[None]
    grid = tct.Grid(0.0, 0.0, 0.1, W, H, 0.5, 1, 0.0, False)
    og = oracle.Grid(0.0, 0.0, 0.1, W, H, 0.5, 0.0, 1)
    rng = np.random.default_rng(6)
    paths, L = 16, 200
    xs = np.linspace(0.5, 5.5, L)
    xy = np.stack([np.broadcast_to(xs, (paths, L)),
                   3.0 + rng.normal(0, 0.3, (paths, L))], 2).astype(np.float32)
    sl = np.zeros((paths, L), np.int32)
    d_xy, d_sl, d_c = _dev(xy, sl, cost)
    tct.tct_refine_paths(grid, d_c, d_sl, d_xy, steps=50, eta=1e-3, lam=1.0)
    torch.cuda.synchronize()
    ref = oracle.refine(og, cost, sl, xy, steps=50, eta=1e-3, lam=1.0)
    got = d_xy.cpu().numpy()
    np.testing.assert_allclose(got, ref, atol=2e-5)
    # descent: the objective went down on every path
    assert np.all(np.abs(got[:, 1:-1, 1] - 3.0).mean(1) < np.abs(xy[:, 1:-1, 1] - 3.0).mean(1))


def test_refinement_on_tomogram_few_steps(tomogram):
    grid, og, cost, _ = tomogram
    rng = np.random.default_rng(7)
    paths, L = 32, 128
    a = rng.uniform(1.0, grid.W * grid.res - 1.0, (paths, 2))
    b = rng.uniform(1.0, grid.W * grid.res - 1.0, (paths, 2))
    t = np.linspace(0, 1, L)[None, :, None]
    xy = (a[:, None] * (1 - t) + b[:, None] * t + rng.normal(0, 0.2, (paths, L, 2))).astype(np.float32)
    sl = np.broadcast_to(rng.integers(0, grid.n_slices, (paths, 1)), (paths, L)).astype(np.int32)
    d_xy, d_sl, d_c = _dev(xy, sl, cost)
    tct.tct_refine_paths(grid, d_c, d_sl, d_xy, steps=3, eta=1e-4, lam=1.0)
    torch.cuda.synchronize()
    ref = oracle.refine(og, cost, sl, xy, steps=3, eta=1e-4, lam=1.0)
    got = d_xy.cpu().numpy()
    # waypoints whose query stayed inside one lattice cell in both precisions agree tightly
    np.testing.assert_allclose(got, ref, atol=1e-4)


def test_refinement_edges(tomogram):
    """Zero steps and two-waypoint paths (both ends fixed) leave the paths as
    they are; the longest path (TCT_MAX_PATH_LEN waypoints) matches the
    oracle; too long and too short paths are refused."""
    grid, og, cost, _ = tomogram
    rng = np.random.default_rng(8)
    d_c = _dev(cost)[0]
    for paths, L, steps in ((4, 64, 0), (5, 2, 7)):
        xy = rng.uniform(1.0, 5.0, (paths, L, 2)).astype(np.float32)
        sl = np.zeros((paths, L), np.int32)
        d_xy, d_sl = _dev(xy, sl)
        tct.tct_refine_paths(grid, d_c, d_sl, d_xy, steps=steps, eta=1e-3, lam=1.0)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(d_xy.cpu().numpy(), xy)
    L = tct.MAX_PATH_LEN
    t = np.linspace(0.0, 1.0, L)[None, :, None]
    xy = (np.array([1.0, 1.0]) * (1 - t) + np.array([10.0, 9.0]) * t).astype(np.float32)
    xy[:, 1:-1] += rng.normal(0, 0.1, (1, L - 2, 2)).astype(np.float32)
    sl = np.full((1, L), 2, np.int32)
    d_xy, d_sl = _dev(xy, sl)
    tct.tct_refine_paths(grid, d_c, d_sl, d_xy, steps=2, eta=1e-4, lam=1.0)
    torch.cuda.synchronize()
    ref = oracle.refine(og, cost, sl, xy, steps=2, eta=1e-4, lam=1.0)
    np.testing.assert_allclose(d_xy.cpu().numpy(), ref, atol=1e-4)
    with pytest.raises(tct.TctError, match="limit"):
        big = torch.zeros(1, L + 1, 2, device="cuda")
        tct.tct_refine_paths(grid, d_c, torch.zeros(1, L + 1, dtype=torch.int32, device="cuda"),
                             big, steps=1, eta=1e-3, lam=1.0)
    with pytest.raises(tct.TctError, match="invalid"):
        one = torch.zeros(1, 1, 2, device="cuda")
        tct.tct_refine_paths(grid, d_c, torch.zeros(1, 1, dtype=torch.int32, device="cuda"), one,
                             steps=1, eta=1e-3, lam=1.0)
