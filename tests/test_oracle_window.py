"""The window decomposition the full-size parity tests rely on: the oracle
run on a window plus its halo of 1 + R_p + R_K cells gives, on the window's
core, exactly the elevations, costs, masks and fragile flags of the oracle
run on the whole map (Sec. III-A bins per cell; Eq. 2-6 reach no further
than the halo).  A halo of R_K / 2 cells must change some core costs: the
off-map stencil makes the window's border cells barriers, whose inflation
then reaches the core, so the comparison does see a window cut too tight."""
import numpy as np
import pytest

from conftest import PARAMS_ROBOT

import _windows as W


@pytest.fixture(scope="module")
def small_cave(oracle_mod):
    from paper_2403_07631_gb300 import scenes
    sc = scenes.cave_terrain(seed=21, n_points=300_000, side_cells=160, res=0.05,
                             n_tunnels=3, n_shelves=40)
    sc.n_slices = 40
    b, _ = oracle_mod.bounds(sc.points)
    z_min = float(np.float32(b[2]))
    g = oracle_mod.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, z_min, sc.n_slices)
    eG, eC, _, _, _ = oracle_mod.build(sc.points, g, zmin_from_data=False)
    op = {k: PARAMS_ROBOT[k] for k in oracle_mod.PARAM_FIELDS}
    cT, mask, frag = oracle_mod.evaluate(g, op, eG, eC)
    return sc, z_min, dict(eG=eG, eC=eC, cT=cT, mask=mask, frag=frag)


@pytest.mark.parametrize("ci,cj", [(0, 0), (40, 57), (160 - 24, 160 - 24), (70, 0)])
def test_window_equals_full_map(small_cave, ci, cj):
    sc, z_min, full = small_cave
    hal = W.halo(PARAMS_ROBOT, sc.res)
    assert hal == 12 + 2 + 1
    ij = W.cells(sc.points, sc.x0, sc.y0, sc.res)
    box, core = W.window_bounds(ci, cj, 24, hal, sc.H, sc.W)
    got = W.oracle_window(sc.points, ij, box, sc.res, sc.d_s, z_min, sc.n_slices, PARAMS_ROBOT)
    i_lo, i_hi, j_lo, j_hi = box
    win = (slice(None), slice(i_lo, i_hi), slice(j_lo, j_hi))
    for name, a in zip(("eG", "eC"), got[:2]):
        np.testing.assert_array_equal(a, full[name][win], err_msg=name)
    for name, a in zip(("cT", "mask", "frag"), got[2:]):
        np.testing.assert_array_equal(a[core], full[name][win][core], err_msg=name)


def test_narrower_halo_changes_some_core_cost(small_cave):
    sc, z_min, full = small_cave
    hal = (W.halo(PARAMS_ROBOT, sc.res) - PARAMS_ROBOT["patch_radius"] - 1) // 2
    ij = W.cells(sc.points, sc.x0, sc.y0, sc.res)
    changed = 0
    rng = np.random.default_rng(0)
    for _ in range(6):
        ci, cj = (int(v) for v in rng.integers(hal, 160 - 24 - hal, 2))
        box, core = W.window_bounds(ci, cj, 24, hal, sc.H, sc.W)
        got = W.oracle_window(sc.points, ij, box, sc.res, sc.d_s, z_min, sc.n_slices,
                              PARAMS_ROBOT)
        i_lo, i_hi, j_lo, j_hi = box
        win = (slice(None), slice(i_lo, i_hi), slice(j_lo, j_hi))
        changed += int((got[2][core] != full["cT"][win][core]).sum())
    assert changed > 0
