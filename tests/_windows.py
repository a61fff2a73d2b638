"""Cutting a window out of a map for the oracle.

The cost of a cell depends on the elevations within 1 + R_p + R_K cells of
it (Eq. 2 gradient stencil, the p_s patch of Eq. 4, the inflation window of
Eq. 6), and its elevations only on the points of that cell (Sec. III-A).
So the oracle run on a window plus a halo of that width gives the core of
the window exactly as a run on the whole map would.  Points are rasterized
on the full grid and moved to the centres of the same cells of the window's
own grid, so that no rounding of the rasterization can move them.
"""
import numpy as np

import oracle


def cells(points, x0, y0, res):
    """Full-grid (row, column) of every point: floor(fl32(fl32(x - x0) / r_g))."""
    r = np.float32(res)
    j = np.floor((points[:, 0] - np.float32(x0)) / r).astype(np.int64)
    i = np.floor((points[:, 1] - np.float32(y0)) / r).astype(np.int64)
    return i, j


def halo(params, res):
    return (oracle.kernel(params, res).shape[0] - 1) // 2 + params["patch_radius"] + 1


def window_points(points, ij, i_lo, i_hi, j_lo, j_hi, res):
    """Points of cells [i_lo, i_hi) x [j_lo, j_hi), at the centres of the same
    cells of a grid with origin (0, 0) at cell (i_lo, j_lo)."""
    i, j = ij
    sel = (i >= i_lo) & (i < i_hi) & (j >= j_lo) & (j < j_hi)
    r = np.float64(res)
    out = np.empty((int(sel.sum()), 3), np.float32)
    out[:, 0] = (j[sel] - j_lo + 0.5) * r
    out[:, 1] = (i[sel] - i_lo + 0.5) * r
    out[:, 2] = points[sel, 2]
    return out


def window_bounds(ci, cj, core, hal, H, W):
    """The window with core [ci, ci+core) x [cj, cj+core) and its halo, clipped
    to the map, and the core's slices within it."""
    i_lo, j_lo = max(ci - hal, 0), max(cj - hal, 0)
    i_hi, j_hi = min(ci + core + hal, H), min(cj + core + hal, W)
    core_sl = (slice(None), slice(ci - i_lo, ci - i_lo + core), slice(cj - j_lo, cj - j_lo + core))
    return (i_lo, i_hi, j_lo, j_hi), core_sl


def oracle_window(points, ij, box, res, d_s, z_min, n_slices, params):
    """(eG, eC, cT, mask, fragile) of the window box = (i_lo, i_hi, j_lo, j_hi)."""
    i_lo, i_hi, j_lo, j_hi = box
    pts = window_points(points, ij, i_lo, i_hi, j_lo, j_hi, res)
    og = oracle.Grid(0.0, 0.0, res, j_hi - j_lo, i_hi - i_lo, d_s, z_min, n_slices)
    eG, eC, _, dropped, _ = oracle.build(pts, og, zmin_from_data=False)
    assert dropped == 0
    op = {k: params[k] for k in oracle.PARAM_FIELDS}
    cT, mask, frag = oracle.evaluate(og, op, eG, eC)
    return eG, eC, cT, mask, frag
