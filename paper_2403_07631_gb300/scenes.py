"""Seeded synthetic point clouds shaped like the paper's scenes.

The paper's own maps (factory, building, forest, overpass, stairs, boxes,
spiral; Sec. IV-A) are not available, so these generators stand in for them:
multi-storey buildings with ramps, walls and overhangs, a parking structure
with a helical ramp, pillars and beams, and fractal cave terrain.

This module holds no arithmetic of the method (no rasterisation, no slices,
no costs).  It only draws points on surfaces from a seeded numpy generator,
and it is the one module both the CUDA path's callers and the oracle tests
take their inputs from.

Horizontal walkable surfaces are sampled with jittered stratification (one
point uniformly placed inside each 0.1 m cell, with a given cell coverage) so
that floors are dense enough to be traversable, as the paper requires of its
maps (Sec. V: the method needs a dense point cloud); everything else is
sampled uniformly at random on its surface.  Noise is Gaussian along the
surface normal.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Scene:
    """A synthetic cloud and the grid it is meant to be tomographed on."""
    name: str
    points: np.ndarray            # [P, 3] float32
    x0: float
    y0: float
    res: float
    W: int
    H: int
    d_s: float
    n_slices: int                 # 0: derive N from the cloud's height range
    meta: dict = field(default_factory=dict)


# ---------------------------------------------------------------- primitives

def _strat_rect(rng, x0, y0, nx, ny, res, z, sigma, coverage=1.0, keep=None):
    """Jittered stratified samples: one point per kept cell of an nx*ny block."""
    jj, ii = np.meshgrid(np.arange(nx), np.arange(ny))
    jj = jj.ravel()
    ii = ii.ravel()
    x = x0 + (jj + rng.random(jj.size)) * res
    y = y0 + (ii + rng.random(ii.size)) * res
    sel = np.ones(x.size, bool)
    if coverage < 1.0:
        sel &= rng.random(x.size) < coverage
    if keep is not None:
        sel &= keep(x, y)
    x, y = x[sel], y[sel]
    zz = (z(x, y) if callable(z) else np.full(x.size, z)) + rng.normal(0.0, sigma, x.size)
    return np.stack([x, y, zz], 1)


def _rand_rect_h(rng, n, x0, y0, sx, sy, z, sigma, keep=None):
    """n uniform points on a horizontal rectangle (rejection for `keep`)."""
    out = []
    need = n
    while need > 0:
        m = int(need * 1.3) + 16
        x = x0 + rng.random(m) * sx
        y = y0 + rng.random(m) * sy
        if keep is not None:
            s = keep(x, y)
            x, y = x[s], y[s]
        x, y = x[:need], y[:need]
        zz = (z(x, y) if callable(z) else np.full(x.size, z)) + rng.normal(0.0, sigma, x.size)
        out.append(np.stack([x, y, zz], 1))
        need -= x.size
    return np.concatenate(out) if out else np.zeros((0, 3))


def _rand_wall(rng, n, p0, p1, z0, z1, sigma):
    """n uniform points on the vertical rectangle above segment p0-p1."""
    t = rng.random(n)
    z = z0 + rng.random(n) * (z1 - z0)
    p0 = np.asarray(p0, float)
    p1 = np.asarray(p1, float)
    d = p1 - p0
    nrm = np.array([-d[1], d[0]]) / max(np.hypot(*d), 1e-12)
    off = rng.normal(0.0, sigma, n)
    x = p0[0] + t * d[0] + off * nrm[0]
    y = p0[1] + t * d[1] + off * nrm[1]
    return np.stack([x, y, z], 1)


def _rand_box_sides(rng, n, cx, cy, hx, hy, z0, z1, sigma):
    """n points on the four vertical faces of an axis-aligned box."""
    w = np.array([hx, hy, hx, hy], float)
    per = rng.multinomial(n, w / w.sum())
    c = [(cx - hx, cy - hy), (cx + hx, cy - hy), (cx + hx, cy + hy), (cx - hx, cy + hy)]
    parts = [_rand_wall(rng, per[s], c[s], c[(s + 1) % 4], z0, z1, sigma) for s in range(4)]
    return np.concatenate(parts)


def _finish(rng, parts, n_points, topup):
    pts = np.concatenate([p for p in parts if len(p)])
    if len(pts) > n_points:
        pts = pts[np.sort(rng.choice(len(pts), n_points, replace=False))]
    elif len(pts) < n_points:
        pts = np.concatenate([pts, topup(n_points - len(pts))])
    return np.ascontiguousarray(pts, dtype=np.float32)


# ------------------------------------------------------- multi-storey building

def building(seed: int, n_points: int, side_cells: int = 200, res: float = 0.1,
             floors: list[float] | None = None, ceilings: list[float] | None = None,
             ramp_deg: float = 15.0, sigma: float = 0.01, wall_height: float | None = None,
             name: str = "building") -> Scene:
    """A square building: floor slabs (tops at `floors`), slab undersides or a
    roof at `ceilings`, four outer walls, and one straight ramp of `ramp_deg`
    from each floor to the next through an opening in the upper slab."""
    rng = np.random.default_rng(seed)
    L = side_cells * res
    floors = [0.0, 3.0] if floors is None else floors
    ceilings = [2.8, 5.8] if ceilings is None else ceilings
    top = max(ceilings + floors)
    wall_height = top if wall_height is None else wall_height
    # ramps: straight, 2 m wide (or narrower on small maps), along +x
    ramps = []
    for f in range(len(floors) - 1):
        rise = floors[f + 1] - floors[f]
        run = rise / math.tan(math.radians(ramp_deg))
        width = min(2.0, 0.15 * L)
        run = min(run, 0.8 * L)
        x_start = 0.1 * L
        y_start = 0.1 * L + (f % 3) * (width + 0.05 * L)
        y_start = min(y_start, L - width - 0.05 * L)
        ramps.append((x_start, y_start, run, width, floors[f], rise))

    def outside_openings(level_z):
        # the slab whose top is level_z has an opening above every ramp arriving at it
        rs = [r for r in ramps if abs(r[4] + r[5] - level_z) < 1e-9]

        def keep(x, y):
            ok = np.ones(x.size, bool)
            for (xs, ys, run, wd, _, _) in rs:
                ok &= ~((x >= xs) & (x < xs + run) & (y >= ys) & (y < ys + wd))
            return ok
        return keep

    def slab_openings(ceiling_z):
        # a slab underside just below a floor shares that floor's openings
        above = [fz for fz in floors if 0.0 < fz - ceiling_z <= 0.5]
        return outside_openings(above[0]) if above else None

    parts = []
    n_floor_cells = side_cells * side_cells
    for fz in floors:
        parts.append(_strat_rect(rng, 0.0, 0.0, side_cells, side_cells, res, fz, sigma,
                                 keep=outside_openings(fz)))
    for (xs, ys, run, wd, z0, rise) in ramps:
        nx, ny = max(1, int(round(run / res))), max(1, int(round(wd / res)))
        slope = rise / run
        parts.append(_strat_rect(rng, xs, ys, nx, ny, res,
                                 lambda x, y, xs=xs, z0=z0, s=slope: z0 + (x - xs) * s, sigma))
    used = sum(len(p) for p in parts)
    rest = max(0, n_points - used)
    ceil_area = len(ceilings) * L * L
    wall_area = 4 * L * wall_height
    n_ceil = int(rest * ceil_area / (ceil_area + wall_area))
    n_wall = rest - n_ceil
    for cz in ceilings:
        parts.append(_rand_rect_h(rng, n_ceil // len(ceilings), 0.0, 0.0, L, L, cz, sigma,
                                  keep=slab_openings(cz)))
    e = 0.2 * res
    corners = [(e, e), (L - e, e), (L - e, L - e), (e, L - e)]
    per = rng.multinomial(n_wall, [0.25] * 4)
    for s in range(4):
        parts.append(_rand_wall(rng, per[s], corners[s], corners[(s + 1) % 4],
                                min(floors) - 0.05, wall_height, sigma))

    def topup(m):
        return _rand_rect_h(rng, m, 0.0, 0.0, L, L, floors[0], sigma)

    pts = _finish(rng, parts, n_points, topup)
    return Scene(name, pts, 0.0, 0.0, res, side_cells, side_cells, 0.5, 0,
                 dict(seed=seed, floors=floors, ceilings=ceilings, ramp_deg=ramp_deg,
                      n_floor_cells=n_floor_cells))


def two_storey_building(seed: int = 1, n_points: int = 200_000) -> Scene:
    """Two-storey building over 20 x 20 m: floors z=0 and 3, ceilings 2.8 and
    5.8, four walls, one 15 deg ramp, sigma 0.01 m; grid 200 x 200 at 0.1 m,
    d_s = 0.5 and N derived from the cloud (12 slices)."""
    return building(seed, n_points, 200, 0.1, [0.0, 3.0], [2.8, 5.8], 15.0, 0.01,
                    name="two-storey building 200k pts, 200x200 @0.1 m")


# ---------------------------------------------------------- parking structure

def parking_structure(seed: int = 2, n_points: int = 5_000_000, side_cells: int = 1000,
                      res: float = 0.1, n_pillars: int = 400, n_beams: int = 300) -> Scene:
    """Five-level parking structure over 100 x 100 x 20 m: floor tops every
    4 m with 0.3 m slabs, a helical ramp (radius 15 m, 8 deg) around the
    centre, box pillars through all levels, overhanging beams 1.6-2.4 m above
    the floors, sigma 0.02 m; grid 1000 x 1000 at 0.1 m, 40 slices."""
    rng = np.random.default_rng(seed)
    L = side_cells * res
    sigma = 0.02
    levels = [0.0, 4.0, 8.0, 12.0, 16.0]
    cx = cy = L / 2
    R_in, R_out = 13.5, 16.5
    rise = 4.0
    run = rise / math.tan(math.radians(8.0))
    span = run / 15.0                      # radians of helix per level at r = 15 m

    def sector(level):                     # angular sector of the ramp arriving at level
        f = levels.index(level) - 1
        a0 = (f * span) % (2 * math.pi)
        return a0, span

    def in_sector(x, y, a0, sp):
        r = np.hypot(x - cx, y - cy)
        a = (np.arctan2(y - cy, x - cx) - a0) % (2 * math.pi)
        return (r >= R_in) & (r < R_out) & (a < sp)

    pillars = []
    while len(pillars) < n_pillars:
        px, py = rng.random(2) * (L - 2.0) + 1.0
        if abs(math.hypot(px - cx, py - cy) - 15.0) < 3.0:
            continue
        pillars.append((px, py, rng.uniform(0.2, 0.4), rng.uniform(0.2, 0.4)))
    pill = np.array(pillars)

    def floor_keep(level):
        def keep(x, y):
            ok = np.ones(x.size, bool)
            if level > 0.0:
                a0, sp = sector(level)
                ok &= ~in_sector(x, y, a0, sp)
            return ok
        return keep

    parts = []
    coverage = {0.0: 1.0, 4.0: 1.0, 8.0: 1.0, 12.0: 0.5, 16.0: 0.5}
    for lv in levels:
        parts.append(_strat_rect(rng, 0.0, 0.0, side_cells, side_cells, res, lv, sigma,
                                 coverage=coverage[lv], keep=floor_keep(lv)))
    # helical ramp between consecutive levels
    n_ramp_cells = int(round((math.pi * (R_out ** 2 - R_in ** 2)) / (res * res)))
    for f in range(len(levels) - 1):
        a0 = (f * span) % (2 * math.pi)
        jx0 = int((cx - R_out) / res)
        nx = int(2 * R_out / res) + 1

        def zf(x, y, a0=a0, z0=levels[f]):
            a = (np.arctan2(y - cy, x - cx) - a0) % (2 * math.pi)
            return z0 + rise * a / span

        parts.append(_strat_rect(rng, jx0 * res, jx0 * res, nx, nx, res, zf, sigma,
                                 keep=lambda x, y, a0=a0: in_sector(x, y, a0, span)))
    del n_ramp_cells
    # slab undersides of the upper levels
    for lv in levels[1:]:
        parts.append(_rand_rect_h(rng, side_cells * side_cells // 10, 0.0, 0.0, L, L, lv - 0.3, sigma,
                                  keep=floor_keep(lv)))
    # pillars through all levels
    per = rng.multinomial(875 * len(pill), np.ones(len(pill)) / len(pill))
    for (px, py, hx, hy), m in zip(pill, per):
        parts.append(_rand_box_sides(rng, m, px, py, hx, hy, 0.0, 16.0, sigma))
    # overhanging beams: undersides 1.6-2.4 m above a floor, 0.3 m wide, 4-12 m long
    per = rng.multinomial(500 * n_beams, np.ones(n_beams) / n_beams)
    for m in per:
        lv = levels[rng.integers(0, 4)]
        z = lv + rng.uniform(1.6, 2.4)
        ln = rng.uniform(4.0, 12.0)
        if rng.random() < 0.5:
            x0, y0, sx, sy = rng.uniform(0, L - ln), rng.uniform(0, L - 0.3), ln, 0.3
        else:
            x0, y0, sx, sy = rng.uniform(0, L - 0.3), rng.uniform(0, L - ln), 0.3, ln
        parts.append(_rand_rect_h(rng, m, x0, y0, sx, sy, z, sigma))

    def topup(m):
        return _rand_rect_h(rng, m, 0.0, 0.0, L, L, 16.0, sigma, keep=floor_keep(16.0))

    pts = _finish(rng, parts, n_points, topup)
    name = f"parking structure {n_points / 1e6:g}M pts, {side_cells}x{side_cells} @{res:g} m, 40 slices"
    return Scene(name, pts, 0.0, 0.0, res,
                 side_cells, side_cells, 0.5, 40,
                 dict(seed=seed, levels=levels, n_pillars=n_pillars, n_beams=n_beams))


# ------------------------------------------------------------- batched maps

def batched_maps(seed_base: int = 3000, count: int = 64, p_lo: int = 50_000,
                 p_hi: int = 4_000_000, side_lo: int = 128, side_hi: int = 1024) -> list[Scene]:
    """Many independent buildings of uneven size: points log-uniform in
    [p_lo, p_hi], grid side log-uniform in [side_lo, side_hi] at 0.1 m, slice
    counts uniform in 4..48, 1-5 floors, ramps U(5, 25) deg and ceiling gaps
    U(0.4, 3) m."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed_base + i)
        n_pts = int(round(math.exp(rng.uniform(math.log(p_lo), math.log(p_hi)))))
        side = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        n_sl = int(rng.integers(4, 49))
        n_fl = int(rng.integers(1, 6))
        floors, ceilings = [], []
        z = 0.0
        for f in range(n_fl):
            floors.append(round(z, 3))
            gap = float(rng.uniform(0.4, 3.0))
            ceilings.append(round(z + gap, 3))
            z = z + gap + 0.2
        ramp = float(rng.uniform(5.0, 25.0))
        sc = building(seed_base + i, n_pts, side, 0.1, floors, ceilings, ramp, 0.01,
                      name=f"map {i}")
        sc.n_slices = n_sl
        out.append(sc)
    return out


# ------------------------------------------------------------- cave terrain

def _value_noise(rng, x, y, spacing, extent):
    """Smooth noise in [-1, 1]: random values on a lattice `spacing` apart,
    interpolated with a smoothstep."""
    n = int(math.ceil(extent / spacing)) + 2
    lat = rng.uniform(-1.0, 1.0, (n, n))
    u, v = x / spacing, y / spacing
    i0 = np.clip(np.floor(v).astype(np.int64), 0, n - 2)
    j0 = np.clip(np.floor(u).astype(np.int64), 0, n - 2)
    fu, fv = u - j0, v - i0
    su, sv = fu * fu * (3 - 2 * fu), fv * fv * (3 - 2 * fv)
    a = lat[i0, j0] * (1 - su) + lat[i0, j0 + 1] * su
    b = lat[i0 + 1, j0] * (1 - su) + lat[i0 + 1, j0 + 1] * su
    return a * (1 - sv) + b * sv


def _fractal(seed, x, y, extent, amplitude, octaves=5, base=50.0):
    rng = np.random.default_rng(seed)
    z = np.zeros_like(x)
    amp, spacing, total = 1.0, base, 0.0
    for _ in range(octaves):
        z += amp * _value_noise(rng, x, y, spacing, extent)
        total += amp
        amp *= 0.5
        spacing *= 0.5
    return amplitude * z / total


def cave_terrain(seed: int = 5, n_points: int = 60_000_000, side_cells: int = 4000,
                 res: float = 0.05, n_tunnels: int = 30, n_shelves: int = 2000) -> Scene:
    """Multi-layer terrain over 200 x 200 x 40 m: fractal value-noise ground
    (5 octaves, amplitude 6 m) sampled once per 0.05 m cell, cave tunnels
    beneath it as noise-perturbed tubes of radius 2-4 m, and overhanging rock
    shelves 1-3.5 m above the ground; grid 4000 x 4000 at 0.05 m, 80 slices."""
    rng = np.random.default_rng(seed)
    L = side_cells * res
    sigma = 0.02

    def ground(x, y):
        return 20.0 + _fractal(seed, x, y, L, 6.0)

    parts = [_strat_rect(rng, 0.0, 0.0, side_cells, side_cells, res, ground, sigma)]
    n_ground = len(parts[0])
    # shelves: horizontal undersides above the local ground
    shelf_area = []
    shelves = []
    for _ in range(n_shelves):
        sx, sy = rng.uniform(1.0, 4.0), rng.uniform(0.5, 2.0)
        x0, y0 = rng.uniform(0, L - sx), rng.uniform(0, L - sy)
        z = float(ground(np.array([x0 + sx / 2]), np.array([y0 + sy / 2]))[0]) + rng.uniform(1.0, 3.5)
        shelves.append((x0, y0, sx, sy, z))
        shelf_area.append(sx * sy)
    n_shelf_pts = int(min(4_000_000, 0.07 * n_points))
    per = rng.multinomial(n_shelf_pts, np.array(shelf_area) / np.sum(shelf_area))
    for (x0, y0, sx, sy, z), m in zip(shelves, per):
        parts.append(_rand_rect_h(rng, m, x0, y0, sx, sy, z, sigma))
    # tunnels: tubes along noise-perturbed paths 6-10 m below the ground, as
    # long as 0.5-1.25 map sides (100-250 m on the 200 m map)
    n_tun_pts = max(0, n_points - n_ground - n_shelf_pts)
    lengths = rng.uniform(0.5 * L, 1.25 * L, n_tunnels)
    radii = rng.uniform(2.0, 4.0, n_tunnels)
    area = 2 * math.pi * radii * lengths
    per = rng.multinomial(n_tun_pts, area / area.sum())
    tunnel_points = []
    for t in range(n_tunnels):
        m = int(per[t])
        if m == 0:
            continue
        sx, sy = rng.uniform(0.05 * L, 0.95 * L, 2)
        head = rng.uniform(0, 2 * math.pi)
        depth = rng.uniform(6.0, 10.0)
        # centre line sampled every 0.5 m with a slowly wandering heading
        ns = int(lengths[t] / 0.5) + 1
        turn = np.cumsum(rng.normal(0.0, 0.05, ns))
        hx, hy = np.cos(head + turn), np.sin(head + turn)
        cx = np.clip(sx + np.cumsum(hx) * 0.5, 1.0, L - 1.0)
        cy = np.clip(sy + np.cumsum(hy) * 0.5, 1.0, L - 1.0)
        cz = ground(cx, cy) - depth
        tunnel_points.append((float(cx[ns // 2]), float(cy[ns // 2])))
        k = rng.integers(0, ns, m)
        phi = rng.uniform(0.0, 2 * math.pi, m)
        r = radii[t] * (1.0 + 0.15 * rng.uniform(-1.0, 1.0, m))
        nx, ny = -hy[k], hx[k]
        x = cx[k] + r * np.cos(phi) * nx
        y = cy[k] + r * np.cos(phi) * ny
        z = cz[k] + r * np.sin(phi) + rng.normal(0.0, sigma, m)
        parts.append(np.stack([x, y, z], 1).astype(np.float32))

    def topup(m):
        return _rand_rect_h(rng, m, 0.0, 0.0, L, L, ground, sigma)

    pts = _finish(rng, [p.astype(np.float32) for p in parts], n_points, topup)
    return Scene(f"cave terrain {n_points / 1e6:g}M pts, {side_cells}x{side_cells} @{res:g} m, 80 slices",
                 pts, 0.0, 0.0, res, side_cells, side_cells, 0.5, 80,
                 dict(seed=seed, n_tunnels=n_tunnels, n_shelves=n_shelves,
                      tunnel_points=tunnel_points))


# ------------------------------------------------------------ query paths

def straight_paths(walkable: np.ndarray, x0: float, y0: float, res: float, paths: int = 256,
                   length: int = 512, seed: int = 4, noise: float = 0.2) -> np.ndarray:
    """Waypoint paths for the cost queries: `paths` straight lines of `length`
    waypoints between random cells of the boolean [H, W] map `walkable`
    (cell centres), the interior waypoints jittered by N(0, noise) metres.
    Returns float32 [paths, length, 2] world (x, y)."""
    rng = np.random.default_rng(seed)
    H, W = walkable.shape
    cells = np.flatnonzero(walkable.reshape(-1))
    if len(cells) == 0:
        raise ValueError("no walkable cell to start or end a path on")
    pick = cells[rng.integers(0, len(cells), (paths, 2))]
    ends = np.stack([x0 + (pick % W + 0.5) * res, y0 + (pick // W + 0.5) * res], -1)
    t = np.linspace(0.0, 1.0, length)[None, :, None]
    xy = ends[:, :1] * (1 - t) + ends[:, 1:] * t
    xy[:, 1:-1] += noise * rng.standard_normal((paths, length - 2, 2))
    return xy.astype(np.float32)
