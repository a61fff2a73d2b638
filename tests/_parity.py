"""Shared helpers of the GPU parity tests: run the CUDA path through the
C ABI and the FP64 oracle on the same seeded inputs, and compare.

Tolerances (written here once, used by every parity test):
- elevations (ground, ceiling) and every integer / byte output: bit-exact;
- costs: |gpu - oracle| <= 1e-5 * max(1, |oracle|) on cells whose cost the
  oracle marks as pinned (fragile bit 0 clear); float32 arithmetic on
  elevations of tens of metres leaves absolute errors near 1e-6 on costs of
  order 1-50, so the floor of 1 keeps costs near 0 from failing on rounding;
- traversable mask: exact on cells whose mask is pinned (fragile bit 1 clear);
- keep flags: exact against the oracle's chain run on the GPU's own layers
  (the decision in float32, as the kernel takes it), and exact against the
  oracle's own layers whenever the oracle reports the chain robust;
- fragile cells (left out of the cost and mask checks) must stay rare: every
  cost check also bounds their fraction by FRAGILE_MAX and prints it, so an
  oracle that marked too many cells fragile could not make a check vacuous.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2403_07631_gb300 import tct

COST_RTOL = 1e-5
FRAGILE_MAX = 1e-3


def oracle_params(p: dict) -> dict:
    return {k: p[k] for k in oracle.PARAM_FIELDS}


def gpu_build_evaluate(points: np.ndarray, grid: tct.Grid, params: dict, stride: int = 3,
                       misalign: bool = False):
    dev = torch.device("cuda")
    pts = torch.from_numpy(np.ascontiguousarray(points, np.float32))
    if stride == 4:
        pts = torch.cat([pts, torch.ones(len(pts), 1)], 1).contiguous()
    if misalign:
        # a buffer whose base is 4 bytes past a 16-byte boundary: scalar path
        buf = torch.empty(pts.numel() + 1, dtype=torch.float32, device=dev)
        buf[1:] = pts.reshape(-1).to(dev)
        pts_d = buf[1:].view(-1, pts.shape[1])
    else:
        pts_d = pts.to(dev)
    ws, ground, ceil, cost, mask, keep, stats = tct.alloc_outputs(grid, len(points), dev, params)
    tct.tct_build_evaluate(pts_d, grid, params, ws, ground, ceil, cost, mask, keep, stats)
    torch.cuda.synchronize()
    return dict(ground=ground.cpu().numpy(), ceil=ceil.cpu().numpy(), cost=cost.cpu().numpy(),
                mask=mask.cpu().numpy(), keep=keep.cpu().numpy(), stats=tct.stats_from(stats))


def gpu_build(points: np.ndarray, grid: tct.Grid, stride: int = 3):
    dev = torch.device("cuda")
    pts = torch.from_numpy(np.ascontiguousarray(points, np.float32))
    if stride == 4:
        pts = torch.cat([pts, torch.zeros(len(pts), 1)], 1).contiguous()
    pts = pts.to(dev)
    ws = torch.empty(tct.tct_workspace_bytes(grid, len(points)), dtype=torch.uint8, device=dev)
    ground = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    ceil = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    stats = torch.zeros(tct.STATS_BYTES, dtype=torch.uint8, device=dev)
    tct.tct_build(pts, grid, ws, ground, ceil, stats)
    torch.cuda.synchronize()
    return ground.cpu().numpy(), ceil.cpu().numpy(), tct.stats_from(stats)


def gpu_evaluate(eG: np.ndarray, eC: np.ndarray, grid: tct.Grid, params: dict, aux: bool = True):
    dev = torch.device("cuda")
    g = torch.from_numpy(np.ascontiguousarray(eG, np.float32)).to(dev)
    c = torch.from_numpy(np.ascontiguousarray(eC, np.float32)).to(dev)
    ws = torch.empty(tct.tct_workspace_bytes(grid, 0, params), dtype=torch.uint8, device=dev)
    cost = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    mask = torch.empty(grid.shape, dtype=torch.uint8, device=dev)
    keep = torch.empty(grid.n_slices, dtype=torch.uint8, device=dev)
    a = torch.full((5,) + grid.shape, float("nan"), dtype=torch.float32, device=dev) if aux else None
    stats = torch.zeros(tct.STATS_BYTES, dtype=torch.uint8, device=dev)
    tct.tct_evaluate(grid, params, g, c, ws, cost, mask, keep, a, stats)
    torch.cuda.synchronize()
    return dict(cost=cost.cpu().numpy(), mask=mask.cpu().numpy(), keep=keep.cpu().numpy(),
                aux=None if a is None else a.cpu().numpy(), stats=tct.stats_from(stats))


def oracle_grid(grid: tct.Grid) -> oracle.Grid:
    return oracle.Grid(grid.x0, grid.y0, grid.res, grid.W, grid.H, grid.d_s, grid.z_min,
                       grid.n_slices)


def oracle_all(points: np.ndarray, grid: tct.Grid, params: dict):
    eG, eC, og, dropped, bad = oracle.build(points, oracle_grid(grid), grid.zmin_from_data)
    op = oracle_params(params)
    cT, mask, frag = oracle.evaluate(og, op, eG, eC)
    keep, robust = oracle.simplify(eG, cT, op["c_b"], frag,
                                   keep_ends=bool(params.get("flags", 0) & tct.KEEP_ENDS))
    return dict(ground=eG, ceil=eC, cost=cT, mask=mask, fragile=frag, keep=keep, robust=robust,
                dropped=dropped, nonfinite=bad, grid=og)


def fragile_fraction(fragile: np.ndarray, max_frac: float | None = FRAGILE_MAX) -> float:
    """Share of the cells the oracle leaves out of the checks; printed, and
    bounded by max_frac unless that is None (a caller bounding a total)."""
    n = int(np.count_nonzero(fragile))
    frac = n / max(fragile.size, 1)
    print(f"fragile cells: {n} of {fragile.size} ({frac:.2e})")
    if max_frac is not None:
        assert frac <= max_frac, f"{n} of {fragile.size} cells fragile, above {max_frac}"
    return frac


def assert_costs(cost_gpu: np.ndarray, cost_ref: np.ndarray, fragile: np.ndarray,
                 max_fragile: float | None = FRAGILE_MAX):
    fragile_fraction(fragile, max_fragile)
    ok = (fragile & 1) == 0
    err = np.abs(cost_gpu.astype(np.float64) - cost_ref)
    lim = COST_RTOL * np.maximum(1.0, np.abs(cost_ref))
    bad = ok & ~(err <= lim)
    if bad.any():
        idx = np.argwhere(bad)[:5]
        raise AssertionError(f"{int(bad.sum())} costs out of tolerance, e.g. "
                             + ", ".join(f"{tuple(i)}: gpu {cost_gpu[tuple(i)]!r} oracle "
                                         f"{cost_ref[tuple(i)]!r}" for i in idx))


def assert_masks(mask_gpu: np.ndarray, mask_ref: np.ndarray, fragile: np.ndarray):
    ok = (fragile & 2) == 0
    bad = ok & (mask_gpu != mask_ref)
    if bad.any():
        idx = np.argwhere(bad)[:5]
        raise AssertionError(f"{int(bad.sum())} mask cells differ, e.g. {idx.tolist()}")


def assert_keep(keep_gpu, ground_gpu, cost_gpu, ref, params):
    c_b = float(np.float32(params["c_b"]))
    keep_ends = bool(params.get("flags", 0) & tct.KEEP_ENDS)
    # the chain on the GPU's own layers: the decision in float32
    k_own, _ = oracle.simplify(ground_gpu, cost_gpu.astype(np.float64), c_b, None,
                               keep_ends=keep_ends)
    np.testing.assert_array_equal(keep_gpu, k_own)
    if ref["robust"]:
        np.testing.assert_array_equal(keep_gpu, ref["keep"])


def assert_equal_layers(a: np.ndarray, b: np.ndarray, what: str):
    if not np.array_equal(a, b):
        bad = np.argwhere(a != b)
        i = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} cells differ, e.g. {i}: gpu {a[i]!r} oracle {b[i]!r}")
