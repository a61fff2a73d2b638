"""Python binding of libtct (include/tct.h): argument marshalling only.

Every function has the name of the C entry point it calls and takes torch
tensors for the device buffers; the work runs in the library's CUDA kernels
on the current torch stream.  There is no fallback: if libtct.so has not
been built (``paper_2403_07631_gb300.build``) or no GPU is present, the calls
raise.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import torch

from . import build as _build

MAX_SLICES = 127
OK = 0
GRID_ZMIN_FROM_DATA = 1
KEEP_ENDS = 1
ALLOW_COARSE = 2
DEV_NONFINITE = 1
DEV_BAD_QUERY = 2
MAX_PATH_LEN = 2048
NOALLOC_SCRATCH_BYTES = 32 << 20


class TctGrid(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_float), ("y0", ctypes.c_float), ("res", ctypes.c_float),
                ("W", ctypes.c_int32), ("H", ctypes.c_int32), ("d_s", ctypes.c_float),
                ("z_min", ctypes.c_float), ("n_slices", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class TctParams(ctypes.Structure):
    _fields_ = [("d_min", ctypes.c_float), ("d_ref", ctypes.c_float),
                ("theta_b", ctypes.c_float), ("theta_s", ctypes.c_float),
                ("theta_p", ctypes.c_float), ("c_b", ctypes.c_float),
                ("alpha_d", ctypes.c_float), ("alpha_b", ctypes.c_float),
                ("alpha_s", ctypes.c_float), ("d_inf", ctypes.c_float), ("d_sm", ctypes.c_float),
                ("patch_radius", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class TctStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_slices", ctypes.c_int32),
                ("n_points", ctypes.c_int64), ("n_dropped", ctypes.c_int64),
                ("n_nonfinite", ctypes.c_int64), ("z_min", ctypes.c_float),
                ("z_max", ctypes.c_float), ("n_kept", ctypes.c_int32),
                ("reserved", ctypes.c_int32),
                ("valid_cells", ctypes.c_int64 * (MAX_SLICES + 1)),
                ("trav_cells", ctypes.c_int64 * (MAX_SLICES + 1))]


STATS_BYTES = ctypes.sizeof(TctStats)
MAX_BATCH = 64
TILE_AUTO, TILE_64, TILE_32, TILE_64x56, TILE_64x40, TILE_128x56 = 0, 1, 2, 3, 4, 5


class TctMap(ctypes.Structure):
    _fields_ = [("d_xyz", ctypes.c_void_p), ("n", ctypes.c_int64), ("stride", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("grid", TctGrid),
                ("d_ground", ctypes.c_void_p), ("d_ceil", ctypes.c_void_p),
                ("d_cost", ctypes.c_void_p), ("d_mask", ctypes.c_void_p),
                ("d_keep", ctypes.c_void_p), ("d_stats", ctypes.c_void_p)]


class TctHostIO(ctypes.Structure):
    _fields_ = [("h_xyz", ctypes.c_void_p), ("h_ground", ctypes.c_void_p),
                ("h_ceil", ctypes.c_void_p), ("h_cost", ctypes.c_void_p),
                ("h_mask", ctypes.c_void_p), ("h_keep", ctypes.c_void_p),
                ("flags", ctypes.c_uint32), ("n_kept", ctypes.c_int32)]


HOST_KEPT_ONLY = 1


class TctTuning(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("points_per_block", ctypes.c_int32), ("reserved", ctypes.c_int32)]

_P = ctypes.c_void_p
_SIGNATURES = {
    "tct_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tct_version": (ctypes.c_int, []),
    "tct_params_default": (None, [ctypes.POINTER(TctParams)]),
    "tct_plan_grid": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.POINTER(TctGrid)]),
    "tct_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(TctGrid), ctypes.c_int64,
                                              ctypes.POINTER(TctParams)]),
    "tct_bounds": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, _P, _P, _P]),
    "tct_build": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(TctGrid),
                                 _P, ctypes.c_size_t, _P, _P, _P, _P]),
    "tct_evaluate": (ctypes.c_int, [ctypes.POINTER(TctGrid), ctypes.POINTER(TctParams), _P, _P,
                                    _P, ctypes.c_size_t, _P, _P, _P, _P, _P, _P]),
    "tct_build_evaluate": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.POINTER(TctGrid), ctypes.POINTER(TctParams), _P,
                                          ctypes.c_size_t, _P, _P, _P, _P, _P, _P, _P]),
    "tct_build_evaluate_noalloc": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32,
                                                  ctypes.POINTER(TctGrid),
                                                  ctypes.POINTER(TctParams), _P, _P, _P, _P, _P,
                                                  _P, _P]),
    "tct_sample_cost": (ctypes.c_int, [ctypes.POINTER(TctGrid), _P, _P, _P, _P, ctypes.c_int64,
                                       _P, _P, _P, _P]),
    "tct_sample_cost_backward": (ctypes.c_int, [ctypes.POINTER(TctGrid), _P, _P, _P, _P,
                                                ctypes.c_int64, _P, _P, _P, _P]),
    "tct_refine_paths": (ctypes.c_int, [ctypes.POINTER(TctGrid), _P, _P, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                        ctypes.c_float, _P, _P]),
    "tct_workspace_bytes_batched": (ctypes.c_size_t, [ctypes.POINTER(TctMap), ctypes.c_int32,
                                                      ctypes.POINTER(TctParams)]),
    "tct_build_evaluate_batched": (ctypes.c_int, [ctypes.POINTER(TctMap), ctypes.c_int32,
                                                  ctypes.POINTER(TctParams),
                                                  ctypes.POINTER(TctTuning), _P, ctypes.c_size_t,
                                                  _P]),
    "tct_autotune_batched": (ctypes.c_int, [ctypes.POINTER(TctMap), ctypes.c_int32,
                                            ctypes.POINTER(TctParams), _P, ctypes.c_size_t, _P,
                                            ctypes.POINTER(TctTuning)]),
    "tct_timing_enable": (ctypes.c_int, [ctypes.c_int]),
    "tct_timing_read": (ctypes.c_int, [_P, ctypes.c_int]),
    "tct_launch_count": (ctypes.c_int64, []),
    "tct_get_status": (ctypes.c_int, [_P, _P, _P]),
    "tct_build_batched": (ctypes.c_int, [ctypes.POINTER(TctMap), ctypes.c_int32,
                                         ctypes.POINTER(TctTuning), _P, ctypes.c_size_t, _P]),
    "tct_workspace_bytes_evaluate_batched": (ctypes.c_size_t, [ctypes.POINTER(TctMap),
                                                               ctypes.c_int32,
                                                               ctypes.POINTER(TctParams)]),
    "tct_evaluate_batched": (ctypes.c_int, [ctypes.POINTER(TctMap), ctypes.c_int32,
                                            ctypes.POINTER(TctParams), _P, ctypes.c_size_t, _P]),
    "tct_build_evaluate_host": (ctypes.c_int, [ctypes.POINTER(TctHostIO), ctypes.c_int64,
                                               ctypes.c_int32, ctypes.POINTER(TctGrid),
                                               ctypes.POINTER(TctParams), _P, ctypes.c_size_t, _P,
                                               _P, _P, _P, _P, _P, _P, _P]),
    "tct_planner_create": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_float,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "tct_planner_destroy": (None, [_P]),
    "tct_plan_paths": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P, _P, _P,
                                      ctypes.c_int32]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libtct.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libtct.so is not built ({_build.LIB}); run "
                               "paper_2403_07631_gb300.build.build() first")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class TctError(RuntimeError):
    def __init__(self, fn: str, status: int):
        msg = load().tct_status_string(status).decode()
        super().__init__(f"{fn} failed: {msg} ({status})")
        self.status = status


def _check(fn: str, status: int):
    if status != OK:
        raise TctError(fn, status)


# ------------------------------------------------------------- value types

@dataclass
class Grid:
    """Tomogram geometry (tct_grid)."""
    x0: float
    y0: float
    res: float
    W: int
    H: int
    d_s: float
    n_slices: int
    z_min: float = 0.0
    zmin_from_data: bool = True

    def c(self) -> TctGrid:
        return TctGrid(self.x0, self.y0, self.res, self.W, self.H, self.d_s, self.z_min,
                       self.n_slices, GRID_ZMIN_FROM_DATA if self.zmin_from_data else 0)

    @property
    def shape(self):
        return (self.n_slices, self.H, self.W)


def params_default() -> dict:
    """tct_params_default: Table I with the Fig. 3 inflation distances."""
    p = TctParams()
    load().tct_params_default(ctypes.byref(p))
    return {f: getattr(p, f) for f, _ in TctParams._fields_}


def robot_params() -> dict:
    """The benchmark robot: height 0.5 m, max slope 30 deg, inflation 0.3 m."""
    p = params_default()
    p.update(theta_s=math.tan(math.radians(30.0)), d_inf=0.3, d_sm=0.4)
    return p


def _params_c(p: dict) -> TctParams:
    full = {"flags": 0}
    full.update(p)
    return TctParams(*[full[f] for f, _ in TctParams._fields_])


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _points(xyz: torch.Tensor):
    if xyz.dtype != torch.float32 or xyz.dim() != 2 or xyz.shape[1] not in (3, 4):
        raise ValueError("points must be a [P,3] or [P,4] float32 tensor")
    if not xyz.is_contiguous():
        raise ValueError("points must be contiguous")
    return xyz.shape[0], xyz.shape[1]


# ------------------------------------------------------------ entry points

def tct_version() -> int:
    return load().tct_version()


def tct_status_string(status: int) -> str:
    return load().tct_status_string(status).decode()


def tct_plan_grid(bounds6, res: float, d_s: float) -> Grid:
    """Grid over the cloud bounds {x_min, y_min, z_min, x_max, y_max, z_max}."""
    b = (ctypes.c_float * 6)(*[float(v) for v in bounds6])
    g = TctGrid()
    _check("tct_plan_grid", load().tct_plan_grid(ctypes.cast(b, _P), res, d_s, ctypes.byref(g)))
    return Grid(g.x0, g.y0, g.res, g.W, g.H, g.d_s, g.n_slices, g.z_min, True)


def tct_workspace_bytes(grid: Grid, n_points: int, params: dict | None = None) -> int:
    cp = _params_c(params) if params else None
    n = load().tct_workspace_bytes(ctypes.byref(grid.c()), n_points,
                                   ctypes.byref(cp) if cp else None)
    if n == 0:
        raise TctError("tct_workspace_bytes", -1)
    return n


def tct_bounds(xyz: torch.Tensor, out6: torch.Tensor, stats: torch.Tensor | None = None):
    n, stride = _points(xyz)
    _check("tct_bounds", load().tct_bounds(_ptr(xyz), n, stride, _ptr(out6), _ptr(stats), _stream()))


def tct_build(xyz: torch.Tensor, grid: Grid, ws: torch.Tensor, ground: torch.Tensor,
              ceil: torch.Tensor, stats: torch.Tensor | None = None):
    n, stride = _points(xyz)
    _check("tct_build", load().tct_build(_ptr(xyz), n, stride, ctypes.byref(grid.c()), _ptr(ws),
                                         ws.numel() * ws.element_size(), _ptr(ground), _ptr(ceil),
                                         _ptr(stats), _stream()))


def tct_evaluate(grid: Grid, params: dict, ground: torch.Tensor, ceil: torch.Tensor,
                 ws: torch.Tensor, cost: torch.Tensor, mask: torch.Tensor, keep: torch.Tensor,
                 aux: torch.Tensor | None = None, stats: torch.Tensor | None = None):
    cp = _params_c(params)
    _check("tct_evaluate", load().tct_evaluate(ctypes.byref(grid.c()), ctypes.byref(cp),
                                               _ptr(ground), _ptr(ceil), _ptr(ws),
                                               ws.numel() * ws.element_size(), _ptr(cost),
                                               _ptr(mask), _ptr(keep), _ptr(aux), _ptr(stats),
                                               _stream()))


def tct_build_evaluate(xyz: torch.Tensor, grid: Grid, params: dict, ws: torch.Tensor,
                       ground: torch.Tensor, ceil: torch.Tensor, cost: torch.Tensor,
                       mask: torch.Tensor, keep: torch.Tensor, stats: torch.Tensor | None = None):
    n, stride = _points(xyz)
    cp = _params_c(params)
    _check("tct_build_evaluate",
           load().tct_build_evaluate(_ptr(xyz), n, stride, ctypes.byref(grid.c()),
                                     ctypes.byref(cp), _ptr(ws), ws.numel() * ws.element_size(),
                                     _ptr(ground), _ptr(ceil), _ptr(cost), _ptr(mask), _ptr(keep),
                                     _ptr(stats), _stream()))


def tct_build_evaluate_noalloc(xyz: torch.Tensor, grid: Grid, params: dict, ground: torch.Tensor,
                               ceil: torch.Tensor, cost: torch.Tensor, mask: torch.Tensor,
                               keep: torch.Tensor, stats: torch.Tensor | None = None):
    """tct_build_evaluate with the library's fixed scratch instead of a workspace, for
    callers that cannot allocate device memory; maps needing more than
    NOALLOC_SCRATCH_BYTES of scratch are refused."""
    n, stride = _points(xyz)
    cp = _params_c(params)
    _check("tct_build_evaluate_noalloc",
           load().tct_build_evaluate_noalloc(_ptr(xyz), n, stride, ctypes.byref(grid.c()),
                                             ctypes.byref(cp), _ptr(ground), _ptr(ceil),
                                             _ptr(cost), _ptr(mask), _ptr(keep), _ptr(stats),
                                             _stream()))


def _queries(xy: torch.Tensor, slice_idx: torch.Tensor):
    if xy.dtype != torch.float32 or xy.shape[-1] != 2 or not xy.is_contiguous():
        raise ValueError("query points must be a contiguous [..., 2] float32 tensor")
    if slice_idx.dtype != torch.int32 or not slice_idx.is_contiguous():
        raise ValueError("slice indices must be a contiguous int32 tensor")
    q = xy.numel() // 2
    if slice_idx.numel() != q:
        raise ValueError("one slice index per query point")
    return q


def tct_sample_cost(grid: Grid, cost: torch.Tensor | None, ground: torch.Tensor | None,
                    xy: torch.Tensor, slice_idx: torch.Tensor, cost_out: torch.Tensor | None,
                    elev_out: torch.Tensor | None, stats: torch.Tensor | None = None):
    q = _queries(xy, slice_idx)
    _check("tct_sample_cost",
           load().tct_sample_cost(ctypes.byref(grid.c()), _ptr(cost), _ptr(ground), _ptr(xy),
                                  _ptr(slice_idx), q, _ptr(cost_out), _ptr(elev_out), _ptr(stats),
                                  _stream()))


def tct_sample_cost_backward(grid: Grid, cost: torch.Tensor | None, ground: torch.Tensor | None,
                             xy: torch.Tensor, slice_idx: torch.Tensor,
                             gcost: torch.Tensor | None, gelev: torch.Tensor | None,
                             gxy: torch.Tensor):
    q = _queries(xy, slice_idx)
    _check("tct_sample_cost_backward",
           load().tct_sample_cost_backward(ctypes.byref(grid.c()), _ptr(cost), _ptr(ground),
                                           _ptr(xy), _ptr(slice_idx), q, _ptr(gcost),
                                           _ptr(gelev), _ptr(gxy), _stream()))


def tct_refine_paths(grid: Grid, cost: torch.Tensor, slice_idx: torch.Tensor, xy: torch.Tensor,
                     steps: int, eta: float, lam: float):
    """In place: `steps` descent steps on every path of xy [paths, len, 2]."""
    if xy.dim() != 3:
        raise ValueError("paths must be [paths, len, 2]")
    _queries(xy, slice_idx)
    _check("tct_refine_paths",
           load().tct_refine_paths(ctypes.byref(grid.c()), _ptr(cost), _ptr(slice_idx),
                                   xy.shape[0], xy.shape[1], steps, eta, lam, _ptr(xy),
                                   _stream()))


class SampleCost(torch.autograd.Function):
    """Differentiable C(q), e^G(q): forward and backward are the library's
    tct_sample_cost and tct_sample_cost_backward kernels.  Only the query
    coordinates receive a gradient."""

    @staticmethod
    def forward(ctx, xy, slice_idx, cost, ground, grid):
        xy = xy.contiguous()
        c = torch.empty(xy.shape[:-1], dtype=torch.float32, device=xy.device)
        e = torch.empty(xy.shape[:-1], dtype=torch.float32, device=xy.device)
        tct_sample_cost(grid, cost, ground, xy, slice_idx, c, e)
        ctx.save_for_backward(xy, slice_idx, cost, ground)
        ctx.grid = grid
        return c, e

    @staticmethod
    def backward(ctx, gc, ge):
        xy, slice_idx, cost, ground = ctx.saved_tensors
        gxy = torch.empty_like(xy)
        tct_sample_cost_backward(ctx.grid, cost, ground, xy, slice_idx,
                                 None if gc is None else gc.contiguous(),
                                 None if ge is None else ge.contiguous(), gxy)
        return gxy, None, None, None, None


def sample_cost(xy: torch.Tensor, slice_idx: torch.Tensor, cost: torch.Tensor,
                ground: torch.Tensor, grid: Grid):
    """(cost, elevation) at the queries, differentiable with respect to xy."""
    return SampleCost.apply(xy, slice_idx, cost, ground, grid)


@dataclass
class MapBuffers:
    """One map of a batch: its points and its own output tensors (device)."""
    xyz: torch.Tensor
    grid: Grid
    ground: torch.Tensor
    ceil: torch.Tensor
    cost: torch.Tensor
    mask: torch.Tensor
    keep: torch.Tensor
    stats: torch.Tensor | None = None

    @staticmethod
    def allocate(xyz: torch.Tensor, grid: Grid) -> "MapBuffers":
        dev = xyz.device
        return MapBuffers(xyz, grid,
                          torch.empty(grid.shape, dtype=torch.float32, device=dev),
                          torch.empty(grid.shape, dtype=torch.float32, device=dev),
                          torch.empty(grid.shape, dtype=torch.float32, device=dev),
                          torch.empty(grid.shape, dtype=torch.uint8, device=dev),
                          torch.empty(grid.n_slices, dtype=torch.uint8, device=dev),
                          torch.zeros(STATS_BYTES, dtype=torch.uint8, device=dev))


def _maps_c(maps: list[MapBuffers]):
    arr = (TctMap * len(maps))()
    for i, m in enumerate(maps):
        n, stride = _points(m.xyz)
        arr[i] = TctMap(m.xyz.data_ptr(), n, stride, 0, m.grid.c(), m.ground.data_ptr(),
                        m.ceil.data_ptr(), m.cost.data_ptr(), m.mask.data_ptr(),
                        m.keep.data_ptr(), m.stats.data_ptr() if m.stats is not None else None)
    return arr


def tct_workspace_bytes_batched(maps: list[MapBuffers], params: dict) -> int:
    arr = _maps_c(maps)
    cp = _params_c(params)
    n = load().tct_workspace_bytes_batched(arr, len(maps), ctypes.byref(cp))
    if n == 0:
        raise TctError("tct_workspace_bytes_batched", -1)
    return n


def tct_build_evaluate_batched(maps: list[MapBuffers], params: dict, ws: torch.Tensor,
                               tuning: TctTuning | None = None):
    arr = _maps_c(maps)
    cp = _params_c(params)
    _check("tct_build_evaluate_batched",
           load().tct_build_evaluate_batched(arr, len(maps), ctypes.byref(cp),
                                             ctypes.byref(tuning) if tuning is not None else None,
                                             _ptr(ws), ws.numel() * ws.element_size(), _stream()))


def tct_build_batched(maps: list[MapBuffers], ws: torch.Tensor, tuning: TctTuning | None = None):
    """Ground and ceiling layers of every map (the construction alone)."""
    arr = _maps_c(maps)
    _check("tct_build_batched",
           load().tct_build_batched(arr, len(maps),
                                    ctypes.byref(tuning) if tuning is not None else None,
                                    _ptr(ws), ws.numel() * ws.element_size(), _stream()))


def tct_workspace_bytes_evaluate_batched(maps: list[MapBuffers], params: dict) -> int:
    arr = _maps_c(maps)
    cp = _params_c(params)
    n = load().tct_workspace_bytes_evaluate_batched(arr, len(maps), ctypes.byref(cp))
    if n == 0:
        raise TctError("tct_workspace_bytes_evaluate_batched", -1)
    return n


def tct_evaluate_batched(maps: list[MapBuffers], params: dict, ws: torch.Tensor):
    """Costs, masks and keep flags of every map from the layers in its ground / ceil."""
    arr = _maps_c(maps)
    cp = _params_c(params)
    _check("tct_evaluate_batched",
           load().tct_evaluate_batched(arr, len(maps), ctypes.byref(cp), _ptr(ws),
                                       ws.numel() * ws.element_size(), _stream()))


def tct_autotune_batched(maps: list[MapBuffers], params: dict, ws: torch.Tensor) -> TctTuning:
    arr = _maps_c(maps)
    cp = _params_c(params)
    out = TctTuning()
    _check("tct_autotune_batched",
           load().tct_autotune_batched(arr, len(maps), ctypes.byref(cp), _ptr(ws),
                                       ws.numel() * ws.element_size(), _stream(),
                                       ctypes.byref(out)))
    return out


# --------------------------------------------------------------- helpers

def stats_from(t: torch.Tensor) -> TctStats:
    """Copy a device stats block (uint8 tensor of STATS_BYTES) into a TctStats."""
    host = t.detach().to("cpu").numpy().tobytes()
    return TctStats.from_buffer_copy(host)


def alloc_outputs(grid: Grid, n_points: int, device="cuda", params: dict | None = None):
    """Device buffers for tct_build_evaluate: (ws, ground, ceil, cost, mask, keep, stats)."""
    shape = grid.shape
    ws = torch.empty(tct_workspace_bytes(grid, n_points, params), dtype=torch.uint8, device=device)
    ground = torch.empty(shape, dtype=torch.float32, device=device)
    ceil = torch.empty(shape, dtype=torch.float32, device=device)
    cost = torch.empty(shape, dtype=torch.float32, device=device)
    mask = torch.empty(shape, dtype=torch.uint8, device=device)
    keep = torch.empty(grid.n_slices, dtype=torch.uint8, device=device)
    stats = torch.zeros(STATS_BYTES, dtype=torch.uint8, device=device)
    return ws, ground, ceil, cost, mask, keep, stats


def tct_build_evaluate_host(h_xyz: torch.Tensor, grid: Grid, params: dict, ws: torch.Tensor,
                            d_xyz: torch.Tensor, ground: torch.Tensor, ceil: torch.Tensor,
                            cost: torch.Tensor, mask: torch.Tensor, keep: torch.Tensor,
                            stats: torch.Tensor | None = None, h_ground=None, h_ceil=None,
                            h_cost=None, h_mask=None, h_keep=None, kept_only: bool = False) -> int:
    """Host cloud in, host layers out (pinned CPU tensors for asynchronous
    copies), through the caller's device buffers, on the current stream.
    Returns the number of slices copied (the kept ones with kept_only)."""
    if h_xyz.is_cuda or d_xyz.shape != h_xyz.shape:
        raise ValueError("h_xyz must be a host tensor shaped like d_xyz")
    n, stride = _points(h_xyz)
    io = TctHostIO(_ptr(h_xyz), _ptr(h_ground), _ptr(h_ceil), _ptr(h_cost), _ptr(h_mask),
                   _ptr(h_keep), HOST_KEPT_ONLY if kept_only else 0, 0)
    cp = _params_c(params)
    _check("tct_build_evaluate_host",
           load().tct_build_evaluate_host(ctypes.byref(io), n, stride, ctypes.byref(grid.c()),
                                          ctypes.byref(cp), _ptr(ws),
                                          ws.numel() * ws.element_size(), _ptr(d_xyz),
                                          _ptr(ground), _ptr(ceil), _ptr(cost), _ptr(mask),
                                          _ptr(keep), _ptr(stats), _stream()))
    return io.n_kept


def tct_get_status(stats: torch.Tensor) -> int:
    """The device status word (TCT_DEV_* bits) of a stats block, at a sync
    point on the current stream."""
    out = ctypes.c_int32(0)
    _check("tct_get_status", load().tct_get_status(_ptr(stats), ctypes.byref(out),
                                                   _stream()))
    return out.value


def tct_timing_enable(on: bool = True):
    _check("tct_timing_enable", load().tct_timing_enable(1 if on else 0))


def tct_timing_read() -> list[float]:
    """Phase times (ms) of the last timed call: partition, slice stack, chain."""
    buf = (ctypes.c_float * 3)()
    n = load().tct_timing_read(ctypes.cast(buf, _P), 3)
    if n < 0:
        raise TctError("tct_timing_read", n)
    return [float(buf[i]) for i in range(n)]


def tct_launch_count() -> int:
    return int(load().tct_launch_count())


class Planner:
    """Path search across the kept slices (tct_planner_*, a host stage of the
    library): ground / cost are host numpy [N, H, W] float32 layers, keep
    the [N] keep flags (None: all slices).  The library copies what it needs
    (12 bytes per kept slice and cell) when the planner is made."""

    def __init__(self, grid: Grid, ground, cost, keep=None, c_b: float = 50.0):
        import numpy as np
        self.ground = np.ascontiguousarray(ground, dtype=np.float32)
        self.cost = np.ascontiguousarray(cost, dtype=np.float32)
        self.keep = None if keep is None else np.ascontiguousarray(keep, dtype=np.uint8)
        if self.ground.shape != grid.shape or self.cost.shape != grid.shape:
            raise ValueError(f"layers must be {grid.shape}")
        if self.keep is not None and self.keep.shape != (grid.n_slices,):
            raise ValueError("keep must have one flag per slice")
        self.grid = grid
        h = ctypes.c_void_p()
        _check("tct_planner_create",
               load().tct_planner_create(ctypes.byref(grid.c()), self.ground.ctypes.data,
                                         self.cost.ctypes.data,
                                         None if self.keep is None else self.keep.ctypes.data,
                                         float(c_b), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().tct_planner_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def plan(self, starts, goals, max_len: int = 4096, n_threads: int = 0):
        """Plans every (start, goal) pair, each (i, j, slice).  Returns
        (paths: list of int32 [len, 3] arrays, costs: float64 [n], expanded:
        int64 [n]); an unreachable goal gives an empty path and cost inf."""
        import numpy as np
        st = np.ascontiguousarray(np.asarray(starts, dtype=np.int32).reshape(-1, 3))
        go = np.ascontiguousarray(np.asarray(goals, dtype=np.int32).reshape(-1, 3))
        if st.shape != go.shape:
            raise ValueError("starts and goals differ in count")
        n = len(st)
        out = np.zeros((n, max_len, 3), np.int32)
        lens = np.zeros(n, np.int32)
        costs = np.zeros(n, np.float64)
        expanded = np.zeros(n, np.int64)
        _check("tct_plan_paths",
               load().tct_plan_paths(self._h, n, st.ctypes.data, go.ctypes.data, max_len,
                                     out.ctypes.data, lens.ctypes.data, costs.ctypes.data,
                                     expanded.ctypes.data, n_threads))
        return [out[q, :lens[q]].copy() for q in range(n)], costs, expanded
