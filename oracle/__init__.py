"""FP64 CPU oracle for point-cloud tomography (arXiv 2403.07631).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2403_07631_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, brute force); this module
only builds it with gcc, loads it with ctypes and moves numpy arrays in and
out.  Every function cites the passage of the paper it restates:

- ``derive_grid``      Sec. III-A (planes d_s apart, the first d_s above the
                       lowest point, the last above the highest point)
- ``build``            Alg. 1 (construction) and Sec. III-A (ground = highest point
                       of the lower group, ceiling = lowest of the upper group)
- ``kernel``           Eq. 6 (inflation weights)
- ``evaluate``         Sec. III-B, Eq. 1-6 (interval, gradient, terrain and
                       initial costs, inflation, traversable mask)
- ``simplify``         Sec. III-C, Eq. 7-9 (sequential slice-removal chain)
- ``sample``           the cost / elevation queries C(q), e^G(q) of Eq. 10 (bilinear,
                       with the gradient of the interpolant); ``sample_f64`` at
                       FP64 query coordinates
- ``refine``           descent on path waypoints with those queries (an objective of ours)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")


def compile_library(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP when available); returns the .so path."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


class OracleGrid(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_float), ("y0", ctypes.c_float), ("res", ctypes.c_float),
                ("W", ctypes.c_int32), ("H", ctypes.c_int32), ("d_s", ctypes.c_float),
                ("z_min", ctypes.c_float), ("N", ctypes.c_int32)]


class OracleParams(ctypes.Structure):
    _fields_ = [("d_min", ctypes.c_float), ("d_ref", ctypes.c_float),
                ("theta_b", ctypes.c_float), ("theta_s", ctypes.c_float),
                ("theta_p", ctypes.c_float), ("c_b", ctypes.c_float),
                ("alpha_d", ctypes.c_float), ("alpha_b", ctypes.c_float),
                ("alpha_s", ctypes.c_float), ("d_inf", ctypes.c_float),
                ("d_sm", ctypes.c_float), ("patch_radius", ctypes.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(compile_library())
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_plane_heights.argtypes = [ctypes.POINTER(OracleGrid), P]
        lib.oracle_bounds.argtypes = [P, i64, i32, P, P]
        lib.oracle_derive_grid.argtypes = [P, i64, i32, ctypes.c_float, ctypes.c_float,
                                           ctypes.POINTER(OracleGrid)]
        lib.oracle_build.argtypes = [P, i64, i32, ctypes.POINTER(OracleGrid), i32, P, P, P, P]
        lib.oracle_kernel.argtypes = [ctypes.POINTER(OracleParams), ctypes.c_float, P, P, i32]
        lib.oracle_evaluate.argtypes = [ctypes.POINTER(OracleGrid), ctypes.POINTER(OracleParams),
                                        P, P, P, P, P, P]
        lib.oracle_simplify.argtypes = [i32, i32, i32, P, P, P, ctypes.c_double, i32, P, P, P]
        lib.oracle_sample.argtypes = [ctypes.POINTER(OracleGrid), P, i32, P, P, i64, P, P]
        lib.oracle_sample_f64.argtypes = [ctypes.POINTER(OracleGrid), P, i32, P, P, i64, P, P]
        lib.oracle_refine.argtypes = [ctypes.POINTER(OracleGrid), P, P, i32, i32, i32,
                                      ctypes.c_double, ctypes.c_double, P]
        for f in ("oracle_plane_heights", "oracle_bounds", "oracle_derive_grid", "oracle_build",
                  "oracle_kernel", "oracle_evaluate", "oracle_simplify", "oracle_sample",
                  "oracle_sample_f64", "oracle_refine"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    """Threads the oracle's parallel-for over slices uses (OMP_NUM_THREADS)."""
    return int(_load().oracle_num_threads())


@dataclass
class Grid:
    """Tomogram geometry: cell (0,0) starts at (x0, y0); rows i run along +y."""
    x0: float
    y0: float
    res: float
    W: int
    H: int
    d_s: float
    z_min: float
    N: int

    def c(self) -> OracleGrid:
        return OracleGrid(self.x0, self.y0, self.res, self.W, self.H, self.d_s, self.z_min, self.N)

    @staticmethod
    def from_c(g: OracleGrid) -> "Grid":
        return Grid(g.x0, g.y0, g.res, g.W, g.H, g.d_s, g.z_min, g.N)


PARAM_FIELDS = ("d_min", "d_ref", "theta_b", "theta_s", "theta_p", "c_b", "alpha_d",
                "alpha_b", "alpha_s", "d_inf", "d_sm", "patch_radius")


def _params(p: dict) -> OracleParams:
    return OracleParams(*[p[k] for k in PARAM_FIELDS])


def _points(xyz: np.ndarray) -> tuple[np.ndarray, int]:
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    if xyz.ndim != 2 or xyz.shape[1] not in (3, 4):
        raise ValueError("points must be [P,3] or [P,4] float32")
    return xyz, xyz.shape[1]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str, allow=(0,)):
    if rc not in allow:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def plane_heights(g: Grid) -> np.ndarray:
    """Sec. III-A: h_k = z_min + (k+1) d_s, k = 0..N-1, rounded once to float32."""
    h = np.empty(g.N, np.float32)
    _check(_load().oracle_plane_heights(ctypes.byref(g.c()), _ptr(h)), "plane_heights")
    return h


def bounds(xyz: np.ndarray) -> tuple[np.ndarray, int]:
    """Min/max of x, y, z over the finite points, and the count of non-finite ones."""
    xyz, stride = _points(xyz)
    out = np.empty(6, np.float64)
    bad = ctypes.c_int64(0)
    _check(_load().oracle_bounds(_ptr(xyz), len(xyz), stride, _ptr(out), ctypes.byref(bad)), "bounds")
    return out, bad.value


def derive_grid(xyz: np.ndarray, res: float, d_s: float) -> Grid:
    """Sec. III-A: grid over the cloud's footprint and the plane count N."""
    xyz, stride = _points(xyz)
    g = OracleGrid()
    _check(_load().oracle_derive_grid(_ptr(xyz), len(xyz), stride, res, d_s, ctypes.byref(g)),
           "derive_grid")
    return Grid.from_c(g)


def build(xyz: np.ndarray, g: Grid, zmin_from_data: bool = True):
    """The construction of Alg. 1 by brute force.  Returns (eG, eC, grid, n_dropped, n_nonfinite);
    eG/eC are [N,H,W] float32 with -inf/+inf for invalid cells."""
    xyz, stride = _points(xyz)
    cg = g.c()
    eG = np.empty((g.N, g.H, g.W), np.float32)
    eC = np.empty((g.N, g.H, g.W), np.float32)
    dropped, bad = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = _load().oracle_build(_ptr(xyz), len(xyz), stride, ctypes.byref(cg), int(zmin_from_data),
                              _ptr(eG), _ptr(eC), ctypes.byref(dropped), ctypes.byref(bad))
    _check(rc, "build", allow=(0, -3))
    return eG, eC, Grid.from_c(cg), dropped.value, bad.value


def kernel(p: dict, res: float) -> np.ndarray:
    """Eq. 6: the (2R+1)x(2R+1) inflation weights K(m, n), rows indexed by n."""
    cp = _params(p)
    R = ctypes.c_int32(0)
    lib = _load()
    _check(lib.oracle_kernel(ctypes.byref(cp), res, ctypes.byref(R), None, 0), "kernel")
    side = 2 * R.value + 1
    K = np.empty((side, side), np.float64)
    _check(lib.oracle_kernel(ctypes.byref(cp), res, ctypes.byref(R), _ptr(K), side * side), "kernel")
    return K


def evaluate(g: Grid, p: dict, eG: np.ndarray, eC: np.ndarray, want_aux: bool = False):
    """Sec. III-B, Eq. 1-6.  Returns (cT float64, mask uint8, fragile uint8[, aux]);
    aux = float64 [5,N,H,W] with m^xy, m^grad, c^I, c^G, c^init."""
    eG = np.ascontiguousarray(eG, np.float32)
    eC = np.ascontiguousarray(eC, np.float32)
    shape = (g.N, g.H, g.W)
    if eG.shape != shape or eC.shape != shape:
        raise ValueError(f"elevations must be {shape}")
    cT = np.empty(shape, np.float64)
    mask = np.empty(shape, np.uint8)
    frag = np.empty(shape, np.uint8)
    aux = np.empty((5,) + shape, np.float64) if want_aux else None
    cg, cp = g.c(), _params(p)
    rc = _load().oracle_evaluate(ctypes.byref(cg), ctypes.byref(cp), _ptr(eG), _ptr(eC), _ptr(cT),
                                 _ptr(mask), _ptr(frag), _ptr(aux) if want_aux else None)
    _check(rc, "evaluate")
    return (cT, mask, frag, aux) if want_aux else (cT, mask, frag)


def simplify(eG: np.ndarray, cT: np.ndarray, c_b: float, fragile: np.ndarray | None = None,
             keep_ends: bool = False, want_counts: bool = False):
    """Sec. III-C, Eq. 7-9: the sequential chain.  Returns (keep uint8[N], robust bool)
    and, with want_counts, int64 [N,3]: unique, surely unique, possibly unique cells."""
    eG = np.ascontiguousarray(eG, np.float32)
    cT = np.ascontiguousarray(cT, np.float64)
    N, H, W = eG.shape
    if cT.shape != eG.shape:
        raise ValueError("cT and eG shapes differ")
    f = None if fragile is None else np.ascontiguousarray(fragile, np.uint8)
    keep = np.empty(N, np.uint8)
    robust = np.zeros(1, np.uint8)
    counts = np.zeros((N, 3), np.int64)
    rc = _load().oracle_simplify(N, H, W, _ptr(eG), _ptr(cT), None if f is None else _ptr(f),
                                 float(c_b), int(keep_ends), _ptr(keep), _ptr(robust),
                                 _ptr(counts))
    _check(rc, "simplify")
    return (keep, bool(robust[0]), counts) if want_counts else (keep, bool(robust[0]))


def sample(g: Grid, layer: np.ndarray, xy: np.ndarray, slice_idx: np.ndarray,
           is_ground: bool = False):
    """Bilinear query of slice `slice_idx[t]` of `layer` ([N,H,W] float32) at xy[t];
    returns (values float64 [Q], gradient float64 [Q,2])."""
    layer = np.ascontiguousarray(layer, np.float32)
    xy = np.ascontiguousarray(xy, np.float32).reshape(-1, 2)
    sl = np.ascontiguousarray(slice_idx, np.int32).reshape(-1)
    q = len(xy)
    out = np.empty(q, np.float64)
    grad = np.empty((q, 2), np.float64)
    _check(_load().oracle_sample(ctypes.byref(g.c()), _ptr(layer), int(is_ground), _ptr(xy),
                                 _ptr(sl), q, _ptr(out), _ptr(grad)), "sample")
    return out, grad


def sample_f64(g: Grid, layer: np.ndarray, xy: np.ndarray, slice_idx: np.ndarray,
               is_ground: bool = False):
    """``sample`` at FP64 query coordinates (for central differences whose step
    lies below a float32 ulp of the coordinate)."""
    layer = np.ascontiguousarray(layer, np.float32)
    xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
    sl = np.ascontiguousarray(slice_idx, np.int32).reshape(-1)
    q = len(xy)
    out = np.empty(q, np.float64)
    grad = np.empty((q, 2), np.float64)
    _check(_load().oracle_sample_f64(ctypes.byref(g.c()), _ptr(layer), int(is_ground), _ptr(xy),
                                     _ptr(sl), q, _ptr(out), _ptr(grad)), "sample_f64")
    return out, grad


def refine(g: Grid, cost: np.ndarray, slice_idx: np.ndarray, xy: np.ndarray, steps: int,
           eta: float, lam: float) -> np.ndarray:
    """`steps` descent steps on every path of xy [paths, len, 2]; returns the new xy (float64)."""
    cost = np.ascontiguousarray(cost, np.float32)
    X = np.array(xy, dtype=np.float64, order="C")
    paths, length = X.shape[0], X.shape[1]
    sl = np.ascontiguousarray(slice_idx, np.int32).reshape(paths, length)
    _check(_load().oracle_refine(ctypes.byref(g.c()), _ptr(cost), _ptr(sl), paths, length, steps,
                                 float(eta), float(lam), _ptr(X)), "refine")
    return X
