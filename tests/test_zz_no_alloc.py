"""tct_build_evaluate_noalloc: the entry point for callers that cannot
allocate device memory (a control loop with memory reserved at start-up, a
plug-in whose host owns the allocator) takes its scratch from a fixed array
inside the library.  Its results must match tct_build_evaluate with a
caller-provided workspace, call after call, although every call reuses the
same array and finds the previous call's leftovers in it.

This file is named to be collected last, so that a failure here comes after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from conftest import PARAMS_ROBOT  # noqa: E402
from _parity import COST_RTOL  # noqa: E402
from paper_2403_07631_gb300 import build, scenes, tct  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tct.load()


def _outputs(grid, dev):
    return (torch.empty(grid.shape, dtype=torch.float32, device=dev),
            torch.empty(grid.shape, dtype=torch.float32, device=dev),
            torch.empty(grid.shape, dtype=torch.float32, device=dev),
            torch.empty(grid.shape, dtype=torch.uint8, device=dev),
            torch.empty(grid.n_slices, dtype=torch.uint8, device=dev),
            torch.zeros(tct.STATS_BYTES, dtype=torch.uint8, device=dev))


def _noalloc_call(lib, pts, grid, params, outs):
    ground, ceil, cost, mask, keep, stats = outs
    p = tct.TctParams(*[dict({"flags": 0}, **params)[f] for f, _ in tct.TctParams._fields_])
    g = grid.c()
    v = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    return lib.tct_build_evaluate_noalloc(v(pts), pts.shape[0], pts.shape[1], ctypes.byref(g),
                                          ctypes.byref(p), v(ground), v(ceil), v(cost), v(mask),
                                          v(keep), v(stats),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _compare(a, b):
    ga, ca, ta, ma, ka, sa = [t.cpu().numpy() for t in a]
    gb, cb, tb, mb, kb, sb = [t.cpu().numpy() for t in b]
    np.testing.assert_array_equal(ga, gb)
    np.testing.assert_array_equal(ca, cb)
    err = np.abs(ta.astype(np.float64) - tb.astype(np.float64))
    assert np.all(err <= COST_RTOL * np.maximum(1.0, np.abs(tb.astype(np.float64))))
    np.testing.assert_array_equal(ma, mb)
    np.testing.assert_array_equal(ka, kb)
    st_a, st_b = tct.TctStats.from_buffer_copy(sa.tobytes()), tct.TctStats.from_buffer_copy(sb.tobytes())
    assert (st_a.n_kept, st_a.n_dropped, st_a.n_points) == (st_b.n_kept, st_b.n_dropped, st_b.n_points)
    assert list(st_a.trav_cells) == list(st_b.trav_cells)


def test_noalloc_matches_workspace_entry_point_twice(lib):
    dev = torch.device("cuda")
    params = PARAMS_ROBOT
    # two different maps in a row: the second call finds the first one's
    # leftovers in the shared scratch
    cases = [scenes.two_storey_building(),
             scenes.building(41, 90_000, side_cells=130, floors=[0.0, 1.4, 2.9],
                             ceilings=[1.2, 2.7, 4.4])]
    for sc in cases:
        grid = tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, sc.n_slices or 12, 0.0, True)
        assert tct.tct_workspace_bytes(grid, len(sc.points), params) <= tct.NOALLOC_SCRATCH_BYTES
        pts = torch.from_numpy(sc.points).to(dev)
        ref = _outputs(grid, dev)
        ws = torch.empty(tct.tct_workspace_bytes(grid, len(sc.points), params), dtype=torch.uint8,
                         device=dev)
        tct.tct_build_evaluate(pts, grid, params, ws, *ref)
        got = _outputs(grid, dev)
        assert _noalloc_call(lib, pts, grid, params, got) == tct.OK
        torch.cuda.synchronize()
        _compare(got, ref)


def test_noalloc_refuses_maps_beyond_its_scratch(lib):
    # 2000 x 2000 cells need ~48 MB of scratch: refused before any launch
    grid = tct.Grid(0.0, 0.0, 0.1, 2000, 2000, 0.5, 4, 0.0, True)
    dev = torch.device("cuda")
    pts = torch.zeros((16, 3), dtype=torch.float32, device=dev)
    outs = [torch.empty(1, device=dev)] * 6
    assert tct.tct_workspace_bytes(grid, 16, PARAMS_ROBOT) > tct.NOALLOC_SCRATCH_BYTES
    assert _noalloc_call(lib, pts, grid, PARAMS_ROBOT, outs) == -2
