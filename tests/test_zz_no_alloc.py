"""swof_volume_noalloc: the volume / minimum-depth reduction for callers that
may not allocate device memory (a caller capturing its own CUDA graph, a host
whose device memory all belongs to its own pool allocator, a real-time loop
that must not synchronise on an allocation).

It is called through the C ABI on caller-owned device buffers and must give
the same volume and minimum depth as the context's own diagnostics
(swof_get_diagnostics), within the budget tolerance the parity tests use,
on two calls in a row (the second on a later state, so stale scratch from
the first call would show).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import paper_1307_4839_gb300 as sw
import swof_inputs as si

pytestmark = pytest.mark.gpu


def _call(lib, h, nx, ny, dtype, dx, dy, out, stream):
    return lib.swof_volume_noalloc(ctypes.c_void_p(h.data_ptr()), nx, ny, dtype, dx, dy,
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("precision", [sw.FP64, sw.FP32])
def test_noalloc_volume_matches_diagnostics_on_two_calls(precision):
    import torch
    assert torch.cuda.is_available()
    sw.build()
    lib = sw.load()
    w = si.random_state(203, 141, seed=77, dry_frac=0.3)
    s = sw.Solver.from_workload(w, precision)
    tdt = torch.float64 if precision == sw.FP64 else torch.float32
    h = torch.empty((w.ny, w.nx), dtype=tdt, device="cuda")
    q1 = torch.empty_like(h)
    q2 = torch.empty_like(h)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        if call == 1:
            s.step(15)
        s.get_state_device(h, q1, q2)
        torch.cuda.synchronize()
        d = s.diagnostics()
        assert _call(lib, h, w.nx, w.ny, precision, w.dx, w.dy, out, stream) == sw.OK
        torch.cuda.synchronize()
        vol, mn = out.cpu().numpy()
        assert abs(vol - d["volume"]) <= 1e-12 * d["volume"], (call, vol, d["volume"])
        assert mn == d["min_h"], (call, mn, d["min_h"])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    lib = sw.load()
    h = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert _call(lib, h, 1, sw.NOALLOC_MAX_ROWS + 1, sw.FP64, 1.0, 1.0, out, 0) == sw.EINVAL
    assert _call(lib, h, 2, 2, 7, 1.0, 1.0, out, 0) == sw.EINVAL
    assert lib.swof_volume_noalloc(None, 2, 2, sw.FP64, 1.0, 1.0, ctypes.c_void_p(out.data_ptr()), None) == sw.EINVAL


def test_noalloc_min_depth_keeps_nan():
    """A depth field holding a NaN reports NaN as its minimum (a positivity
    check on out[1] must not pass such a field)."""
    import torch
    lib = sw.load()
    h = torch.rand((37, 53), dtype=torch.float64, device="cuda")
    h[20, 7] = float("nan")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert _call(lib, h, 53, 37, sw.FP64, 1.0, 1.0, out, torch.cuda.current_stream().cuda_stream) == sw.OK
    torch.cuda.synchronize()
    assert torch.isnan(out[1]).item() and torch.isnan(out[0]).item()
