"""cr_kkt_residual_noalloc: the KKT residual for callers that cannot allocate.

Processes that reserve their whole device-memory budget at start-up, or loops
that must not call cudaMalloc/cudaFree (those calls can synchronize the
device), use this entry point: it keeps its scratch in a fixed array inside
the library and allocates nothing.  This file checks, through the C ABI, that
it returns what cr_kkt_residual returns for the same iterate, on two calls in
a row (also at a size where every warp walks several rows), that calls after
the first one on a device change no device-memory figure, and that an
oversized problem is refused with a clear message.  It is named so that
pytest collects it after every other test file.
"""
import ctypes

import numpy as np
import pytest

from paper_1407_7220_gb300 import datagen

pytestmark = pytest.mark.gpu


def _noalloc(crg, st, N, n, out):
    L = crg.lib()
    rc = L.cr_kkt_residual_noalloc(N, n, ctypes.c_void_p(st["theta"]), st["ld"], ctypes.c_void_p(st["X"]),
                                   ctypes.c_void_p(st["y"]), ctypes.c_void_p(st["xi"]), ctypes.c_void_p(st["mu"]),
                                   st["sigma"], None, ctypes.c_void_p(out.data_ptr()))
    assert rc == crg.CR_OK, L.cr_last_error(None)


def test_noalloc_matches_kkt_residual_on_two_calls():
    import torch
    import paper_1407_7220_gb300 as crg

    N, n = 700, 3
    X, yb, _ = datagen.make("sq2", N=N, n=n)
    s = crg.Solver(X, yb, gamma=0.1, theta_dtype="f32")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    for k in (30, 45):            # two calls in a row, on two different iterates
        s.iterate(k)
        ref = s.kkt_residual()   # existing entry point (blocks until the handle's work is done)
        _noalloc(crg, s.device_state(), N, n, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = np.array([ref["kkt"], np.nan, np.nan, ref["infeas_norm"], ref["gap_norm"]])
        # maxima are exact; sums agree to FP64 rounding (different summation order)
        assert got[0] == pytest.approx(want[0], rel=1e-12, abs=1e-300)
        assert got[3] == pytest.approx(want[3], rel=1e-10, abs=1e-300)
        assert got[4] == pytest.approx(want[4], rel=1e-9, abs=1e-14)
        assert got[0] == max(got[1], got[2])


def test_noalloc_more_rows_than_warps():
    # N above 64 warps x SMs: every warp of the row kernel walks several rows
    import torch
    import paper_1407_7220_gb300 as crg

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    N, n = 12000, 2
    assert N > 64 * sms
    X, yb, _ = datagen.make("sq2", N=N, n=n)
    s = crg.Solver(X, yb, gamma=0.1, theta_dtype="f32")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    for k in (4, 3):
        s.iterate(k)
        ref = s.kkt_residual()
        _noalloc(crg, s.device_state(), N, n, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(ref["kkt"], rel=1e-12, abs=1e-300)
        assert got[3] == pytest.approx(ref["infeas_norm"], rel=1e-10, abs=1e-300)
        assert got[4] == pytest.approx(ref["gap_norm"], rel=1e-9, abs=1e-14)
    s.close()


def test_noalloc_calls_after_the_first_leave_device_memory_unchanged():
    # the first call on a device may load the library's module and its scratch array (lazy
    # module loading); every later call must not change the device's free memory
    import torch
    import paper_1407_7220_gb300 as crg

    N, n = 500, 2
    X, yb, _ = datagen.make("sq2", N=N, n=n)
    s = crg.Solver(X, yb, gamma=0.1, theta_dtype="f32")
    s.iterate(10)
    st = s.device_state()
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    _noalloc(crg, st, N, n, out)          # warm-up call (set-up on this device)
    torch.cuda.synchronize()
    free0, total0 = torch.cuda.mem_get_info()
    for _ in range(3):
        _noalloc(crg, st, N, n, out)
        torch.cuda.synchronize()
        free1, total1 = torch.cuda.mem_get_info()
        assert (free1, total1) == (free0, total0)
    assert np.isfinite(out.cpu().numpy()).all()
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1407_7220_gb300 as crg

    L = crg.lib()
    one = ctypes.c_void_p(1)
    rc = L.cr_kkt_residual_noalloc(70000, 2, one, 70000, one, one, one, None, 1.0, None, one)
    assert rc == crg.CR_EINVAL
    assert b"exceeds the fixed scratch" in L.cr_last_error(None)
