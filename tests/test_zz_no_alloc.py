"""The allocation-free single update (fms_mean_shift_step_noalloc), through the C ABI.

Some callers may not allocate device memory while they run (real-time or
allocator-free runtimes, hosts without a pool to lend a workspace); this entry
point serves them from a fixed scratch array inside the library.  Its results
must agree with fms_mean_shift_step (which takes a caller workspace) within
the tolerance of the step parity tests, on consecutive calls that reuse the
same scratch, and it must refuse requests whose scratch would not fit.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")

_f = fms._lib.fms_mean_shift_step_noalloc
_f.restype = ctypes.c_int
_f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p,
               ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]


def _noalloc(X, Y, h):
    out = torch.empty_like(Y)
    W = torch.empty(Y.shape[0], dtype=torch.float32, device=Y.device)
    rc = _f(X.data_ptr(), X.shape[0], X.shape[1], h, Y.data_ptr(), Y.shape[0], out.data_ptr(),
            W.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return rc, out, W


def _problem(seed, n, m, d):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, 60, (6, d))
    X = (c[rng.integers(0, 6, n)] + 2.0 * rng.standard_normal((n, d))).astype(np.float32)
    Y = (X[rng.integers(0, n, m)] + rng.standard_normal((m, d))).astype(np.float32)
    return torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()


def test_noalloc_matches_workspace_step_on_consecutive_calls():
    h = 3.0
    for seed, n, m, d in [(1, 50_000, 300, 3), (2, 20_011, 1000, 2), (3, 9_000, 77, 16)]:
        X, Y = _problem(seed, n, m, d)
        rc, out, W = _noalloc(X, Y, h)
        assert rc == fms.FMS_OK
        ref, refW = fms.mean_shift_step(X, Y, h, with_wsum=True)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        tol = 2e-4 * h + 2.0 ** -20 * np.abs(b).max()
        assert np.abs(a - b).max() <= tol
        wa, wb = W.cpu().numpy(), refW.cpu().numpy()
        assert np.all(np.abs(wa - wb) <= 1e-5 * np.abs(wb))


def test_noalloc_refuses_requests_that_do_not_fit():
    n, d = 2_000_000, 3          # 32 MB of packed points alone
    X = torch.zeros((n, d), device="cuda")
    Y = torch.zeros((4, d), device="cuda")
    rc, _, _ = _noalloc(X, Y, 1.0)
    assert rc == fms.FMS_ERR_WORKSPACE
    need = fms._lib.fms_step_workspace_size(n, d, 4)
    assert need > (16 << 20)
    # and still works afterwards
    X2, Y2 = _problem(9, 1000, 10, 3)
    rc, out, _ = _noalloc(X2, Y2, 2.0)
    assert rc == fms.FMS_OK
    ref = fms.mean_shift_step(X2, Y2, 2.0)
    assert torch.allclose(out, ref, rtol=0, atol=1e-3)
