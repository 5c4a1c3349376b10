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
import json
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")

_f = fms._lib.fms_mean_shift_step_noalloc
_f.restype = ctypes.c_int
_f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p,
               ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]


def _noalloc(X, Y, h, out=None, W=None):
    out = torch.empty_like(Y) if out is None else out
    W = torch.empty(Y.shape[0], dtype=torch.float32, device=Y.device) if W is None else W
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


def test_noalloc_allocates_no_device_memory():
    # the point of the entry point: repeated calls leave the device's free
    # memory and torch's allocator untouched (outputs are preallocated; one
    # warm-up call first, since the first call on a device may load code)
    X, Y = _problem(4, 30_000, 200, 3)
    out = torch.empty_like(Y)
    W = torch.empty(Y.shape[0], dtype=torch.float32, device=Y.device)
    assert _noalloc(X, Y, 2.5, out, W)[0] == fms.FMS_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(5):
        assert _noalloc(X, Y, 2.5, out, W)[0] == fms.FMS_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0


# Child process (no torch): device buffers through the CUDA runtime the library
# itself loaded, one call, a device reset (a new context, in which the scratch
# array may sit elsewhere), the same call again, and the allocating workspace
# form for reference.
_CHILD = r"""
import ctypes, json, sys
import numpy as np
lib = ctypes.CDLL(sys.argv[1])
rt_path = next(l.split()[-1] for l in open("/proc/self/maps") if "libcudart" in l)
rt = ctypes.CDLL(rt_path)
P = ctypes.c_void_p
def dmalloc(nb):
    p = P()
    assert rt.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(nb)) == 0
    return p
def h2d(p, a):
    assert rt.cudaMemcpy(p, a.ctypes.data_as(P), ctypes.c_size_t(a.nbytes), 1) == 0
def d2h(a, p):
    assert rt.cudaMemcpy(a.ctypes.data_as(P), p, ctypes.c_size_t(a.nbytes), 2) == 0
lib.fms_mean_shift_step_noalloc.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float,
                                            P, ctypes.c_int64, P, P, P]
lib.fms_mean_shift_step.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, P,
                                    ctypes.c_int64, P, P, P, ctypes.c_size_t, P]
rng = np.random.default_rng(7)
n, m, d, h = 20000, 150, 3, 2.0
c = rng.uniform(0, 40, (5, d))
X = (c[rng.integers(0, 5, n)] + rng.standard_normal((n, d))).astype(np.float32)
Y = (X[rng.integers(0, n, m)] + 0.5 * rng.standard_normal((m, d))).astype(np.float32)
def run(fn):
    dX, dY, dO = dmalloc(X.nbytes), dmalloc(Y.nbytes), dmalloc(Y.nbytes)
    h2d(dX, X); h2d(dY, Y)
    if fn == "noalloc":
        rc = lib.fms_mean_shift_step_noalloc(dX, n, d, h, dY, m, dO, None, None)
    else:
        rc = lib.fms_mean_shift_step(dX, n, d, h, dY, m, dO, None, None, 0, None)
    assert rc == 0, rc
    assert rt.cudaDeviceSynchronize() == 0
    out = np.empty_like(Y)
    d2h(out, dO)
    for p in (dX, dY, dO):
        rt.cudaFree(p)
    return out
a = run("noalloc")
assert rt.cudaDeviceReset() == 0
b = run("noalloc")
r = run("workspace")
print(json.dumps({"reset_diff": float(np.abs(a - b).max()),
                  "vs_workspace": float(np.abs(b.astype(np.float64) - r).max()),
                  "scale": float(np.abs(r).max())}))
"""


def test_noalloc_after_a_device_reset():
    p = subprocess.run([sys.executable, "-c", _CHILD, fms._lib._name], capture_output=True,
                       text=True, timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
    res = json.loads(p.stdout.strip().splitlines()[-1])
    assert res["reset_diff"] == 0.0, res        # same kernels, same inputs, same bits
    h = 2.0
    assert res["vs_workspace"] <= 2e-4 * h + 2.0 ** -20 * res["scale"], res
