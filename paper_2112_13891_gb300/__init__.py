"""Python binding of the GB300 Faster Mean-shift library (libfms_gb300.so).

Argument marshalling only: every step of the clustering runs in the library's
CUDA kernels.  Tensors must be CUDA tensors; work is issued on the current
torch stream.  The library is required -- there is no fallback: importing
this package raises if ``libfms_gb300.so`` has not been built (run
``python -m paper_2112_13891_gb300.build`` or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfms_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(python -m paper_2112_13891_gb300.build)")

_lib = ctypes.CDLL(LIB_PATH)

FMS_OK, FMS_ERR_INVALID_ARG, FMS_ERR_NONFINITE, FMS_ERR_CAPACITY = 0, 1, 2, 3
FMS_ERR_TIMEOUT, FMS_ERR_CUDA, FMS_ERR_WORKSPACE, FMS_ERR_UNSUPPORTED = 4, 5, 6, 7
PRECISION = {"auto": 0, "fp32": 1, "tensor": 2}
KERNEL = {"gaussian": 0, "flat": 1}
METRIC = {"euclidean": 0, "cosine": 1}
MAX_DIM = 64


class FmsOptions(ctypes.Structure):
    _fields_ = [("all_seeds", ctypes.c_int32), ("n_initial", ctypes.c_int32),
                ("L", ctypes.c_float), ("gamma", ctypes.c_float),
                ("merge_radius", ctypes.c_float), ("skip_refine", ctypes.c_int32),
                ("rng_seed", ctypes.c_uint64), ("seed_indices", ctypes.c_void_p),
                ("n_seed_indices", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("metric", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class FmsStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("n_seeds_final", ctypes.c_int32), ("n_converged", ctypes.c_int32),
                ("n_discarded", ctypes.c_int32), ("n_kept", ctypes.c_int32),
                ("n_modes", ctypes.c_int32), ("refine_iterations", ctypes.c_int32),
                ("t_star_last", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("evals", ctypes.c_int64), ("score_evals", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_uint64), ("step_kernel_ms", ctypes.c_double),
                ("step_launches", ctypes.c_int32), ("coarse_launches", ctypes.c_int32),
                ("step_evals", ctypes.c_int64), ("round_kernel_ms", ctypes.c_double),
                ("round_evals", ctypes.c_int64), ("round_launches", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("phase_ms", ctypes.c_double * 4),
                ("coarse_kernel_ms", ctypes.c_double), ("coarse_evals", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            if k.startswith("reserved"):
                continue
            v = getattr(self, k)
            out[k] = list(v) if k == "phase_ms" else v
        return out


_P, _I32, _I64, _F32, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t

_lib.fms_strerror.restype = ctypes.c_char_p
_lib.fms_strerror.argtypes = [ctypes.c_int]
_lib.fms_options_default.restype = None
_lib.fms_options_default.argtypes = [ctypes.POINTER(FmsOptions)]
_lib.fms_workspace_size.restype = _SZ
_lib.fms_workspace_size.argtypes = [_I64, _I32, ctypes.POINTER(FmsOptions)]
_lib.fms_cluster.restype = ctypes.c_int
_lib.fms_cluster.argtypes = [_P, _I64, _I32, _F32, _F32, _I32, ctypes.POINTER(FmsOptions), _P,
                             _I32, ctypes.POINTER(_I32), _P, _P, _P, _SZ,
                             ctypes.POINTER(FmsStats), _P]
_lib.fms_cluster_host_workspace_size.restype = _SZ
_lib.fms_cluster_host_workspace_size.argtypes = [_I64, _I32, _I32, ctypes.POINTER(FmsOptions)]
_lib.fms_cluster_host.restype = ctypes.c_int
_lib.fms_cluster_host.argtypes = [_P, _I64, _I32, _F32, _F32, _I32, ctypes.POINTER(FmsOptions),
                                  _P, _I32, ctypes.POINTER(_I32), _P, _P, _P, _SZ,
                                  ctypes.POINTER(FmsStats), _P]
_lib.fms_selftest_bounded_wait.restype = ctypes.c_int
_lib.fms_selftest_bounded_wait.argtypes = [_I32, _I64, ctypes.POINTER(ctypes.c_uint32), _P]
_lib.fms_cluster_frames.restype = ctypes.c_int
_lib.fms_cluster_frames.argtypes = [_P, _I32, _I64, _I32, _F32, _F32, _I32,
                                    ctypes.POINTER(FmsOptions), _F32, _P, _I32, _P, _P, _P, _P,
                                    _P, _SZ, ctypes.POINTER(FmsStats), _P]
_lib.fms_select_seeds.restype = ctypes.c_int
_lib.fms_select_seeds.argtypes = [_I64, ctypes.c_uint64, _I64, _I64, _P, _P]
_lib.fms_step_workspace_size.restype = _SZ
_lib.fms_step_workspace_size.argtypes = [_I64, _I32, _I64]
_lib.fms_mean_shift_step.restype = ctypes.c_int
_lib.fms_mean_shift_step.argtypes = [_P, _I64, _I32, _F32, _P, _I64, _P, _P, _P, _SZ, _P]
_lib.fms_coarse_step_workspace_size.restype = _SZ
_lib.fms_coarse_step_workspace_size.argtypes = [_I64, _I32, _I64]
_lib.fms_mean_shift_step_coarse.restype = ctypes.c_int
_lib.fms_mean_shift_step_coarse.argtypes = [_P, _I64, _I32, _F32, _P, _I64, _P, _P, _P, _SZ, _P]
_lib.fms_label_points.restype = ctypes.c_int
_lib.fms_label_points.argtypes = [_P, _I64, _I32, _P, _I32, _P, _P, _P]


class FmsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (status {code})")


def strerror(code: int) -> str:
    return _lib.fms_strerror(int(code)).decode()


def _check(code: int, where: str):
    if code != FMS_OK:
        raise FmsError(code, where)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _points(x: torch.Tensor) -> torch.Tensor:
    if not x.is_cuda:
        raise ValueError("points must be a CUDA tensor")
    if x.dim() != 2:
        raise ValueError("points must be [n, d]")
    return x.to(torch.float32).contiguous()


def make_options(*, all_seeds=False, n_initial=128, L=8.0, gamma=0.95, merge_radius=0.0,
                 skip_refine=False, rng_seed=0, seed_indices=None, profile=False,
                 precision="auto", kernel="gaussian", metric="euclidean") -> FmsOptions:
    o = FmsOptions()
    _lib.fms_options_default(ctypes.byref(o))
    o.all_seeds = int(bool(all_seeds))
    o.n_initial = int(n_initial)
    o.L = float(L)
    o.gamma = float(gamma)
    o.merge_radius = float(merge_radius)
    o.skip_refine = int(bool(skip_refine))
    o.rng_seed = int(rng_seed) & ((1 << 64) - 1)
    if seed_indices is not None:
        o.seed_indices = seed_indices.data_ptr()
        o.n_seed_indices = int(seed_indices.numel())
    o.profile = int(bool(profile))
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.kernel = KERNEL[kernel] if isinstance(kernel, str) else int(kernel)
    o.metric = METRIC[metric] if isinstance(metric, str) else int(metric)
    return o


_NEED_CACHE: dict = {}


def _workspace_need(n: int, d: int, o: FmsOptions) -> int:
    """fms_workspace_size, remembered per (device, n, d, options)."""
    key = (torch.cuda.current_device(), n, d, bytes(o))
    need = _NEED_CACHE.get(key)
    if need is None:
        need = int(_lib.fms_workspace_size(n, d, ctypes.byref(o)))
        if len(_NEED_CACHE) > 256:
            _NEED_CACHE.clear()
        _NEED_CACHE[key] = need
    return need


def workspace_size(n: int, d: int, **opts) -> int:
    o = make_options(**opts)
    return int(_lib.fms_workspace_size(int(n), int(d), ctypes.byref(o)))


class ClusterResult:
    """modes [M, d] float32 (canonical order), labels [n] int32, margins [n]
    float32 or None, stats (dict, converted from fms_stats on first use),
    status."""

    __slots__ = ("modes", "labels", "margins", "_stats", "status")

    def __init__(self, modes, labels, margins, stats, status):
        self.modes = modes
        self.labels = labels
        self.margins = margins
        self._stats = stats
        self.status = status

    @property
    def stats(self) -> dict:
        if not isinstance(self._stats, dict):
            self._stats = self._stats.as_dict()
        return self._stats


class Workspace:
    """A reusable device workspace for repeated calls of the same shape."""

    def __init__(self, nbytes: int, device=None):
        self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device or "cuda")

    @property
    def nbytes(self):
        return self.buf.numel()


def cluster(points: torch.Tensor, h: float, tol: float = 0.0, max_iter: int = 300, *,
            all_seeds=False, n_initial=128, L=8.0, gamma=0.95, merge_radius=0.0,
            skip_refine=False, rng_seed=0, seed_indices=None, max_modes=None, margins=True,
            workspace: Workspace = None, profile=False, precision="auto", kernel="gaussian",
            metric="euclidean", out=None) -> ClusterResult:
    """Faster Mean-shift clustering of the rows of `points` (fms_cluster).

    `out` may pass preallocated (modes [max_modes, d], labels [n], margins [n]).
    """
    X = _points(points)
    n, d = X.shape
    if seed_indices is not None:
        seed_indices = seed_indices.to(device=X.device, dtype=torch.int32).contiguous()
    o = make_options(all_seeds=all_seeds, n_initial=n_initial, L=L, gamma=gamma,
                     merge_radius=merge_radius, skip_refine=skip_refine, rng_seed=rng_seed,
                     seed_indices=seed_indices, profile=profile, precision=precision,
                     kernel=kernel, metric=metric)
    if out is not None:
        modes, labels, mar = out
        cap = modes.shape[0]
    else:
        cap = int(max_modes) if max_modes is not None else n
        modes = torch.empty((max(cap, 1), d), dtype=torch.float32, device=X.device)
        labels = torch.empty(n, dtype=torch.int32, device=X.device)
        mar = torch.empty(n, dtype=torch.float32, device=X.device) if margins else None
    need = _workspace_need(n, d, o)
    if workspace is None or workspace.nbytes < need:
        workspace = Workspace(need, X.device)
    nm = _I32(0)
    st = FmsStats()
    code = _lib.fms_cluster(_ptr(X), n, d, float(h), float(tol), int(max_iter), ctypes.byref(o),
                            _ptr(modes), cap, ctypes.byref(nm), _ptr(labels), _ptr(mar),
                            _ptr(workspace.buf), workspace.nbytes, ctypes.byref(st), _stream())
    if code not in (FMS_OK, FMS_ERR_CAPACITY):
        raise FmsError(code, "fms_cluster")
    M = nm.value
    return ClusterResult(modes=modes[: min(M, cap)], labels=labels, margins=mar, stats=st,
                         status=code)


def cluster_host(points: torch.Tensor, h: float, tol: float = 0.0, max_iter: int = 300, *,
                 all_seeds=False, n_initial=128, L=8.0, gamma=0.95, merge_radius=0.0,
                 skip_refine=False, rng_seed=0, max_modes=256, margins=False,
                 workspace: Workspace = None, precision="auto", kernel="gaussian",
                 metric="euclidean", out=None, device=None) -> ClusterResult:
    """fms_cluster_host: `points` is a CPU float32 [n, d] tensor (page-locked
    for asynchronous copies); the results come back in CPU tensors, copied
    under the call's own synchronisation.  `out` may pass preallocated CPU
    tensors (modes [max_modes, d], labels [n], margins [n] or None)."""
    if points.is_cuda:
        raise ValueError("cluster_host takes host (CPU) points; use cluster() for device tensors")
    X = points.contiguous().float()
    if X.dim() != 2:
        raise ValueError("points must be [n, d]")
    n, d = X.shape
    o = make_options(all_seeds=all_seeds, n_initial=n_initial, L=L, gamma=gamma,
                     merge_radius=merge_radius, skip_refine=skip_refine, rng_seed=rng_seed,
                     precision=precision, kernel=kernel, metric=metric)
    if out is not None:
        modes, labels, mar = out
        cap = modes.shape[0]
    else:
        cap = int(max_modes)
        modes = torch.empty((max(cap, 1), d), dtype=torch.float32).pin_memory()
        labels = torch.empty(n, dtype=torch.int32).pin_memory()
        mar = torch.empty(n, dtype=torch.float32).pin_memory() if margins else None
    need = int(_lib.fms_cluster_host_workspace_size(n, d, cap, ctypes.byref(o)))
    if need == 0:
        raise FmsError(FMS_ERR_INVALID_ARG, "fms_cluster_host_workspace_size")
    if workspace is None or workspace.nbytes < need:
        workspace = Workspace(need, device)
    nm = _I32(0)
    st = FmsStats()
    code = _lib.fms_cluster_host(_ptr(X), n, d, float(h), float(tol), int(max_iter),
                                 ctypes.byref(o), _ptr(modes), cap, ctypes.byref(nm),
                                 _ptr(labels), _ptr(mar), _ptr(workspace.buf), workspace.nbytes,
                                 ctypes.byref(st), _stream())
    if code not in (FMS_OK, FMS_ERR_CAPACITY):
        raise FmsError(code, "fms_cluster_host")
    M = nm.value
    return ClusterResult(modes=modes[: min(M, cap)], labels=labels, margins=mar, stats=st,
                         status=code)


def selftest_bounded_wait(variant: int = 0, spins: int = 1000):
    """Run fms_selftest_bounded_wait: returns (status code, status word)."""
    word = ctypes.c_uint32(0)
    code = _lib.fms_selftest_bounded_wait(int(variant), int(spins), ctypes.byref(word), _stream())
    return code, word.value


@dataclass
class FramesResult:
    modes: list          # per frame: [M_f, d] tensor
    labels: torch.Tensor  # [F, n]
    margins: torch.Tensor
    seed_counts: list    # N_f, the seed count frame f started with
    stats: dict
    status: int


def cluster_frames(frames, h: float, tol: float = 0.0, max_iter: int = 300, *, H=32.0,
                   n_initial=128, L=8.0, gamma=0.95, merge_radius=0.0, skip_refine=False,
                   rng_seed=0, max_modes=256, precision="auto", kernel="gaussian",
                   metric="euclidean",
                   workspace: Workspace = None) -> FramesResult:
    """Faster Mean-shift over a frame sequence (fms_cluster_frames): `frames`
    is a [F, n, d] CUDA tensor or a list of F [n, d] tensors."""
    if isinstance(frames, (list, tuple)):
        frames = torch.stack([_points(f) for f in frames])
    frames = frames.contiguous().float()
    F, n, d = frames.shape
    o = make_options(n_initial=n_initial, L=L, gamma=gamma, merge_radius=merge_radius,
                     skip_refine=skip_refine, rng_seed=rng_seed, precision=precision,
                     kernel=kernel, metric=metric)
    cap = max(int(max_modes), 1)
    modes = torch.empty((F, cap, d), dtype=torch.float32, device=frames.device)
    labels = torch.empty((F, n), dtype=torch.int32, device=frames.device)
    mar = torch.empty((F, n), dtype=torch.float32, device=frames.device)
    nm = (_I32 * F)()
    starts = (_I32 * F)()
    need = int(_lib.fms_workspace_size(n, d, ctypes.byref(o)))
    if workspace is None or workspace.nbytes < need:
        workspace = Workspace(need, frames.device)
    st = FmsStats()
    code = _lib.fms_cluster_frames(_ptr(frames), F, n, d, float(h), float(tol), int(max_iter),
                                   ctypes.byref(o), float(H), _ptr(modes), cap, nm, _ptr(labels),
                                   _ptr(mar), starts, _ptr(workspace.buf), workspace.nbytes,
                                   ctypes.byref(st), _stream())
    if code not in (FMS_OK, FMS_ERR_CAPACITY):
        raise FmsError(code, "fms_cluster_frames")
    return FramesResult(modes=[modes[f, : min(nm[f], cap)] for f in range(F)], labels=labels,
                        margins=mar, seed_counts=list(starts), stats=st.as_dict(), status=code)


def select_seeds(n: int, rng_seed: int, start: int, count: int, device="cuda") -> torch.Tensor:
    """Entries [start, start+count) of the keyed seed permutation (fms_select_seeds)."""
    out = torch.empty(max(int(count), 0), dtype=torch.int32, device=device)
    _check(_lib.fms_select_seeds(int(n), int(rng_seed) & ((1 << 64) - 1), int(start), int(count),
                                 _ptr(out), _stream()), "fms_select_seeds")
    return out


def mean_shift_step(points: torch.Tensor, seeds: torch.Tensor, h: float, with_wsum=False,
                    workspace: Workspace = None):
    """One Gaussian mean-shift update of each row of `seeds` (fms_mean_shift_step)."""
    X = _points(points)
    Y = _points(seeds)
    n, d = X.shape
    m = Y.shape[0]
    out = torch.empty_like(Y)
    wsum = torch.empty(m, dtype=torch.float32, device=X.device) if with_wsum else None
    need = int(_lib.fms_step_workspace_size(n, d, m))
    if workspace is None or workspace.nbytes < need:
        workspace = Workspace(need, X.device)
    _check(_lib.fms_mean_shift_step(_ptr(X), n, d, float(h), _ptr(Y), m, _ptr(out), _ptr(wsum),
                                    _ptr(workspace.buf), workspace.nbytes, _stream()),
           "fms_mean_shift_step")
    return (out, wsum) if with_wsum else out


def mean_shift_step_coarse(points: torch.Tensor, seeds: torch.Tensor, h: float,
                           with_wsum=False, workspace: Workspace = None):
    """One coarse (tensor-core, BF16-weight) update of each row of `seeds`
    (fms_mean_shift_step_coarse); 1 <= d <= 32."""
    X = _points(points)
    Y = _points(seeds)
    n, d = X.shape
    m = Y.shape[0]
    out = torch.empty_like(Y)
    wsum = torch.empty(m, dtype=torch.float32, device=X.device) if with_wsum else None
    need = int(_lib.fms_coarse_step_workspace_size(n, d, m))
    if need == 0:
        raise FmsError(FMS_ERR_UNSUPPORTED, "fms_mean_shift_step_coarse")
    if workspace is None or workspace.nbytes < need:
        workspace = Workspace(need, X.device)
    _check(_lib.fms_mean_shift_step_coarse(_ptr(X), n, d, float(h), _ptr(Y), m, _ptr(out),
                                           _ptr(wsum), _ptr(workspace.buf), workspace.nbytes,
                                           _stream()),
           "fms_mean_shift_step_coarse")
    return (out, wsum) if with_wsum else out


def label_points(points: torch.Tensor, modes: torch.Tensor, with_margins=True):
    """Nearest-mode labels and margins (fms_label_points)."""
    X = _points(points)
    Mo = _points(modes)
    n, d = X.shape
    labels = torch.empty(n, dtype=torch.int32, device=X.device)
    mar = torch.empty(n, dtype=torch.float32, device=X.device) if with_margins else None
    _check(_lib.fms_label_points(_ptr(X), n, d, _ptr(Mo), Mo.shape[0], _ptr(labels), _ptr(mar),
                                 _stream()), "fms_label_points")
    return (labels, mar) if with_margins else labels


# ---------------------------------------------------------------------------
# Differentiable unrolled steps (fms_unrolled_forward / fms_unrolled_backward)
# ---------------------------------------------------------------------------

_F64 = ctypes.c_double
for _sfx, _fh in (("", _F32), ("_f64", _F64)):
    getattr(_lib, "fms_unrolled_ckpt_size" + _sfx).restype = _SZ
    getattr(_lib, "fms_unrolled_ckpt_size" + _sfx).argtypes = [_I32, _I64, _I64, _I32, _I32, _I32]
    getattr(_lib, "fms_unrolled_workspace_size" + _sfx).restype = _SZ
    getattr(_lib, "fms_unrolled_workspace_size" + _sfx).argtypes = [_I32, _I64, _I64, _I32, _I32,
                                                                    _I32]
    getattr(_lib, "fms_unrolled_forward" + _sfx).restype = ctypes.c_int
    getattr(_lib, "fms_unrolled_forward" + _sfx).argtypes = [_P, _P, _I32, _I64, _I64, _I32, _fh,
                                                             _I32, _I32, _P, _P, _SZ, _P, _SZ, _P]
    getattr(_lib, "fms_unrolled_backward" + _sfx).restype = ctypes.c_int
    getattr(_lib, "fms_unrolled_backward" + _sfx).argtypes = [_P, _I32, _I64, _I64, _I32, _fh,
                                                              _I32, _I32, _P, _SZ, _P, _P, _P, _P,
                                                              _P, _SZ, _P]


def _batched(x: torch.Tensor, name: str, dtype=torch.float32) -> torch.Tensor:
    if not x.is_cuda or x.dim() != 3:
        raise ValueError(f"{name} must be a CUDA tensor [B, rows, d]")
    return x.to(dtype).contiguous()


def _unrolled_sfx(dtype) -> str:
    """FP64 tensors take the *_f64 entry points (gradient checks), others FP32."""
    return "_f64" if dtype == torch.float64 else ""


def unrolled_forward(X: torch.Tensor, Y0: torch.Tensor, h: float, T: int, k: int):
    """T Gaussian updates of every row of Y0 (per set) against X; returns (Y_T, ckpt).
    FP64 inputs run the FP64 kernels, anything else FP32."""
    dt = torch.float64 if X.dtype == torch.float64 else torch.float32
    sfx = _unrolled_sfx(dt)
    X, Y0 = _batched(X, "X", dt), _batched(Y0, "Y0", dt)
    B, n, d = X.shape
    m = Y0.shape[1]
    cb = int(getattr(_lib, "fms_unrolled_ckpt_size" + sfx)(B, n, m, d, T, k))
    wb = int(getattr(_lib, "fms_unrolled_workspace_size" + sfx)(B, n, m, d, T, k))
    if cb == 0 or wb == 0:
        raise FmsError(FMS_ERR_INVALID_ARG, "fms_unrolled_forward" + sfx)
    ckpt = torch.empty(cb, dtype=torch.uint8, device=X.device)
    ws = torch.empty(wb, dtype=torch.uint8, device=X.device)
    out = torch.empty_like(Y0)
    _check(getattr(_lib, "fms_unrolled_forward" + sfx)(
        _ptr(X), _ptr(Y0), B, n, m, d, float(h), int(T), int(k), _ptr(out), _ptr(ckpt), cb,
        _ptr(ws), wb, _stream()), "fms_unrolled_forward" + sfx)
    return out, ckpt


def unrolled_backward(X: torch.Tensor, ckpt: torch.Tensor, m: int, h: float, T: int, k: int,
                      grad_out: torch.Tensor):
    """Adjoint of unrolled_forward: returns (dL/dX, dL/dY0, dL/dh per set as float64),
    in X's precision (FP64 or FP32)."""
    dt = torch.float64 if X.dtype == torch.float64 else torch.float32
    sfx = _unrolled_sfx(dt)
    X, G = _batched(X, "X", dt), _batched(grad_out, "grad_out", dt)
    B, n, d = X.shape
    wb = int(getattr(_lib, "fms_unrolled_workspace_size" + sfx)(B, n, m, d, T, k))
    ws = torch.empty(wb, dtype=torch.uint8, device=X.device)
    dX = torch.empty_like(X)
    dY = torch.empty((B, m, d), dtype=dt, device=X.device)
    dh = torch.empty(B, dtype=torch.float64, device=X.device)
    _check(getattr(_lib, "fms_unrolled_backward" + sfx)(
        _ptr(X), B, n, m, d, float(h), int(T), int(k), _ptr(ckpt), ckpt.numel(), _ptr(G),
        _ptr(dX), _ptr(dY), _ptr(dh), _ptr(ws), wb, _stream()), "fms_unrolled_backward" + sfx)
    return dX, dY, dh


class UnrolledMeanShift(torch.autograd.Function):
    """Y_T = T Gaussian mean-shift updates of Y0 against X (per set), differentiable
    in X, Y0 and h by the library's adjoint kernels (weights recomputed tile by
    tile, positions checkpointed every k updates)."""

    @staticmethod
    def forward(ctx, X, Y0, h, T, k):
        hv = float(h)
        out, ckpt = unrolled_forward(X.detach(), Y0.detach(), hv, T, k)
        ctx.save_for_backward(X.detach(), ckpt)
        ctx.cfg = (hv, int(T), int(k), Y0.shape[1], torch.is_tensor(h))
        return out

    @staticmethod
    def backward(ctx, grad_out):
        X, ckpt = ctx.saved_tensors
        hv, T, k, m, h_is_tensor = ctx.cfg
        dX, dY, dh = unrolled_backward(X, ckpt, m, hv, T, k, grad_out)
        gh = dh.sum().to(X.dtype).reshape(()) if h_is_tensor else None
        return dX, dY, gh, None, None


def unrolled_mean_shift(X: torch.Tensor, Y0: torch.Tensor, h, T: int = 20, k: int = 5):
    return UnrolledMeanShift.apply(X, Y0, h, T, k)


# ---------------------------------------------------------------------------
# Batched clustering (fms_cluster_batched)
# ---------------------------------------------------------------------------

_lib.fms_batched_workspace_size.restype = _SZ
_lib.fms_batched_workspace_size.argtypes = [_P, _I32, _I32, ctypes.POINTER(FmsOptions)]
_lib.fms_cluster_batched.restype = ctypes.c_int
_lib.fms_cluster_batched.argtypes = [_P, _P, _I32, _I32, _F32, _F32, _I32,
                                     ctypes.POINTER(FmsOptions), _P, _I32, _P, _P, _P, _P, _SZ,
                                     ctypes.POINTER(FmsStats), _P]


@dataclass
class BatchedResult:
    modes: list            # per set: [M_b, d] float32 tensors (views of one buffer)
    n_modes: torch.Tensor  # [B] int32 (device)
    labels: torch.Tensor   # [total] int32, indices into the point's own set's modes
    margins: torch.Tensor
    stats: dict
    status: int


def cluster_batched(points, h: float, tol: float = 0.0, max_iter: int = 300, *, offsets=None,
                    n_initial=128, L=8.0, gamma=0.95, merge_radius=0.0, skip_refine=False,
                    all_seeds=False, rng_seed=0, max_modes=256, margins=True,
                    workspace: Workspace = None, kernel="gaussian",
                    metric="euclidean") -> BatchedResult:
    """Cluster many point sets at once.  `points` is a list of [n_b, d] CUDA
    tensors, or one [total, d] tensor with host `offsets` (B+1 ints)."""
    import numpy as np
    if offsets is None:
        sizes = [int(p.shape[0]) for p in points]
        X = torch.cat([_points(p) for p in points], dim=0)
        offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    else:
        X = _points(points)
        offsets = np.asarray(offsets, dtype=np.int64)
    B = len(offsets) - 1
    total, d = X.shape
    o = make_options(all_seeds=all_seeds, n_initial=n_initial, L=L, gamma=gamma,
                     merge_radius=merge_radius, skip_refine=skip_refine, rng_seed=rng_seed,
                     kernel=kernel, metric=metric)
    offs = np.ascontiguousarray(offsets)
    optr = offs.ctypes.data_as(ctypes.c_void_p)
    need = int(_lib.fms_batched_workspace_size(optr, B, d, ctypes.byref(o)))
    if need == 0:
        raise FmsError(FMS_ERR_INVALID_ARG, "fms_batched_workspace_size")
    if workspace is None or workspace.nbytes < need:
        workspace = Workspace(need, X.device)
    modes = torch.empty((B, max(int(max_modes), 1), d), dtype=torch.float32, device=X.device)
    n_modes = torch.empty(B, dtype=torch.int32, device=X.device)
    labels = torch.empty(total, dtype=torch.int32, device=X.device)
    mar = torch.empty(total, dtype=torch.float32, device=X.device) if margins else None
    st = FmsStats()
    code = _lib.fms_cluster_batched(_ptr(X), optr, B, d, float(h), float(tol), int(max_iter),
                                    ctypes.byref(o), _ptr(modes), int(max_modes), _ptr(n_modes),
                                    _ptr(labels), _ptr(mar), _ptr(workspace.buf), workspace.nbytes,
                                    ctypes.byref(st), _stream())
    if code not in (FMS_OK, FMS_ERR_CAPACITY):
        raise FmsError(code, "fms_cluster_batched")
    counts = n_modes.cpu().tolist()
    per = [modes[b, : min(counts[b], int(max_modes))] for b in range(B)]
    return BatchedResult(modes=per, n_modes=n_modes, labels=labels, margins=mar,
                         stats=st.as_dict(), status=code)


# ---------------------------------------------------------------------------
# Measured pipe rates (fms_probe_pipe_rates)
# ---------------------------------------------------------------------------

_lib.fms_probe_pipe_rates.restype = ctypes.c_int
_lib.fms_probe_pipe_rates.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int32]


_lib.fms_probe_tensor_rates.restype = ctypes.c_int
_lib.fms_probe_tensor_rates.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int32]


def probe_tensor_rates() -> dict:
    """BF16 tcgen05 FLOP per clock per SM (completed MMAs, M = 128, K = 16) for
    N = 16 .. 256, with one and with two issuing threads per SM."""
    out = (ctypes.c_double * 10)()
    _check(_lib.fms_probe_tensor_rates(out, 10), "fms_probe_tensor_rates")
    return {f"n{n}": {"one_issuer": out[2 * i], "two_issuers": out[2 * i + 1]}
            for i, n in enumerate((16, 32, 64, 128, 256))}


def probe_pipe_rates() -> dict:
    """FP32 / SFU throughputs of the current device per clock and per SM."""
    out = (ctypes.c_double * 4)()
    _check(_lib.fms_probe_pipe_rates(out, 4), "fms_probe_pipe_rates")
    return {"ffma_ops_per_clk_sm": out[0], "ffma2_ops_per_clk_sm": out[1],
            "ex2_per_clk_sm": out[2], "eval_mix_units_per_clk_sm": out[3]}
