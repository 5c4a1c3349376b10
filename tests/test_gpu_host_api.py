"""fms_cluster_host: the clustering with host input and output buffers.

The call uploads pageable points into its workspace (page-locked ones are
read in place by the kernels), runs fms_cluster's path and queues the
copy-backs of pageable outputs before its final synchronisation (page-locked
ones are written in place).  It must give the same bits as fms_cluster on
device buffers (same kernels, same arguments), take the CUDA-graph form on
repeated calls, honour max_modes and give the same bits with pageable and
page-locked host memory.
"""
import ctypes

import numpy as np
import pytest
import torch

import fms_inputs as fi
import oracle as orc
from fms_compare import compare_clustering

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")


def test_host_call_equals_device_call():
    w = fi.paper_3d(n=40_000)
    Xh = torch.from_numpy(w.X).pin_memory()
    dev = fms.cluster(Xh.cuda(), w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
    host = fms.cluster_host(Xh, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0, margins=True)
    torch.cuda.synchronize()
    assert host.stats["n_modes"] == dev.stats["n_modes"]
    assert torch.equal(host.modes, dev.modes.cpu())
    assert torch.equal(host.labels, dev.labels.cpu())
    assert torch.equal(host.margins, dev.margins.cpu())
    ref = orc.cluster(w.X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=0)
    cmp = compare_clustering(host.modes.numpy(), host.labels.numpy(), ref, w.h)
    assert cmp["mode_ok"] and cmp["label_mismatch"] == 0, cmp


def test_repeated_host_calls_take_the_graph_form():
    w = fi.separated_blobs(seed=3, k=7, d=3, per=400, sigma=0.6, h=1.5)
    Xh = torch.from_numpy(w.X).pin_memory()
    n, d = Xh.shape
    cap = 64
    o = fms.make_options(gamma=0.95, rng_seed=1)
    ws = fms.Workspace(int(fms._lib.fms_cluster_host_workspace_size(n, d, cap, ctypes.byref(o))),
                       "cuda")
    modes = torch.empty((cap, d)).pin_memory()
    labels = torch.empty(n, dtype=torch.int32).pin_memory()
    outs = []
    for _ in range(3):
        r = fms.cluster_host(Xh, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=1, workspace=ws,
                             out=(modes, labels, None))
        outs.append((r.modes.clone(), labels.clone(), r.stats["graph"]))
    assert [o_[2] for o_ in outs] == [0, 1, 1]
    for o_ in outs[1:]:
        assert torch.equal(o_[0], outs[0][0]) and torch.equal(o_[1], outs[0][1])
    assert outs[0][0].shape[0] == 7


def test_capacity_and_pageable_buffers():
    w = fi.separated_blobs(seed=4, k=5, d=2, per=300, sigma=0.5, h=1.2)
    X = torch.from_numpy(w.X)                      # pageable host memory
    full = fms.cluster_host(X, w.h, w.tol, w.max_iter, rng_seed=2)
    assert full.status == fms.FMS_OK and full.modes.shape[0] == 5
    modes = torch.empty((2, 2))
    labels = torch.empty(X.shape[0], dtype=torch.int32)
    cut = fms.cluster_host(X, w.h, w.tol, w.max_iter, rng_seed=2, out=(modes, labels, None))
    assert cut.status == fms.FMS_ERR_CAPACITY
    assert cut.stats["n_modes"] == 5
    assert torch.equal(cut.modes, full.modes[:2])
    assert torch.equal(labels, full.labels)


def test_pageable_and_page_locked_buffers_give_the_same_bits():
    w = fi.paper_3d(n=30_000)
    Xp = torch.from_numpy(w.X)                       # pageable: copied in and out
    Xl = Xp.pin_memory()                             # page-locked: used in place
    n, d = Xp.shape
    outs = []
    for X, pin in ((Xp, False), (Xl, True)):
        modes = torch.empty((64, d))
        labels = torch.full((n,), -5, dtype=torch.int32)
        margins = torch.full((n,), float("nan"))
        if pin:
            modes, labels, margins = modes.pin_memory(), labels.pin_memory(), margins.pin_memory()
        r = fms.cluster_host(X, w.h, w.tol, w.max_iter, gamma=0.95, rng_seed=4,
                             out=(modes, labels, margins))
        assert r.status == fms.FMS_OK
        outs.append((r.modes.clone(), labels.clone(), margins.clone()))
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
    assert (outs[1][1] >= 0).all()


def test_host_call_argument_errors():
    X = torch.rand(100, 3)
    with pytest.raises(ValueError):
        fms.cluster_host(X.cuda(), 0.5)
    n, d = X.shape
    nm = ctypes.c_int32(0)
    labels = torch.empty(n, dtype=torch.int32)
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    code = fms._lib.fms_cluster_host(ctypes.c_void_p(X.data_ptr()), n, d, 0.5, 0.0, 100, None,
                                     None, 0, ctypes.byref(nm), ctypes.c_void_p(labels.data_ptr()),
                                     None, ctypes.c_void_p(small.data_ptr()), 256, None,
                                     fms._stream())
    assert code == 6   # FMS_ERR_WORKSPACE
    code = fms._lib.fms_cluster_host(ctypes.c_void_p(X.data_ptr()), n, d, -1.0, 0.0, 100, None,
                                     None, 0, ctypes.byref(nm), ctypes.c_void_p(labels.data_ptr()),
                                     None, None, 0, None, fms._stream())
    assert code == 1   # FMS_ERR_INVALID_ARG (h <= 0)
