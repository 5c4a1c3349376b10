"""Failure detection without a GPU fault: the bounded mbarrier waits of the
tensor-core step give up after their poll bound, set the timeout bit of the
status word and return, and the context stays usable."""
import pytest
import torch

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")

FMS_ERR_TIMEOUT = 4


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_wait_that_nothing_completes_times_out(variant):
    code, word = fms.selftest_bounded_wait(variant, spins=2000)
    assert code == FMS_ERR_TIMEOUT
    assert word == 2          # the timeout bit only: the completed phase was then seen


def test_context_usable_after_timeouts():
    for v in range(3):
        fms.selftest_bounded_wait(v, spins=500)
    X = torch.randn(5000, 3, device="cuda")
    r = fms.cluster(X, 1.0)
    torch.cuda.synchronize()
    assert r.stats["n_modes"] >= 1
    assert r.labels.shape[0] == 5000


def test_invalid_arguments():
    assert fms.selftest_bounded_wait(3, 10)[0] == 1
    assert fms.selftest_bounded_wait(0, 0)[0] == 1
