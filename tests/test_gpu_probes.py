"""The measured pipe and tensor-core rates (fms_probe_pipe_rates,
fms_probe_tensor_rates) that bench.py divides by.

Per clock and per SM, so independent of the SM clock of the moment: FP32 FMA
at most 128 lanes x 2 FLOP... counted here as operations (at most 128 per
clock per SM), MUFU.EX2 at most 32, and the BF16 tensor rate positive and
not above 2 x the nominal dense rate per SM (2.25 PFLOP/s / (152 SMs x
2.07 GHz) ~ 7,150 FLOP per clock per SM) -- a rate far above that would mean
the timed MMAs did not complete.
"""
import pytest

pytestmark = pytest.mark.gpu

fms = pytest.importorskip("paper_2112_13891_gb300")


def test_pipe_rates_are_plausible():
    r = fms.probe_pipe_rates()
    assert 64 <= r["ffma_ops_per_clk_sm"] <= 129
    assert 64 <= r["ffma2_ops_per_clk_sm"] <= 129
    assert 8 <= r["ex2_per_clk_sm"] <= 33


def test_tensor_rates_are_plausible_and_grow_with_n():
    r = fms.probe_tensor_rates()
    one = [r[f"n{n}"]["one_issuer"] for n in (16, 32, 64, 128, 256)]
    two = [r[f"n{n}"]["two_issuers"] for n in (16, 32, 64, 128, 256)]
    for v in one + two:
        assert 0 < v <= 2 * 7150, (one, two)
    # a wider N does at least as much work per MMA: the rate does not fall much
    assert one[-1] >= 0.8 * one[0]
