"""The FP64 throughput probe that supplies the step kernels' roofline denominator.  Its rate per
SM clock is bounded by the unit count the nominal peak assumes (2 operations per clock per SM);
on GB300 it measures 32/19 = 1.684 for fused multiply-add, multiply and add alike, and for the
three interleaved, independent of the number of warps.  Its TFLOP/s cannot exceed the nominal peak at the maximum SM clock."""
import pytest

from paper_2304_09724_gb300 import shweno as S

NOMINAL_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


@pytest.mark.gpu
def test_fp64_probe_rate():
    import torch

    torch.cuda.set_device(0)
    tf, per_clk = S.shweno_fp64_probe(S.FP64_FMA, 8, 1 << 14)
    assert 1.5 <= per_clk <= 2.05, per_clk
    assert 0.3 * NOMINAL_TFLOPS <= tf <= 1.02 * NOMINAL_TFLOPS, tf
    # one warp per scheduler already fills the pipe, and multiply and add issue at the same rate
    _, per_clk4 = S.shweno_fp64_probe(S.FP64_FMA, 4, 1 << 14)
    assert per_clk4 >= 0.95 * per_clk, (per_clk4, per_clk)
    for op in (S.FP64_MUL, S.FP64_ADD, S.FP64_MIX):
        tf_op, per_clk_op = S.shweno_fp64_probe(op, 8, 1 << 14)
        assert abs(per_clk_op / per_clk - 1.0) < 0.05, (op, per_clk_op, per_clk)
        assert tf_op < (0.8 if op == S.FP64_MIX else 0.55) * tf  # fewer flops per operation
