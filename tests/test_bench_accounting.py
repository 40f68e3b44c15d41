"""Host-side accounting of bench.py: the algorithmic work behind the roofline
numbers (no GPU).  Each figure is recomputed here from its definition."""
import os

import pytest

import bench
from workloads import CONFIGS


def test_jacobian_flops_r200():
    # reverse mode (d_y < r): d_y x w times W_2^T (w x w), then d_y x w times
    # W_1^T (w x r), 2 flops per multiply-add; three slice products issued
    w = CONFIGS["r200_dis_bf16"]
    d_y, width, r = 100, 400, 200
    assert (w.d_y, w.r, list(w.widths)) == (d_y, r, [r, width, width, d_y])
    assert bench.jacobian_flops(w) == 2 * d_y * width * width + 2 * d_y * r * width == 48e6
    assert bench.jacobian_flops(w, 3) == 144e6


def test_jacobian_order_follows_the_cheaper_mode():
    # the paper's network with d_y = 25: reverse mode, 44 MFLOP against 324
    # MFLOP forward
    w = CONFIGS["paper_ndr_bf16"]
    rev = 2 * 25 * (200 * 400 + 5 * 400 * 400)
    assert bench.jacobian_flops(w) == rev
    from workloads import heterogeneous_workloads
    h = heterogeneous_workloads()[1]             # r = 64 < d_y = 100: forward is cheaper
    fwd = 2 * 64 * (128 * 128 + 128 * 100)
    assert bench.jacobian_flops(h) == fwd < 2 * 100 * (64 * 128 + 128 * 128)


def test_tensor_flops_per_proposal_r200():
    # forward 2(200*400 + 400*400 + 400*100) + Jacobian 48e6 + Gram 2*100^2*200
    # + two projections 2*2*4225*200
    w = CONFIGS["r200_dis_bf16"]
    ref = 2 * (200 * 400 + 400 * 400 + 400 * 100) + 48e6 + 2 * 100 ** 2 * 200 + 4 * 4225 * 200
    assert bench.tensor_flops_per_proposal(w) == ref


def test_geometry_work_woodbury_with_tensor_core_gram():
    # only the bordered (d_y + 1) Cholesky remains in the kernel
    wk = bench.geometry_work(200, 100, tc_gram=True)
    assert wk["fp32"] == 0
    assert wk["df"] == pytest.approx(101 ** 3 / 3)
    assert wk["fp32_charge"] == pytest.approx(12 * 101 ** 3 / 3)


def test_geometry_work_woodbury_in_kernel_gram():
    # FP32 Gram J J^T plus the double-float products K b and K a
    wk = bench.geometry_work(200, 100, tc_gram=False)
    assert wk["fp32"] == 100 * 101 * 200
    assert wk["df"] == pytest.approx(101 ** 3 / 3 + 4 * 200 * 100)


def test_geometry_work_r_sized_path():
    # d_y >= r: FP32 J^T J and the FP64-accurate bordered r-factor with the
    # reverse-density products and the gradient
    r, d_y = 64, 80
    wk = bench.geometry_work(r, d_y)
    assert wk["fp32"] == r * (r + 1) * d_y
    assert wk["df"] == pytest.approx((r + 1) ** 3 / 3 + 2 * r * r + 2 * r * d_y)


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2.07 GHz x 2 flops per fused multiply-add
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2.07e9 * 2 / 1e12)


def test_geometry_traffic_reads_the_committed_summary():
    tpc = bench.geometry_traffic_per_chain("r200_dis_bf16")
    path = os.path.join(bench.ROOT, "profiles", "k_wb_geometry_r200_dis_bf16.txt")
    with open(path) as fh:
        line = [ln for ln in fh if ln.strip().startswith("dram_bytes_per_chain:")][0]
    assert tpc == float(line.split(":")[1])
