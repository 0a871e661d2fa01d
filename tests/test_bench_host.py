"""Host arithmetic of bench.py (no GPU): the algorithmic bytes behind the
roofline figures and the whole-job value, against their closed forms."""

import bench


def test_dual_mm_pass_bytes_closed_forms():
    HW, L = 1242 * 375, 128
    # 16-bit kernel with uint8 deltas and uint8 costs: the horizontal pass reads the
    # deltas of c + lambda_v and writes those of lambda_h (1 B each per pixel-label)
    # plus a 4-byte base per pixel each way; the vertical pass also reads c
    b = bench.dmm_pass_bytes(16, 1, 1, HW, L)
    assert b[0] == HW * (2 * L + 8) == 122_958_000
    assert b[1] == HW * (3 * L + 8)
    # int16 deltas and uint16 costs
    b = bench.dmm_pass_bytes(16, 2, 2, HW, L)
    assert b[0] == HW * (4 * L + 8) and b[1] == HW * (6 * L + 8)
    # int32 kernel: c + lambda_v in, lambda_h out; lambda_h in, lambda_v out
    b = bench.dmm_pass_bytes(32, 4, 1, HW, L)
    assert b[0] == HW * L * 9 and b[1] == HW * L * 8


def test_job_value_counts_every_rank():
    # 2 ranks, 10 steps of 1e6 units each in 1 s (max over ranks): 20 M units/s
    assert bench.job_value(1_000_000, 10, 2, 1000.0) == 20.0


def test_check_kernel_bytes_per_pixel():
    # reads u_left and the mirrored u_right (2 x 4 B), writes the mask (1 B), the
    # checked disparity and the right view's disparity (2 x 4 B)
    assert bench.LR_CHECK_BYTES == 2 * 4 + 1 + 2 * 4


def test_issue_peak_from_unit_counts():
    # 152 SMs x 4 schedulers x one warp-instruction per cycle at 2.07 GHz
    assert abs(bench.ISSUE_PEAK_GINST_S - 152 * 4 * 2.07) < 1e-9
