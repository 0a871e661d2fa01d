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


def test_survey_bytes_of_the_frame_and_of_a_pass():
    HW, L = 1242 * 375, 128
    # compulsory bytes with int16 duals: horizontal c 1 + lambda_v 2 + lambda_h 2,
    # vertical lambda_h 2 + lambda_v 2 bytes per pixel-label
    p = bench.survey_pass_bytes(HW, L)
    assert p[0] == HW * L * 5 and p[1] == HW * L * 4
    # the 1242x375x128 frame: cost 0.060 + Dual MM 5.25 + linearise 0.05 + PD 2.79
    # = 8.15 GB (10 Dual MM and 100 PD iterations in 5 warps)
    f = bench.survey_frame_bytes(HW, L, 1, 10, 100, 5)
    assert f == HW * (2 + L) + HW * L * 88 + HW * 23 * 5 + HW * 60 * 100
    assert abs(f / 1e9 - 8.15) < 0.01


def test_lane_group_kernel_storage_bytes():
    HW, L = 1242 * 375, 128
    # both passes read the unary deltas and the cost and write the output deltas
    b = bench.dmm_pass_bytes(8, 1, 1, HW, L)
    assert b[0] == b[1] == HW * (3 * L + 8)


def test_profile_figures_are_keyed_to_the_kernel_source():
    import hashlib
    import os
    tag = bench.source_tag("lr.cu")
    path = os.path.join(os.path.dirname(bench.__file__), "paper_1601_06274_gb300", "csrc", "lr.cu")
    assert tag == hashlib.sha256(open(path, "rb").read()).hexdigest()[:12]
    for key in bench.NCU_TRAFFIC:
        assert len(key) == 3 and len(key[2]) == 12
