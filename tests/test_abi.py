"""The C ABI library builds, loads and exports every symbol of include/dm.h;
host-side argument checking works without a GPU (no compute call is made)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1601_06274_gb300 import build, dm
    build.build()
    return dm.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "dm.h")).read()
    return re.findall(r"DM_API\s+[\w\s\*]+?\b(dm_\w+)\s*\(", src)


def test_header_declares_the_boundary():
    names = set(declared_symbols())
    for required in ("dm_create", "dm_cost_volume", "dm_discrete", "dm_refine", "dm_solve"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_default_params_and_create(lib):
    from paper_1601_06274_gb300 import dm
    p = dm.default_params()
    assert p.struct_size == ctypes.sizeof(dm.DmParams)
    assert (p.census_win, p.w_hi, p.w_lo, p.eps, p.delta, p.C, p.warps) == (5, 8, 4, 0.25, 1.0, 2.0, 5)
    h = ctypes.c_void_p()
    assert lib.dm_create(375, 1242, 128, ctypes.byref(p), ctypes.byref(h)) == 0
    nbytes = ctypes.c_size_t()
    assert lib.dm_workspace_bytes(h, ctypes.byref(nbytes)) == 0
    # cost volume + two int32 duals + two message scratches dominate
    assert nbytes.value >= 375 * 1242 * 128 * (1 + 4 * 4)
    assert lib.dm_destroy(h) == 0


@pytest.mark.parametrize("H,W,L,field,value", [
    (0, 10, 16, None, None), (10, 0, 16, None, None), (10, 10, 1, None, None),
    (10, 10, 257, None, None), (10, 10, 16, "census_win", 7), (10, 10, 16, "w_hi", 256),
    (10, 10, 16, "tau", 0.0), (10, 10, 16, "warps", 0), (10, 10, 16, "struct_size", 8),
    (10, 10, 16, "C", -1.0),
])
def test_create_rejects_invalid_arguments(lib, H, W, L, field, value):
    from paper_1601_06274_gb300 import dm
    p = dm.default_params()
    if field is not None:
        setattr(p, field, value)
    h = ctypes.c_void_p()
    assert lib.dm_create(H, W, L, ctypes.byref(p), ctypes.byref(h)) == dm.DM_ERR_ARG
    assert not h.value


@pytest.mark.parametrize("field,value", [("w_hi", 3), ("C", 9.0), ("eps", 0.3)])
def test_penalty_without_integer_taps_disables_discrete_stage(lib, field, value):
    # 3 * 1/4 is not an integer; C = 9 does not reach the cap within 4 labels
    from paper_1601_06274_gb300 import dm
    p = dm.default_params()
    setattr(p, field, value)
    h = ctypes.c_void_p()
    assert lib.dm_create(10, 10, 16, ctypes.byref(p), ctypes.byref(h)) == 0
    assert lib.dm_discrete(h, 1, None) == dm.DM_ERR_ARG
    assert lib.dm_discrete_pass(h, 0) == dm.DM_ERR_ARG
    assert lib.dm_refine(h, 1, None) == dm.DM_ERR_STATE  # no workspace yet, but allowed
    lib.dm_destroy(h)


def test_calls_without_workspace_are_state_errors(lib):
    from paper_1601_06274_gb300 import dm
    p = dm.default_params()
    h = ctypes.c_void_p()
    assert lib.dm_create(8, 8, 16, ctypes.byref(p), ctypes.byref(h)) == 0
    assert lib.dm_discrete(h, 1, None) == dm.DM_ERR_STATE
    assert lib.dm_refine(h, 1, None) == dm.DM_ERR_STATE
    assert lib.dm_cost_volume(h, None, None) == dm.DM_ERR_STATE
    assert lib.dm_bind_workspace(h, ctypes.c_void_p(4096 + 8), 1 << 30) == dm.DM_ERR_WORKSPACE
    assert lib.dm_bind_workspace(h, ctypes.c_void_p(4096), 16) == dm.DM_ERR_WORKSPACE
    assert lib.dm_discrete(None, 1, None) == dm.DM_ERR_ARG
    lib.dm_destroy(h)


def test_error_strings(lib):
    from paper_1601_06274_gb300 import dm
    assert dm.error_string(0) == "ok"
    for code in range(1, 8):
        assert dm.error_string(code) not in ("ok", "unknown status")
    assert dm.error_string(99) == "unknown status"


def _ctx(lib, H=256, W=512, L=96, **kw):
    from paper_1601_06274_gb300 import dm
    p = dm.default_params(**kw)
    h = ctypes.c_void_p()
    assert lib.dm_create(H, W, L, ctypes.byref(p), ctypes.byref(h)) == 0
    return h


def test_tape_size_follows_checkpoints_and_warps(lib):
    h = _ctx(lib)
    n = ctypes.c_size_t()
    slot = 256 * 512 * 4
    # 200 iterations, 5 warps of 40, checkpoint every 20: 10 segments of 20
    assert lib.dm_tape_bytes(h, 200, 20, ctypes.byref(n)) == 0
    assert n.value == (10 * 5 + 20 * 5 + 10 + 4) * slot + 8192
    # checkpoint every 30: segment starts 0 30 40 60 80 90 120 150 160 180
    assert lib.dm_tape_bytes(h, 200, 30, ctypes.byref(n)) == 0
    assert n.value == (10 * 5 + 30 * 5 + 14) * slot + 8192
    # no iterations: the start state only
    assert lib.dm_tape_bytes(h, 0, 20, ctypes.byref(n)) == 0
    assert n.value == (5 + 14) * slot + 8192
    for iters, ck in ((-1, 20), (10, 0), (1 << 21, 20)):
        assert lib.dm_tape_bytes(h, iters, ck, ctypes.byref(n)) == 1
    assert lib.dm_destroy(h) == 0


def test_differentiable_calls_check_state_without_gpu(lib):
    from paper_1601_06274_gb300 import dm
    h = _ctx(lib, 8, 8, 16)
    # no workspace bound: every call that touches device state refuses
    assert lib.dm_set_cost_volume_f32(h, 4096, None, None) == dm.DM_ERR_STATE
    assert lib.dm_set_data_weights(h, None) == dm.DM_ERR_STATE
    assert lib.dm_refine_tape(h, 10, 5, None, None, 0) == dm.DM_ERR_STATE
    assert lib.dm_refine_backward(h, 4096, None, 0, None, None, None, None) == dm.DM_ERR_STATE
    assert lib.dm_set_lambda_r(h, -1.0) == dm.DM_ERR_ARG
    assert lib.dm_set_lambda_r(h, float("nan")) == dm.DM_ERR_ARG
    assert lib.dm_set_lambda_r(h, 2.5) == dm.DM_OK
    assert lib.dm_set_lambda_r(None, 1.0) == dm.DM_ERR_ARG
    assert lib.dm_destroy(h) == 0


def test_batch_create_and_workspace_without_gpu(lib):
    from paper_1601_06274_gb300 import dm
    p = dm.default_params()
    n = 3
    H = (ctypes.c_int * n)(240, 480, 375)
    W = (ctypes.c_int * n)(320, 640, 1242)
    L = (ctypes.c_int * n)(32, 64, 128)
    b = ctypes.c_void_p()
    assert lib.dm_batch_create(n, H, W, L, ctypes.byref(p), ctypes.byref(b)) == 0
    nb = ctypes.c_size_t()
    assert lib.dm_batch_workspace_bytes(b, ctypes.byref(nb)) == 0
    single = 0
    for i in range(n):
        h = ctypes.c_void_p()
        assert lib.dm_create(H[i], W[i], L[i], ctypes.byref(p), ctypes.byref(h)) == 0
        s = ctypes.c_size_t()
        lib.dm_workspace_bytes(h, ctypes.byref(s))
        single += s.value
        lib.dm_destroy(h)
    assert nb.value >= single
    ptrs = (ctypes.c_void_p * n)(1, 2, 3)
    assert lib.dm_batch_solve(b, ptrs, ptrs, 5, 50, None) == dm.DM_ERR_STATE  # no workspace
    assert lib.dm_batch_solve(b, ptrs, ptrs, 0, 50, None) == dm.DM_ERR_ARG
    assert lib.dm_batch_solve(b, ptrs, ptrs, 257, 50, None) == dm.DM_ERR_ARG
    assert lib.dm_batch_replay(b) == dm.DM_ERR_STATE                         # nothing captured
    good = (ctypes.c_int * 5)(2, 32, 8, 4, 96)
    bad = (ctypes.c_int * 5)(2, 48, 8, 4, 96)
    assert lib.dm_batch_set_tuning(b, good) == 0 and lib.dm_batch_set_tuning(b, bad) == dm.DM_ERR_ARG
    out = (ctypes.c_int * 5)()
    assert lib.dm_batch_get_tuning(b, out) == 0 and tuple(out) == (2, 32, 8, 4, 96)
    bad_H = (ctypes.c_int * n)(240, 0, 375)
    b2 = ctypes.c_void_p()
    assert lib.dm_batch_create(n, bad_H, W, L, ctypes.byref(p), ctypes.byref(b2)) == dm.DM_ERR_ARG
    assert lib.dm_batch_destroy(b) == 0


def test_two_view_calls_check_arguments_without_gpu(lib):
    from paper_1601_06274_gb300 import dm
    p = dm.default_params()
    a, b = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.dm_create(8, 8, 16, ctypes.byref(p), ctypes.byref(a)) == 0
    assert lib.dm_create(8, 8, 16, ctypes.byref(p), ctypes.byref(b)) == 0
    fake = ctypes.c_void_p(4096)
    # no workspace bound yet: state errors, before anything reaches the device
    assert lib.dm_cost_volume_mirrored(a, fake, fake) == dm.DM_ERR_STATE
    assert lib.dm_solve_lr(a, b, fake, fake, 1, 1, 1.0, fake, fake, None) == dm.DM_ERR_STATE
    assert lib.dm_solve_lr(None, b, fake, fake, 1, 1, 1.0, fake, fake, None) == dm.DM_ERR_ARG
    # the check's arguments are validated on the host
    for H, W, md, ptrs in [(0, 4, 1.0, (fake, fake, fake, fake)),
                           (4, -1, 1.0, (fake, fake, fake, fake)),
                           (4, 4, -0.5, (fake, fake, fake, fake)),
                           (4, 4, float("nan"), (fake, fake, fake, fake)),
                           (4, 4, float("inf"), (fake, fake, fake, fake)),
                           (4, 4, 1.0, (None, fake, fake, fake)),
                           (4, 4, 1.0, (fake, None, fake, fake)),
                           (4, 4, 1.0, (fake, fake, None, fake)),
                           (4, 4, 1.0, (fake, fake, fake, None))]:
        ul, um, ok, out = ptrs
        assert lib.dm_lr_check(ul, um, H, W, md, ok, out, None, None) == dm.DM_ERR_ARG
    lib.dm_destroy(a)
    lib.dm_destroy(b)


def test_set_minorant_checks_arguments_without_gpu(lib):
    from paper_1601_06274_gb300 import dm
    p = dm.default_params()
    h = ctypes.c_void_p()
    assert lib.dm_create(8, 8, 16, ctypes.byref(p), ctypes.byref(h)) == 0
    assert lib.dm_set_minorant(h, 1, 0, 0, 0) == dm.DM_OK       # naive ignores the rest
    assert lib.dm_set_minorant(h, 2, 3, 1, 4) == dm.DM_OK
    assert lib.dm_set_minorant(h, 0, 0, 0, 0) == dm.DM_OK
    for args in [(3, 3, 1, 4), (-1, 3, 1, 4), (2, 0, 1, 4), (2, 65, 1, 4), (2, 3, 5, 4),
                 (2, 3, -1, 4), (2, 3, 1, 0), (2, 3, 1, 2000)]:
        assert lib.dm_set_minorant(h, *args) == dm.DM_ERR_ARG, args
    assert lib.dm_set_minorant(None, 0, 0, 0, 0) == dm.DM_ERR_ARG
    lib.dm_destroy(h)


def test_flow_calls_check_arguments_without_gpu(lib):
    from paper_1601_06274_gb300 import dm
    p = dm.default_params()
    a, b = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.dm_create(8, 8, 16, ctypes.byref(p), ctypes.byref(a)) == 0
    assert lib.dm_create(8, 8, 8, ctypes.byref(p), ctypes.byref(b)) == 0
    fake = ctypes.c_void_p(4096)
    n = ctypes.c_size_t()
    assert lib.dm_flow_refine_bytes(8, 8, ctypes.byref(n)) == 0 and n.value >= 23 * 8 * 8 * 4
    assert lib.dm_flow_refine_bytes(0, 8, ctypes.byref(n)) == dm.DM_ERR_ARG
    assert lib.dm_flow_cost_volumes(a, b, fake, fake, -2, -2) == dm.DM_ERR_STATE   # no workspace
    assert lib.dm_flow_cost_volumes(None, b, fake, fake, -2, -2) == dm.DM_ERR_ARG
    assert lib.dm_flow_refine(a, b, 10, fake, 1 << 20, fake, fake) == dm.DM_ERR_STATE
    lib.dm_destroy(a)
    lib.dm_destroy(b)


def test_batch_discrete_pass_needs_a_solve(lib):
    from paper_1601_06274_gb300 import dm
    p = dm.default_params()
    n = 2
    H = (ctypes.c_int * n)(8, 12)
    W = (ctypes.c_int * n)(16, 20)
    L = (ctypes.c_int * n)(16, 32)
    b = ctypes.c_void_p()
    assert lib.dm_batch_create(n, H, W, L, ctypes.byref(p), ctypes.byref(b)) == 0
    assert lib.dm_batch_discrete_pass(b, 0) == dm.DM_ERR_STATE
    assert lib.dm_batch_discrete_pass(b, 2) == dm.DM_ERR_ARG
    assert lib.dm_batch_discrete_pass(None, 0) == dm.DM_ERR_ARG
    lib.dm_batch_destroy(b)


def test_capture_and_replay_check_state_without_gpu(lib):
    from paper_1601_06274_gb300 import dm
    p = dm.default_params()
    h = ctypes.c_void_p()
    assert lib.dm_create(8, 8, 16, ctypes.byref(p), ctypes.byref(h)) == 0
    fake = ctypes.c_void_p(4096)
    assert lib.dm_capture(h, fake, fake, 2, 2, fake) == dm.DM_ERR_STATE
    assert lib.dm_replay(h) == dm.DM_ERR_STATE
    assert lib.dm_replay(None) == dm.DM_ERR_ARG
    lib.dm_destroy(h)


def test_noalloc_checks_arguments_without_gpu(lib):
    """dm_discrete_pass_noalloc refuses bad calls in host code, before it looks up
    its scratch array or launches anything (the pointers here are never used)."""
    from paper_1601_06274_gb300 import dm
    p = dm.default_params()
    lam_in, lam_out, err = ctypes.c_void_p(4096), ctypes.c_void_p(8192), ctypes.c_void_p(12288)

    def call(H, W, L, params, which, cost, lin, lout, e):
        pp = ctypes.byref(params) if params is not None else None
        return lib.dm_discrete_pass_noalloc(H, W, L, pp, which, cost, lam_in, lin, lout, e, None)

    # two int32 message arrays of 256 * 256 nodes * 128 labels: 64 MiB > 32 MiB of scratch
    assert call(256, 256, 128, p, 0, lam_in, lam_in, lam_out, err) == dm.DM_ERR_WORKSPACE
    assert call(8, 8, 16, None, 0, lam_in, lam_in, lam_out, err) == dm.DM_ERR_ARG
    assert call(8, 8, 16, p, 2, lam_in, lam_in, lam_out, err) == dm.DM_ERR_ARG        # which
    assert call(8, 8, 16, p, 0, None, lam_in, lam_out, err) == dm.DM_ERR_ARG         # rows need costs
    assert call(8, 8, 16, p, 0, lam_in, lam_in, lam_in, err) == dm.DM_ERR_ARG        # aliased output
    assert call(8, 8, 16, p, 0, lam_in, lam_in, lam_out, None) == dm.DM_ERR_ARG      # no error word
    assert call(0, 8, 16, p, 0, lam_in, lam_in, lam_out, err) == dm.DM_ERR_ARG
    assert call(8, 8, 1, p, 0, lam_in, lam_in, lam_out, err) == dm.DM_ERR_ARG
    assert call(8, 8, 257, p, 0, lam_in, lam_in, lam_out, err) == dm.DM_ERR_ARG
    for bad in (dm.default_params(w_hi=3), dm.default_params(tau=-1.0),
                dm.default_params(struct_size=8)):
        assert call(8, 8, 16, bad, 0, lam_in, lam_in, lam_out, err) == dm.DM_ERR_ARG
