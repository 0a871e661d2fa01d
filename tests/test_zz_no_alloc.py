"""The allocation-free pass (dm_discrete_pass_noalloc) against the context API.

dm_discrete_pass_noalloc serves callers that cannot allocate device memory:
it takes only inputs and outputs and keeps its scratch in a fixed array
inside libdm.so.  Here it must reproduce, bit for bit, the duals that the
workspace-based dm_discrete_pass computes for the same inputs, on calls made
back to back (the fixed scratch keeps the previous call's contents).
"""

import ctypes

import numpy as np
import pytest

from paper_1601_06274_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_06274_gb300 import build, dm as _dm
    build.build()
    return _dm


@pytest.mark.parametrize("H,W,L", [(40, 72, 48), (33, 57, 128), (7, 5, 16)])
def test_noalloc_matches_context_passes(dm, H, W, L):
    import torch
    sp = S.make_pair(H, W, L, planes=3, seed=H + W + L)
    ctx = dm.Context(H, W, L)
    ctx.cost_volume(sp.left, sp.right)
    cost, wh, wv = ctx.cost()
    ref = []
    for it in range(2):
        ctx.discrete_pass(0)
        lh, _ = ctx.duals()
        ctx.discrete_pass(1)
        _, lv = ctx.duals()
        ref.append((lh.clone(), lv.clone()))
    ctx.sync()

    p = dm.default_params()
    lam_v = torch.zeros((H, W, L), dtype=torch.int32, device="cuda")
    lam_h = torch.empty_like(lam_v)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for it in range(2):
        dm.discrete_pass_noalloc(p, 0, cost, wh, lam_v, lam_h, err, stream)
        new_v = torch.empty_like(lam_v)
        dm.discrete_pass_noalloc(p, 1, None, wv, lam_h, new_v, err, stream)
        torch.cuda.synchronize()
        assert torch.equal(lam_h, ref[it][0]), f"lambda_h, iteration {it}"
        assert torch.equal(new_v, ref[it][1]), f"lambda_v, iteration {it}"
        lam_v = new_v
    assert int(err.item()) == 0


def test_noalloc_default_stream_and_error_word(dm):
    import torch
    H, W, L = 9, 13, 16
    cost = torch.zeros((H, W, L), dtype=torch.uint8, device="cuda")
    wh = torch.full((H, W), 3, dtype=torch.uint8, device="cuda")  # no integer penalty table
    wv = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    lam_in = torch.zeros((H, W, L), dtype=torch.int32, device="cuda")
    out = torch.empty_like(lam_in)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    dm.discrete_pass_noalloc(dm.default_params(), 0, cost, wh, lam_in, out, err, None)
    torch.cuda.synchronize()
    assert int(err.item()) != 0


def test_noalloc_rejects_too_large_and_bad_arguments(dm):
    import torch
    p = dm.default_params()
    lib = dm.lib()
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    other = torch.zeros(16, dtype=torch.int32, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    optr = ctypes.c_void_p(other.data_ptr())
    # 2 * 256 * 256 * 128 * 4 bytes = 64 MiB > 32 MiB of fixed scratch
    rc = lib.dm_discrete_pass_noalloc(256, 256, 128, ctypes.byref(p), 0, ptr, ptr, ptr, optr, ptr,
                                      None)
    assert rc == dm.DM_ERR_WORKSPACE
    assert lib.dm_discrete_pass_noalloc(8, 8, 16, ctypes.byref(p), 2, ptr, ptr, ptr, optr, ptr,
                                        None) == dm.DM_ERR_ARG
    assert lib.dm_discrete_pass_noalloc(8, 8, 16, ctypes.byref(p), 0, None, ptr, ptr, optr, ptr,
                                        None) == dm.DM_ERR_ARG
    bad = dm.default_params(w_hi=3)
    assert lib.dm_discrete_pass_noalloc(8, 8, 16, ctypes.byref(bad), 0, ptr, ptr, ptr, optr, ptr,
                                        None) == dm.DM_ERR_ARG
    # the error word is required, the output must not alias the input, and the
    # parameters are checked as dm_create checks them
    assert lib.dm_discrete_pass_noalloc(8, 8, 16, ctypes.byref(p), 0, ptr, ptr, ptr, optr, None,
                                        None) == dm.DM_ERR_ARG
    assert lib.dm_discrete_pass_noalloc(8, 8, 16, ctypes.byref(p), 0, ptr, ptr, ptr, ptr, ptr,
                                        None) == dm.DM_ERR_ARG
    neg = dm.default_params(tau=-1.0)
    assert lib.dm_discrete_pass_noalloc(8, 8, 16, ctypes.byref(neg), 0, ptr, ptr, ptr, optr, ptr,
                                        None) == dm.DM_ERR_ARG


def test_noalloc_binding_checks_its_tensors(dm):
    import torch
    H, W, L = 6, 7, 16
    p = dm.default_params()
    cost = torch.zeros((H, W, L), dtype=torch.uint8, device="cuda")
    wh = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    lam = torch.zeros((H, W, L), dtype=torch.int32, device="cuda")
    out = torch.empty_like(lam)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for args in [(cost.int(), wh, lam, out, err),               # cost of the wrong type
                 (cost, wh[:, :-1], lam, out, err),              # weights of the wrong shape
                 (cost, wh, lam.transpose(0, 1), out, err),      # not contiguous
                 (cost, wh, lam, lam, err),                      # output aliases the input
                 (cost, wh, lam, out, None)]:                    # no error word
        with pytest.raises(dm.DMError):
            dm.discrete_pass_noalloc(p, 0, *args)
