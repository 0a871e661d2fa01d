"""The refinement in one cooperative launch (pd_launch = 0, the default: the
state in shared memory, one region per SM; pd_launch = 2: the state in global
memory with grid barriers) against one launch per iteration (pd_launch = 1):
the same iterates of Eq. cont_iterates (Sec. 2.4) with the data term of
Sec. 3.1, so the refined disparity and the energy agree bit for bit; and the
bounded waits between iterations, which give up with DM_ERR_TIMEOUT and leave
the context usable."""

import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_06274_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_06274_gb300 import build, dm as _dm
    build.build()
    return _dm


def _solve(dm, sp, H, W, L, dmm, pd, launch, **kw):
    ctx = dm.Context(H, W, L, dm.default_params(pd_launch=launch, **kw))
    u = ctx.solve(sp.left, sp.right, dmm, pd).cpu().numpy()
    return ctx, u, ctx.energy()


@pytest.mark.parametrize("H,W,L,pd,warps", [(1, 1, 2, 3, 1), (1, 40, 16, 7, 5), (37, 1, 16, 7, 5),
                                            (9, 33, 32, 0, 5), (17, 65, 64, 1, 5),
                                            (31, 97, 64, 23, 5), (120, 200, 64, 100, 5),
                                            (375, 1242, 128, 100, 5), (64, 64, 32, 40, 1)])
def test_one_launch_equals_launch_per_iteration(dm, H, W, L, pd, warps):
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=H * 7 + W)
    _, u1, e1 = _solve(dm, sp, H, W, L, 3, pd, 1, warps=warps)
    for launch in (0, 2):   # shared-memory regions (where they fit), grid barriers
        _, u, e = _solve(dm, sp, H, W, L, 3, pd, launch, warps=warps)
        assert np.array_equal(u.view(np.uint32), u1.view(np.uint32)), launch
        assert e == e1


def test_one_launch_from_a_given_start_and_float_costs(dm):
    H, W, L, iters = 40, 72, 32, 30
    rng = np.random.default_rng(5)
    cost = rng.uniform(0, 20, (H, W, L)).astype(np.float32)
    u_start = rng.uniform(0, L - 1, (H, W)).astype(np.float32)
    w8 = np.full((H, W), 8, dtype=np.uint8)
    out = []
    for launch in (0, 1, 2):
        ctx = dm.Context(H, W, L, dm.default_params(pd_launch=launch))
        ctx.set_cost_volume_f32(cost, w8, w8)
        ctx.refine(iters, u0=u_start)
        out.append(ctx.disparity().cpu().numpy())
    assert np.array_equal(out[0].view(np.uint32), out[1].view(np.uint32))
    assert np.array_equal(out[2].view(np.uint32), out[1].view(np.uint32))
    # and the oracle, within 1e-3 plus its own float32 spread (random costs
    # leave a few dozen pixels where float32 does not determine the result)
    args = (cost.astype(float), w8.astype(float), w8.astype(float), u_start.astype(float), iters)
    ru, _, _ = O.refine(*args)
    spread = O.fp32_spread(*args)
    assert (np.abs(out[0] - ru) - spread).max() <= 1e-3


@pytest.mark.parametrize("launch", [0, 2])
def test_wait_gives_up_and_the_context_stays_usable(dm, launch):
    """wait_test = 1: the first wait (a neighbour's progress counter, or the
    grid barrier) waits for progress that never comes; every CTA gives up after
    its bounded wait (20 ms in this mode) and returns, and the next
    synchronising call reports DM_ERR_TIMEOUT once."""
    import torch
    H, W, L = 48, 64, 16   # three regions of the shared-memory form
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=3)
    ctx = dm.Context(H, W, L, dm.default_params(wait_test=1, pd_launch=launch))
    ctx.cost_volume(sp.left, sp.right)
    ctx.discrete(2)
    t0 = time.time()
    ctx.refine(20)
    with pytest.raises(dm.DMError) as e:
        ctx.energy()
    assert e.value.code == dm.DM_ERR_TIMEOUT
    assert time.time() - t0 < 10.0
    # reported once; the context's other stages work as before
    cost = O.cost_volume(sp.left, sp.right, L)
    wh, wv = O.edge_weights(sp.left)
    ctx.reset_duals()
    lb = ctx.discrete(2, lower_bounds=True)
    _, rlb, _, _ = O.dmm(cost, wh, wv, 2)
    assert np.array_equal(lb, rlb)
    # and a context without the test skew refines on the same device
    ok = dm.Context(H, W, L)
    u = ok.solve(sp.left, sp.right, 2, 20).cpu().numpy()
    torch.cuda.synchronize()
    assert np.isfinite(ok.energy()) and np.all(np.isfinite(u))
