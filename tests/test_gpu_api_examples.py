"""The public Python API used the way a caller would: one pair, a context, a
batch, the differentiable refinement through autograd, and a warm-started
sequence with uint16 costs (the usage shown in the repository's overview)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_api_walkthrough():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_06274_gb300 import build, dm, synthetic
    build.build()
    pair = synthetic.make_workload(synthetic.KITTI, seed=0)
    H, W, L = 375, 1242, 128

    u, labels, lb = dm.solve(pair.left, pair.right, L=L, dmm_iters=10, pd_iters=100)
    assert u.shape == (H, W) and labels.shape == (H, W) and lb.shape == (10,)
    assert np.all(np.diff(lb) >= 0)

    ctx = dm.Context(H, W, L)
    u2 = ctx.solve(pair.left, pair.right, 10, 100)
    assert torch.equal(u, u2) and np.isfinite(ctx.energy())

    out = dm.batch_solve([(pair.left, pair.right)], labels=[L], dmm_iters=10, pd_iters=100)
    assert torch.equal(out[0][0], u) and np.array_equal(out[0][1], labels)

    cost = torch.rand(H, W, L, device="cuda", requires_grad=True)
    alpha = torch.ones(H, W, device="cuda", requires_grad=True)
    lam = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    ctx.cost_volume(pair.left, pair.right)
    ctx.discrete(10)
    ur = dm.refine_differentiable(ctx, cost, alpha, lam, None, iters=200, ckpt_every=20)
    ur.sum().backward()
    assert cost.grad.shape == cost.shape and alpha.grad.shape == alpha.shape
    assert lam.grad is not None and torch.isfinite(cost.grad).all()

    sctx = dm.Context(H, W, L, dm.default_params(cost_bytes=2))
    s0 = sctx.solve(pair.left, pair.right, 10, 100)
    assert torch.equal(s0, u)   # uint16 storage of the same costs gives the same result
    s1 = sctx.solve_next(pair.left, pair.right, 10, 100)
    assert s1.shape == (H, W)

    u_chk, ok, u_left, u_right = dm.solve_lr(pair.left, pair.right, L=L, dmm_iters=10,
                                             pd_iters=100)
    assert torch.equal(u_left, u) and ok.dtype == torch.uint8 and u_right.shape == (H, W)

    ctx.set_minorant("iterative", max_pass=3, gamma=(1, 4))
    ctx.cost_volume(pair.left, pair.right)
    lb_it = ctx.discrete(3, lower_bounds=True)
    assert ctx.path()[0] == 32 and lb_it.shape == (3,)

    fp = synthetic.make_flow_workload(synthetic.FLOW)
    d1, d2 = dm.solve_flow(fp.img1, fp.img2, lo1=-32, K1=64, lo2=-32, K2=64, dmm_iters=10,
                           pd_iters=100)
    assert d1.shape == (480, 640) and bool(torch.isfinite(d2).all())
