"""Reverse and forward mode of the unrolled refinement on the GPU (the
differentiable form).

Gradients are with respect to the float cost volume, the per-pixel data
weights alpha and the regularisation weight lambda_r (and the start u0); the
loss is the L1 distance of the refined disparity to the synthetic ground truth.

* Where the FP32 and FP64 trajectories take the same branches (up to a few
  tens of iterations), the GPU gradient is compared with the FP64 oracle
  gradient (oracle.refine_grad) and the GPU tangent with FP64 central
  differences of the oracle forward.
* On the 512x256x96 workload with 200 iterations and a checkpoint every 20,
  the unrolled iteration amplifies perturbations (its FP64 central differences
  at h = 1e-3 and h/2 disagree along almost every direction, pinned in
  tests/test_oracle_continuous.py), so FP32 and FP64 trajectories part and
  their gradients with them.  There the reverse mode is checked against the
  forward mode on the GPU's own trajectory: <gu, J v> = <J^T gu, v> on 64
  random directions.
"""

import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_06274_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

G_TOL = 1e-3     # relative (L2) error of an FP32 gradient against the FP64 oracle
U_TOL = 1e-3     # px


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_06274_gb300 import build, dm as _dm
    build.build()
    return _dm


def _problem(H, W, L, seed, planes=4):
    """float cost (census cost + uniform noise, as float32), weights, alpha, u0, gt"""
    sp = S.make_pair(H, W, L, planes=planes, noise_sigma=2.0, seed=seed)
    rng = np.random.default_rng(seed + 1)
    cost = (O.cost_volume(sp.left, sp.right, L) + rng.uniform(0, 1, (H, W, L))).astype(np.float32)
    wh, wv = O.edge_weights(sp.left)
    alpha = rng.uniform(0.5, 1.5, (H, W)).astype(np.float32)
    # a start in general position: the argmin labels moved off the integers, so
    # that no comparison of the first iterations is an exact tie that FP32 and
    # FP64 could resolve differently
    # (and off the ends of the label range, where the clamped interpolation has
    # its kinks)
    u0 = np.argmin(cost, axis=2) + rng.uniform(-0.3, 0.3, (H, W))
    u0 = np.clip(u0, 0.1, L - 1.1).astype(np.float32)
    return sp, cost, wh, wv, alpha, u0


def _away_from_ties(gt, u_ref, margin=0.02):
    """ground truth moved off the oracle's refined disparity where they nearly tie,
    so that both sides take the same sign in the L1 loss"""
    gt = gt.astype(np.float64).copy()
    near = np.abs(u_ref - gt) < margin
    gt[near] = u_ref[near] + margin * np.where(gt[near] >= u_ref[near], 1.0, -1.0) * 2
    return gt


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-30))


def _gpu_grad(dm, ctx, cost, alpha, lam, u0, iters, ckpt, gt):
    import torch
    ctx.set_cost_volume_f32(cost)
    ctx.set_data_weights(alpha)
    ctx.set_lambda_r(lam)
    tape = ctx.refine_tape(iters, ckpt, u0)
    u = ctx.disparity()
    gtt = torch.as_tensor(gt, device=u.device)
    gu = (torch.sign(u.double() - gtt) / u.numel()).float()
    gc, ga, gl, g0 = ctx.refine_backward(gu, tape, u0=True)
    return (u.cpu().numpy().astype(np.float64), gc.cpu().numpy().astype(np.float64),
            ga.cpu().numpy().astype(np.float64), float(gl.cpu().numpy()[0]))


CASES = [  # H, W, L, iters, ckpt, warps, lambda_r
    (24, 40, 32, 30, 7, 5, 1.2),
    (17, 33, 16, 40, 20, 5, 1.0),
    (9, 70, 48, 25, 1, 3, 2.0),
    (40, 8, 24, 12, 50, 1, 0.7),
    (12, 20, 16, 3, 2, 5, 1.0),     # fewer iterations than warps
]


@pytest.mark.parametrize("H,W,L,iters,ckpt,warps,lam", CASES)
def test_gradient_matches_oracle(dm, H, W, L, iters, ckpt, warps, lam):
    sp, cost, wh, wv, alpha, u0 = _problem(H, W, L, seed=H * W + L)
    ctx = dm.Context(H, W, L, dm.default_params(warps=warps))
    ctx.set_cost_volume(np.zeros((H, W, L), np.uint8), wh, wv)
    P = O.Params(warps=warps, lambda_r=lam)
    c64, a64, u064 = cost.astype(np.float64), alpha.astype(np.float64), u0.astype(np.float64)
    ru, _, _ = O.refine(c64, wh.astype(float), wv.astype(float), u064, iters, P, a64)
    gt = _away_from_ties(sp.gt, ru)
    ou, oloss, ogc, oga, ogl = O.refine_grad(c64, wh.astype(float), wv.astype(float), u064, iters,
                                            gt, P, a64)
    u, gc, ga, gl = _gpu_grad(dm, ctx, cost, alpha, lam, u0, iters, ckpt, gt)
    assert np.abs(u - ou).max() <= U_TOL
    assert _rel(gc, ogc) <= G_TOL
    assert _rel(ga, oga) <= G_TOL
    assert gl == pytest.approx(ogl, rel=G_TOL, abs=1e-7)


def test_gradient_with_scalar_alpha(dm):
    # no per-pixel weights: the derivative in the scalar alpha is the sum
    H, W, L, iters = 20, 36, 32, 30
    sp, cost, wh, wv, _, u0 = _problem(H, W, L, seed=9)
    ctx = dm.Context(H, W, L, dm.default_params(alpha=0.8))
    ctx.set_cost_volume(np.zeros((H, W, L), np.uint8), wh, wv)
    P = O.Params(alpha=0.8, lambda_r=1.1)
    c64, u064 = cost.astype(np.float64), u0.astype(np.float64)
    a64 = np.full((H, W), 0.8)
    ru, _, _ = O.refine(c64, wh.astype(float), wv.astype(float), u064, iters, P, a64)
    gt = _away_from_ties(sp.gt, ru)
    _, _, ogc, oga, ogl = O.refine_grad(c64, wh.astype(float), wv.astype(float), u064, iters, gt,
                                        P, a64)
    u, gc, ga, gl = _gpu_grad(dm, ctx, cost, None, 1.1, u0, iters, 20, gt)
    assert _rel(gc, ogc) <= G_TOL
    assert ga.sum() == pytest.approx(oga.sum(), rel=G_TOL)
    assert gl == pytest.approx(ogl, rel=G_TOL)


def test_tape_forward_equals_refine(dm):
    H, W, L = 30, 50, 32
    sp, cost, wh, wv, alpha, u0 = _problem(H, W, L, seed=5)
    ctx = dm.Context(H, W, L)
    ctx.set_cost_volume(np.zeros((H, W, L), np.uint8), wh, wv)
    ctx.set_cost_volume_f32(cost)
    ctx.set_data_weights(alpha)
    ctx.refine(37, u0=u0)
    ref = ctx.disparity().cpu().numpy()
    for ckpt in (1, 6, 20, 100):
        ctx.refine_tape(37, ckpt, u0)
        assert np.array_equal(ctx.disparity().cpu().numpy(), ref)


def test_zero_iterations(dm):
    H, W, L = 8, 12, 16
    sp, cost, wh, wv, alpha, u0 = _problem(H, W, L, seed=6)
    ctx = dm.Context(H, W, L)
    ctx.set_cost_volume(np.zeros((H, W, L), np.uint8), wh, wv)
    ctx.set_cost_volume_f32(cost)
    tape = ctx.refine_tape(0, 20, u0)
    assert np.array_equal(ctx.disparity().cpu().numpy(), u0)
    import torch
    gu = torch.ones((H, W), device="cuda")
    gc, ga, gl, g0 = ctx.refine_backward(gu, tape, u0=True)
    assert float(gc.abs().max()) == 0 and float(ga.abs().max()) == 0 and float(gl[0]) == 0
    assert torch.equal(g0, gu)


def test_stale_tape_is_rejected(dm):
    H, W, L = 8, 12, 16
    sp, cost, wh, wv, alpha, u0 = _problem(H, W, L, seed=7)
    ctx = dm.Context(H, W, L)
    ctx.set_cost_volume(np.zeros((H, W, L), np.uint8), wh, wv)
    ctx.set_cost_volume_f32(cost)
    tape = ctx.refine_tape(10, 5, u0)
    ctx.set_lambda_r(2.0)
    import torch
    with pytest.raises(dm.DMError) as e:
        ctx.refine_backward(torch.zeros((H, W), device="cuda"), tape)
    assert e.value.code == dm.DM_ERR_STATE
    with pytest.raises(dm.DMError) as e:
        ctx.discrete(1)
    assert e.value.code == dm.DM_ERR_STATE


def test_autograd_function(dm):
    import torch
    H, W, L, iters = 16, 24, 32, 30
    sp, cost, wh, wv, alpha, u0 = _problem(H, W, L, seed=8)
    ctx = dm.Context(H, W, L)
    ctx.set_cost_volume(np.zeros((H, W, L), np.uint8), wh, wv)
    c = torch.tensor(cost, device="cuda", requires_grad=True)
    a = torch.tensor(alpha, device="cuda", requires_grad=True)
    lam = torch.tensor(1.3, dtype=torch.float64, requires_grad=True)
    u0t = torch.tensor(u0, device="cuda")
    gt = torch.tensor(sp.gt, device="cuda", dtype=torch.float32)
    u = dm.refine_differentiable(ctx, c, a, lam, u0t, iters, ckpt_every=8)
    # a second forward on the same context before the first backward
    u2 = dm.refine_differentiable(ctx, c, a, lam * 2, u0t, iters, ckpt_every=8)
    (u - gt).abs().mean().backward()
    # the same gradients through the plain calls
    ctx.set_cost_volume_f32(cost)
    ctx.set_data_weights(alpha)
    ctx.set_lambda_r(1.3)
    tape = ctx.refine_tape(iters, 8, u0)
    uu = ctx.disparity()
    assert torch.equal(uu, u.detach())
    gu = torch.sign(uu - gt) / uu.numel()
    gc, ga, gl, _ = ctx.refine_backward(gu, tape)
    assert torch.equal(c.grad, gc) and torch.equal(a.grad, ga)
    assert float(lam.grad) == pytest.approx(float(gl[0]), rel=1e-6)
    assert not torch.equal(u2, u)


# --- forward mode ------------------------------------------------------------------

@pytest.mark.parametrize("H,W,L,iters,lam", [(24, 40, 32, 12, 1.2), (16, 28, 48, 10, 0.8)])
def test_tangent_matches_fp64_central_differences(dm, H, W, L, iters, lam):
    """GPU tangent J v against central differences of the FP64 oracle forward
    (h = 1e-6 along joint directions in cost, alpha, lambda_r and u0); a
    direction whose quotients at h and h/2 disagree straddles a kink and is
    skipped.  The comparison is meaningful only while the FP32 and FP64
    trajectories take the same branches, which the first assertion checks."""
    import torch
    sp, cost, wh, wv, alpha, u0 = _problem(H, W, L, seed=H + W + L)
    # a start in general position 4 labels inside the range: the warps never
    # reach its ends, where the clamped interpolation has kinks that central
    # differences average over, and no two neighbours start equal (equal
    # neighbours meet exact ties after a few iterations)
    u0 = np.random.default_rng(3).uniform(4.1, L - 5.1, size=u0.shape).astype(np.float32)
    ctx = dm.Context(H, W, L)
    ctx.set_cost_volume(np.zeros((H, W, L), np.uint8), wh, wv)
    ctx.set_cost_volume_f32(cost)
    ctx.set_data_weights(alpha)
    ctx.set_lambda_r(lam)
    whf, wvf = wh.astype(float), wv.astype(float)
    c64, a64, u064 = cost.astype(float), alpha.astype(float), u0.astype(float)

    def fwd(c, a, l, uu):
        return O.refine(c, whf, wvf, uu, iters, O.Params(lambda_r=l), a)[0]
    ctx.refine(iters, u0=u0)
    assert np.abs(ctx.disparity().cpu().numpy() - fwd(c64, a64, lam, u064)).max() <= 2e-4
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(12):
        vc, va = rng.normal(size=cost.shape), rng.normal(size=alpha.shape)
        vl, vu = rng.normal(), rng.normal(size=u0.shape)
        du = ctx.refine_jvp(iters, u0, vu.astype(np.float32), vc.astype(np.float32),
                            va.astype(np.float32), vl).cpu().numpy().astype(float)
        vc, va, vu = (v.astype(np.float32).astype(float) for v in (vc, va, vu))
        vl = float(np.float32(vl))

        def q(h):
            return (fwd(c64 + h * vc, a64 + h * va, lam + h * vl, u064 + h * vu)
                    - fwd(c64 - h * vc, a64 - h * va, lam - h * vl, u064 - h * vu)) / (2 * h)
        f1, f2 = q(1e-6), q(5e-7)
        if np.abs(f1 - f2).max() > 1e-6 * max(np.abs(f1).max(), 1.0):
            continue
        checked += 1
        assert _rel(du, f1) <= G_TOL
    assert checked >= 8


def test_gradient_matches_fp64_central_differences(dm):
    """GPU gradient against central differences (h = 1e-3) of the FP64 oracle
    forward along 64 random unit directions in (cost, alpha, lambda_r).  A
    direction whose quotients at h and h/2 differ by more than 1e-4 straddles a
    kink and is counted, not compared.  The case is one where the FP32 and FP64
    trajectories take the same branches (checked first); with many more
    iterations or pixels they part (see the module docstring)."""
    from concurrent.futures import ThreadPoolExecutor
    H, W, L, iters, lam = 24, 40, 32, 30, 1.2
    sp, cost, wh, wv, alpha, u0 = _problem(H, W, L, seed=H * W + L)
    whf, wvf = wh.astype(float), wv.astype(float)
    c64, a64, u064 = cost.astype(float), alpha.astype(float), u0.astype(float)
    ru = O.refine(c64, whf, wvf, u064, iters, O.Params(lambda_r=lam), a64)[0]
    gt = _away_from_ties(sp.gt, ru)
    ctx = dm.Context(H, W, L)
    ctx.set_cost_volume(np.zeros((H, W, L), np.uint8), wh, wv)
    u, gc, ga, gl = _gpu_grad(dm, ctx, cost, alpha, lam, u0, iters, 20, gt)
    assert np.abs(u - ru).max() <= 2e-4

    def lossf(c, a, l):
        return np.abs(O.refine(c, whf, wvf, u064, iters, O.Params(lambda_r=l), a)[0] - gt).mean()
    n = cost.size + alpha.size + 1

    def one(seed):
        v = np.random.default_rng(seed).standard_normal(n)
        v /= np.linalg.norm(v)
        vc, va, vl = v[:cost.size].reshape(cost.shape), v[cost.size:-1].reshape(alpha.shape), v[-1]

        def q(h):
            return (lossf(c64 + h * vc, a64 + h * va, lam + h * vl)
                    - lossf(c64 - h * vc, a64 - h * va, lam - h * vl)) / (2 * h)
        f1, f2 = q(1e-3), q(5e-4)
        return f1, f2, float((gc * vc).sum() + (ga * va).sum() + gl * vl)
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        res = list(ex.map(one, range(1000, 1064)))
    errs = [abs(an - f1) / abs(f1) for f1, f2, an in res if abs(f1 - f2) <= 1e-4 * abs(f1)]
    print(f"{len(errs)} of 64 directions kink-free, max rel error {max(errs, default=0):.2e}")
    assert len(errs) >= 8
    assert max(errs) <= G_TOL


DIFF = dict(H=256, W=512, L=96, iters=200, ckpt=20, seed=0)


def test_adjoint_is_transpose_of_tangent_512x256x96(dm):
    """<gu, J v> = <J^T gu, v> on the 512x256x96 workload (200 iterations, a
    checkpoint every 20) for 64 random directions in (cost, alpha, lambda_r, u0)"""
    import torch
    H, W, L = DIFF["H"], DIFF["W"], DIFF["L"]
    sp, cost, wh, wv, alpha, u0 = _problem(H, W, L, seed=DIFF["seed"], planes=8)
    ctx = dm.Context(H, W, L)
    ctx.set_cost_volume(np.zeros((H, W, L), np.uint8), wh, wv)
    ct, at = torch.tensor(cost, device="cuda"), torch.tensor(alpha, device="cuda")
    u0t = torch.tensor(u0, device="cuda")
    ctx.set_cost_volume_f32(ct)
    ctx.set_data_weights(at)
    ctx.set_lambda_r(1.0)
    tape = ctx.refine_tape(DIFF["iters"], DIFF["ckpt"], u0t)
    u = ctx.disparity().clone()
    gt = torch.tensor(sp.gt, device="cuda", dtype=torch.float64)
    gu = (torch.sign(u.double() - gt) / u.numel()).float()
    gc, ga, gl, g0 = ctx.refine_backward(gu, tape, u0=True)
    gl = float(gl.cpu()[0])
    g = torch.Generator(device="cuda").manual_seed(1234)
    worst = 0.0
    for _ in range(64):
        vc = torch.randn(cost.shape, device="cuda", generator=g)
        va = torch.randn(alpha.shape, device="cuda", generator=g)
        vu = torch.randn(alpha.shape, device="cuda", generator=g)
        vl = float(torch.randn((), device="cuda", generator=g))
        du = ctx.refine_jvp(DIFF["iters"], u0t, vu, vc, va, vl)
        assert torch.equal(ctx.disparity(), u)   # the same trajectory
        prod = gu.double() * du.double()
        lhs = float(prod.sum())
        rhs = float((gc.double() * vc).sum() + (ga.double() * va).sum()
                    + (g0.double() * vu).sum()) + gl * vl
        # relative to the sum of the magnitudes of the products (the scale of the
        # FP32 rounding in either sum), not to their sum, which may cancel
        worst = max(worst, abs(lhs - rhs) / float(prod.abs().sum()))
    print(f"dot-product identity: worst relative difference {worst:.2e}")
    assert worst <= 1e-4


# Config 3's depth: 200 iterations, a checkpoint every 20, 5 warps.  The unrolled
# map is kinked at the 1e-3 scale on almost every instance (see the module
# docstring); in the convex regime (C -> infinity, so q = 0) with a weak
# regulariser, some crops are smooth at that scale along nearly every
# direction, and there the FP32 and FP64 trajectories take the same branches.
# These two were found so by the same h / h/2 test the check applies.
DEEP = [(4, 128, 96, 15), (6, 128, 96, 4)]   # H, W, L, seed


@pytest.mark.parametrize("H,W,L,seed", DEEP)
def test_gradient_at_200_iterations_matches_oracle_and_central_differences(dm, H, W, L, seed):
    iters, ckpt, warps, lam, C = 200, 20, 5, 0.05, 1e7
    sp = S.make_pair(H, W, L, planes=4, noise_sigma=2.0, seed=seed)
    rng = np.random.default_rng(seed + 1)
    cost = (O.cost_volume(sp.left, sp.right, L) + rng.uniform(0, 1, (H, W, L))).astype(np.float32)
    wh, wv = O.edge_weights(sp.left)
    alpha = rng.uniform(0.5, 1.5, (H, W)).astype(np.float32)
    u0 = np.clip(np.argmin(cost, 2) + rng.uniform(-0.3, 0.3, (H, W)), 0.1, L - 1.1).astype(np.float32)
    c64, a64, u064 = cost.astype(np.float64), alpha.astype(np.float64), u0.astype(np.float64)
    whf, wvf = wh.astype(float), wv.astype(float)
    P = O.Params(C=C, lambda_r=lam, warps=warps)
    ru, _, _ = O.refine(c64, whf, wvf, u064, iters, P, a64)
    gt = _away_from_ties(sp.gt, ru)
    ou, _, ogc, oga, ogl = O.refine_grad(c64, whf, wvf, u064, iters, gt, P, a64)
    ctx = dm.Context(H, W, L, dm.default_params(warps=warps, C=C))
    ctx.set_cost_volume(np.zeros((H, W, L), np.uint8), wh, wv)
    u, gc, ga, gl = _gpu_grad(dm, ctx, cost, alpha, lam, u0, iters, ckpt, gt)
    # the FP32 trajectory stays on the FP64 one
    assert np.abs(u - ou).max() <= U_TOL
    # the GPU reverse mode against the oracle's FP64 reverse mode
    assert _rel(gc, ogc) <= G_TOL
    assert _rel(ga, oga) <= G_TOL
    assert gl == pytest.approx(ogl, rel=G_TOL, abs=1e-7)
    # 64 central differences at h = 1e-3 of the FP64 forward;
    # a direction whose quotients at h and h/2 differ straddles a kink
    def lossf(c, a, l):
        uu = O.refine(c, whf, wvf, u064, iters, O.Params(C=C, lambda_r=l, warps=warps), a)[0]
        return np.abs(uu - gt).mean()
    drng = np.random.default_rng(7)
    smooth, errs = 0, []
    for _ in range(64):
        v = drng.standard_normal(cost.size + alpha.size + 1)
        v /= np.linalg.norm(v)
        vc, va, vl = v[:cost.size].reshape(cost.shape), v[cost.size:-1].reshape(alpha.shape), v[-1]

        def q(h):
            return (lossf(c64 + h * vc, a64 + h * va, lam + h * vl)
                    - lossf(c64 - h * vc, a64 - h * va, lam - h * vl)) / (2 * h)
        f1, f2 = q(1e-3), q(5e-4)
        if abs(f1 - f2) > 1e-4 * max(abs(f1), 1e-9):
            continue
        smooth += 1
        an = float((gc * vc).sum() + (ga * va).sum() + gl * vl)
        errs.append(abs(an - f1) / max(abs(f1), 1e-9))
    assert smooth >= 56, f"only {smooth} of 64 directions free of kinks"
    assert max(errs) <= G_TOL
