"""Parity of the two-view path and the consistency check (Sec. 4.1.1) with the
CPU oracle, through the C ABI.

* The mirrored cost volume and edge weights: bit-exact against the oracle's
  right-view cost written from its definition, up to 1242x375x128.
* The mirrored problem's Dual MM: bit-exact labels and lower bounds; its
  refinement within 1e-3 px of the FP64 oracle started from the same labels.
* The check kernel: bit-exact against the oracle's check on the same float32
  disparities (ties, borders, thresholds, non-finite values).
* dm_solve_lr: each view identical to the single-view path, the check identical
  to the oracle's on the GPU's disparities, and against the oracle's own
  two-view result the masks differ only where a disparity sits within the
  refinement's tolerance of a decision boundary.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_06274_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

U_TOL = 1e-3


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_06274_gb300 import build, dm as _dm
    build.build()
    return _dm


def _mirror(a):
    return a[:, ::-1].copy()


def _np(t):
    return t.cpu().numpy()


SHAPES = [(24, 40, 16), (1, 37, 8), (17, 1, 8), (13, 29, 33), (9, 21, 64), (5, 11, 128)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("cost_bytes", [1, 2])
def test_mirrored_cost_volume_is_the_right_view(dm, shape, cost_bytes):
    H, W, L = shape
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=H * 7 + W)
    ctx = dm.Context(H, W, L, dm.default_params(cost_bytes=cost_bytes))
    ctx.cost_volume_mirrored(sp.left, sp.right)
    c, wh, wv = ctx.cost()
    c = _np(c).astype(np.int64) if cost_bytes == 1 else _np(c).view(np.uint16).astype(np.int64)
    ref = O.cost_volume_right(sp.left, sp.right, L)
    assert np.array_equal(c[:, ::-1, :], ref)
    rwh, rwv = O.edge_weights(_mirror(sp.right))
    assert np.array_equal(_np(wh), rwh) and np.array_equal(_np(wv), rwv)


@pytest.mark.parametrize("shape", SHAPES)
def test_mirrored_problem_matches_oracle(dm, shape):
    H, W, L = shape
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=H + W * 3)
    ml, mr = _mirror(sp.right), _mirror(sp.left)
    ctx = dm.Context(H, W, L)
    ctx.cost_volume_mirrored(sp.left, sp.right)
    lb = ctx.discrete(4, lower_bounds=True)
    cost = O.cost_volume(ml, mr, L)
    wh, wv = O.edge_weights(ml)
    rl, rlb, _, _ = O.dmm(cost, wh, wv, 4)
    assert np.array_equal(dm.labels_u16(ctx.labels()), rl) and np.array_equal(lb, rlb)
    ctx.refine(30)
    u = _np(ctx.disparity())
    ru, _, _ = O.refine(cost.astype(np.float64), wh.astype(np.float64), wv.astype(np.float64),
                        rl.astype(np.float64), 30)
    assert np.abs(u - ru).max() <= U_TOL


def _check_inputs(H, W, seed):
    rng = np.random.default_rng(seed)
    ul = rng.uniform(-2, 20, size=(H, W)).astype(np.float32)
    ties = rng.random((H, W)) < 0.15
    ul[ties] = np.floor(ul[ties]) + 0.5                   # rint ties
    ur = rng.uniform(-2, 20, size=(H, W)).astype(np.float32)
    # make about half the pixels consistent, some exactly at the threshold
    ys, xs = np.nonzero(rng.random((H, W)) < 0.5)
    xr = xs - np.rint(ul[ys, xs]).astype(np.int64)
    inside = (xr >= 0) & (xr < W)
    ys, xs, xr = ys[inside], xs[inside], xr[inside]
    delta = rng.choice(np.array([0.0, 0.25, -1.0, 1.0, 1.0000001, -0.999], np.float32),
                       size=len(ys))
    ur[ys, xr] = ul[ys, xs] + delta
    ul.flat[rng.integers(0, H * W, 3)] = np.nan
    ul.flat[rng.integers(0, H * W, 3)] = np.inf
    return ul, ur


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (37, 61), (375, 1242)])
@pytest.mark.parametrize("max_diff", [0.0, 1.0, 2.5])
def test_check_kernel_bit_exact(dm, shape, max_diff):
    import torch
    H, W = shape
    ul, ur = _check_inputs(H, W, H * W + int(max_diff * 4))
    ok_ref, out_ref = O.lr_check(ul, ur, max_diff)
    um = torch.from_numpy(_mirror(ur)).cuda()
    out, ok, ur_gpu = dm.lr_check(torch.from_numpy(ul).cuda(), um, max_diff)
    torch.cuda.synchronize()
    assert np.array_equal(_np(ok), ok_ref)
    assert np.array_equal(_np(out).view(np.uint32), out_ref.view(np.uint32))
    assert np.array_equal(_np(ur_gpu).view(np.uint32), ur.view(np.uint32))


def test_check_rejects_bad_arguments(dm):
    import torch
    u = torch.zeros((4, 4), device="cuda")
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(dm.DMError):
            dm.lr_check(u, u, bad)


@pytest.mark.parametrize("shape,iters", [((24, 40, 16), (4, 30)), ((31, 57, 32), (5, 40)),
                                         ((8, 96, 64), (3, 20))])
def test_solve_lr_small_against_oracle(dm, shape, iters):
    H, W, L = shape
    dmm_iters, pd_iters = iters
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=W)
    s = dm.StereoLR(H, W, L)
    u, ok, ur = s.solve(sp.left, sp.right, dmm_iters, pd_iters, 1.0)
    s.sync()
    ul = _np(s.left.disparity())
    ur = _np(ur)
    ref = O.solve_lr(sp.left, sp.right, L, dmm_iters, pd_iters)
    # both discrete stages bit-exact, both refinements within tolerance
    assert np.array_equal(dm.labels_u16(s.left.labels()), ref["left"]["labels"])
    assert np.array_equal(dm.labels_u16(s.right.labels()), ref["mirrored"]["labels"])
    assert np.abs(ul - ref["u_left"]).max() <= U_TOL
    assert np.abs(ur - ref["u_right"]).max() <= U_TOL
    # the check on the GPU's own disparities: bit-exact
    ok_g, out_g = O.lr_check(ul, ur, 1.0)
    assert np.array_equal(_np(ok), ok_g) and np.array_equal(_np(u), out_g)
    # against the oracle's own disparities the masks may differ only where a
    # disparity is within the tolerance of a decision (rounding or threshold)
    diff = _np(ok) != ref["ok"]
    if diff.any():
        ys, xs = np.nonzero(diff)
        d = ref["u_left"][ys, xs].astype(np.float64)
        near_tie = np.abs(d - np.floor(d) - 0.5) <= 2 * U_TOL
        xr = xs - np.rint(d).astype(np.int64)
        xr_c = np.clip(xr, 0, W - 1)
        margin = np.abs(np.abs(d - ref["u_right"][ys, xr_c]) - 1.0)
        assert np.all(near_tie | (margin <= 2 * U_TOL))


def test_solve_lr_module_function(dm):
    sp = S.make_pair(20, 33, 16, planes=3, seed=9)
    u, ok, ul, ur = dm.solve_lr(sp.left, sp.right, 16, dmm_iters=3, pd_iters=20)
    assert u.shape == ok.shape == ul.shape == ur.shape == (20, 33)
    okn, un = _np(ok), _np(u)
    assert np.array_equal(un[okn == 1], _np(ul)[okn == 1]) and np.all(un[okn == 0] == -1)


def test_solve_lr_full_frame(dm):
    """1242x375x128: the left view is the single-view path bit for bit, the
    right view is the mirrored problem's path bit for bit, the right view's
    cost volume is the oracle's, and the check is the oracle's check on the
    GPU's disparities; on the synthetic scene most pixels pass."""
    import torch
    spec = S.KITTI
    pair = S.make_workload(spec, seed=0)
    H, W, L = spec["H"], spec["W"], spec["L"]
    s = dm.StereoLR(H, W, L)
    u, ok, ur = s.solve(pair.left, pair.right, 10, 100, 1.0)
    s.sync()
    single = dm.Context(H, W, L)
    u1 = single.solve(pair.left, pair.right, 10, 100)
    assert torch.equal(s.left.disparity(), u1)
    mirrored = dm.Context(H, W, L)
    mirrored.cost_volume_mirrored(pair.left, pair.right)
    mirrored.discrete(10)
    mirrored.refine(100)
    um = mirrored.disparity()
    assert torch.equal(ur, torch.flip(um, dims=[1]))
    c, _, _ = mirrored.cost()
    assert np.array_equal(_np(c)[:, ::-1, :], O.cost_volume_right(pair.left, pair.right, L)
                          .astype(np.uint8))
    ok_g, out_g = O.lr_check(_np(u1), _np(ur), 1.0)
    assert np.array_equal(_np(ok), ok_g) and np.array_equal(_np(u), out_g)
    assert ok_g.mean() > 0.8


def test_solve_lr_with_uint16_costs(dm):
    """Two views with uint16 cost storage give the same result as uint8."""
    H, W, L = 20, 36, 32
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=5)
    a = dm.StereoLR(H, W, L)
    b = dm.StereoLR(H, W, L, dm.default_params(cost_bytes=2))
    ua, oka, ura = a.solve(sp.left, sp.right, 3, 20, 1.0)
    ub, okb, urb = b.solve(sp.left, sp.right, 3, 20, 1.0)
    a.sync()
    b.sync()
    assert np.array_equal(_np(oka), _np(okb))
    assert np.array_equal(_np(ua), _np(ub)) and np.array_equal(_np(ura), _np(urb))


@pytest.mark.parametrize("shape", [(1, 17, 8), (9, 1, 8), (2, 3, 4)])
def test_solve_lr_degenerate_shapes(dm, shape):
    H, W, L = shape
    sp = S.make_pair(H, W, L, planes=2, noise_sigma=2.0, seed=H * W)
    u, ok, ul, ur = dm.solve_lr(sp.left, sp.right, L, dmm_iters=2, pd_iters=10)
    ref = O.solve_lr(sp.left, sp.right, L, 2, 10)
    assert np.abs(_np(ul) - ref["u_left"]).max() <= U_TOL
    assert np.abs(_np(ur) - ref["u_right"]).max() <= U_TOL
    ok_g, out_g = O.lr_check(_np(ul), _np(ur), 1.0)
    assert np.array_equal(_np(ok), ok_g) and np.array_equal(_np(u), out_g)
