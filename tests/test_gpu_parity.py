"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Discrete stage: bit-exact (cost volume, edge weights, both duals after every
pass, labels, lower bounds).  Continuous stage: FP32 GPU vs FP64 oracle,
max |u - u_oracle| <= 1e-3 px and relative energy error <= 1e-5.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_06274_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

U_TOL = 1e-3        # px, max-abs on the refined disparity
E_TOL = 1e-5        # relative, continuous energy


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_06274_gb300 import build, dm as _dm
    build.build()
    return _dm


def _ctx(dm, H, W, L, **params):
    return dm.Context(H, W, L, dm.default_params(**params))


def _pair(H, W, L, seed):
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=seed)
    return sp.left, sp.right


def _np(t):
    return t.cpu().numpy()


def _oparams(dmp):
    return O.Params(census_win=dmp.census_win, edge_T=dmp.edge_threshold, w_hi=dmp.w_hi,
                    w_lo=dmp.w_lo, eps=dmp.eps, delta=dmp.delta, C=dmp.C,
                    lambda_r=dmp.lambda_r, alpha=dmp.alpha, tau=dmp.tau, sigma=dmp.sigma,
                    h=dmp.h, warps=dmp.warps)


SHAPES = [(48, 64, 16), (1, 37, 8), (23, 1, 8), (1, 1, 4), (13, 29, 2), (11, 17, 17), (9, 21, 33),
          (7, 19, 64), (6, 13, 100), (5, 11, 128), (4, 9, 129), (3, 7, 256)]


# --- cost volume --------------------------------------------------------------

@pytest.mark.parametrize("H,W,L", SHAPES)
@pytest.mark.parametrize("win", [3, 5])
def test_cost_volume_bit_exact(dm, H, W, L, win):
    left, right = _pair(H, W, L, seed=H * 1000 + W + L)
    ctx = _ctx(dm, H, W, L, census_win=win)
    ctx.cost_volume(left, right)
    c, wh, wv = ctx.cost()
    ctx.sync()
    P = O.Params(census_win=win)
    ref = O.cost_volume(left, right, L, win)
    rwh, rwv = O.edge_weights(left, P)
    assert np.array_equal(_np(c).astype(np.int32), ref)
    # edge weights only exist where there is an edge
    assert np.array_equal(_np(wh)[:, :-1], rwh[:, :-1])
    assert np.array_equal(_np(wv)[:-1, :], rwv[:-1, :])


# --- Dual MM -------------------------------------------------------------------

def _check_passes(dm, ctx, cost, wh, wv, iters, P):
    lam_v = np.zeros(cost.shape, dtype=np.int64)
    for it in range(iters):
        ctx.discrete_pass(0)
        lam_h_ref = O.dmm_pass(cost, wh, wv, 0, lam_v, P)
        lh, lv = ctx.duals()
        ctx.sync()
        assert np.array_equal(_np(lh).astype(np.int64), lam_h_ref), f"lambda_h, iteration {it}"
        ctx.discrete_pass(1)
        lam_v = O.dmm_pass(cost, wh, wv, 1, lam_h_ref, P)
        lh, lv = ctx.duals()
        ctx.sync()
        assert np.array_equal(_np(lv).astype(np.int64), lam_v), f"lambda_v, iteration {it}"


@pytest.mark.parametrize("H,W,L", SHAPES)
@pytest.mark.parametrize("path", [0, 1, 2, 3])  # lane groups pooled / int32 / one warp per chain / lane groups per chain
def test_dmm_passes_bit_exact(dm, H, W, L, path):
    left, right = _pair(H, W, L, seed=7 * H + W + L)
    ctx = _ctx(dm, H, W, L, dmm_path=path)
    ctx.cost_volume(left, right)
    cost = O.cost_volume(left, right, L)
    wh, wv = O.edge_weights(left)
    _check_passes(dm, ctx, cost, wh, wv, 3, O.Params())


@pytest.mark.parametrize("H,W,L", [(500, 16, 64), (16, 520, 48)])
def test_dmm_passes_with_more_chains_than_one_round(dm, H, W, L):
    """64 labels with 500 (then 520) chains in one pass: more chains than the
    GPU holds at three CTAs per SM, so the pass runs in two rounds."""
    left, right = _pair(H, W, L, seed=H + W)
    ctx = _ctx(dm, H, W, L)
    ctx.cost_volume(left, right)
    assert ctx.path()[0] == 8
    cost = O.cost_volume(left, right, L)
    wh, wv = O.edge_weights(left)
    _check_passes(dm, ctx, cost, wh, wv, 2, O.Params())


@pytest.mark.parametrize("H,W,L", [(9, 14, 16), (5, 40, 64), (12, 8, 128), (3, 5, 200)])
@pytest.mark.parametrize("path", [0, 1, 2, 3])
def test_dmm_passes_extreme_costs_and_weights(dm, H, W, L, path):
    # full uint8 cost range and every usable omega (multiples of 4 up to 252)
    rng = np.random.default_rng(H * W * L)
    cost = rng.integers(0, 256, size=(H, W, L)).astype(np.uint8)
    cost[0, 0, :] = 255
    cost[-1, -1, :] = 0
    wh = (4 * rng.integers(0, 64, size=(H, W))).astype(np.uint8)
    wv = (4 * rng.integers(0, 64, size=(H, W))).astype(np.uint8)
    wh[:, -1] = 0
    wv[-1, :] = 0
    ctx = _ctx(dm, H, W, L, dmm_path=path)
    ctx.set_cost_volume(cost, wh, wv)
    _check_passes(dm, ctx, cost.astype(np.int32), wh.astype(np.int32), wv.astype(np.int32), 2,
                  O.Params())


@pytest.mark.parametrize("params", [dict(), dict(C=1.0, eps=0.5), dict(w_hi=12, w_lo=0),
                                    dict(C=3.0, eps=0.25), dict(delta=2.0, eps=0.5, C=2.0)])
def test_dmm_other_penalties(dm, params):
    H, W, L = 10, 26, 24
    left, right = _pair(H, W, L, seed=5)
    ctx = _ctx(dm, H, W, L, **params)
    ctx.cost_volume(left, right)
    P = _oparams(ctx.params)
    cost = O.cost_volume(left, right, L)
    wh, wv = O.edge_weights(left, P)
    _check_passes(dm, ctx, cost, wh, wv, 2, P)


@pytest.mark.parametrize("H,W,L,iters", [(48, 64, 16, 5), (17, 31, 48, 4), (1, 50, 12, 2),
                                         (40, 1, 12, 2), (30, 70, 128, 3)])
@pytest.mark.parametrize("path", [0, 1, 2, 3])
def test_discrete_labels_and_bounds(dm, H, W, L, iters, path):
    left, right = _pair(H, W, L, seed=H + W)
    ctx = _ctx(dm, H, W, L, dmm_path=path)
    ctx.cost_volume(left, right)
    lb = ctx.discrete(iters, lower_bounds=True)
    labels = dm.labels_u16(ctx.labels())
    cost = O.cost_volume(left, right, L)
    wh, wv = O.edge_weights(left)
    rl, rlb, _, _ = O.dmm(cost, wh, wv, iters)
    assert np.array_equal(lb, rlb)
    assert np.array_equal(labels, rl)
    assert np.all(np.diff(lb) >= 0)
    assert lb[-1] <= O.discrete_energy(cost, wh, wv, labels)   # weak duality


@pytest.mark.parametrize("H,W,L", [(7, 9, 16), (5, 33, 64), (9, 6, 128)])
@pytest.mark.parametrize("path", [0, 1, 2, 3])
def test_all_equal_costs_break_ties_to_the_smallest_label(dm, H, W, L, path):
    cost = np.full((H, W, L), 7, dtype=np.uint8)
    wh = np.full((H, W), 8, dtype=np.uint8)
    wv = np.full((H, W), 4, dtype=np.uint8)
    wh[:, -1] = 0
    wv[-1, :] = 0
    ctx = _ctx(dm, H, W, L, dmm_path=path)
    ctx.set_cost_volume(cost, wh, wv)
    _check_passes(dm, ctx, cost.astype(np.int32), wh.astype(np.int32), wv.astype(np.int32), 2,
                  O.Params())
    ctx.reset_duals()
    lb = ctx.discrete(3, lower_bounds=True)
    labels = dm.labels_u16(ctx.labels())
    rl, rlb, _, _ = O.dmm(cost, wh, wv, 3)
    assert np.array_equal(labels, rl) and np.array_equal(lb, rlb)
    assert np.all(labels == 0)


def test_module_level_solve_and_batch_solve(dm):
    spec = S.SMALL
    sp = S.make_workload(spec, seed=6)
    u, labels, lb = dm.solve(sp.left, sp.right, spec["L"], spec["dmm_iters"], spec["pd_iters"])
    ref = O.solve(sp.left, sp.right, spec["L"], spec["dmm_iters"], spec["pd_iters"])
    assert np.array_equal(labels, ref["labels"]) and np.array_equal(lb, ref["lb"])
    assert np.abs(u.cpu().numpy().astype(np.float64) - ref["u"]).max() <= U_TOL
    pairs = [(sp.left, sp.right), (S.random_image(20, 30, 1), S.random_image(20, 30, 2))]
    out = dm.batch_solve(pairs, [16, 32], spec["dmm_iters"], spec["pd_iters"], tune=False)
    for (l, r), n, (bu, bl, blb) in zip(pairs, [16, 32], out):
        rr = O.solve(l, r, n, spec["dmm_iters"], spec["pd_iters"])
        assert np.array_equal(bl, rr["labels"]) and np.array_equal(blb, rr["lb"])
        assert np.abs(bu.cpu().numpy().astype(np.float64) - rr["u"]).max() <= U_TOL
    assert issubclass(dm.DMRefine(), __import__("torch").autograd.Function)


def test_invalid_edge_weight_is_reported(dm):
    H, W, L = 4, 6, 8
    cost = np.zeros((H, W, L), dtype=np.uint8)
    wh = np.full((H, W), 3, dtype=np.uint8)  # 3 * 1/4 is not an integer penalty
    wv = np.zeros((H, W), dtype=np.uint8)
    ctx = _ctx(dm, H, W, L)
    ctx.set_cost_volume(cost, wh, wv)
    with pytest.raises(dm.DMError) as e:
        ctx.discrete(1, lower_bounds=True)
    assert e.value.code == dm.DM_ERR_DEVICE


# --- continuous refinement ------------------------------------------------------

def _refine_case(dm, H, W, L, iters, u0, seed, **params):
    left, right = _pair(H, W, L, seed=seed)
    ctx = _ctx(dm, H, W, L, **params)
    ctx.cost_volume(left, right)
    ctx.refine(iters, u0=u0.astype(np.float32))
    u = _np(ctx.disparity()).astype(np.float64)
    e = ctx.energy()
    P = _oparams(ctx.params)
    cost = O.cost_volume(left, right, L).astype(np.float64)
    wh, wv = O.edge_weights(left, P)
    ru, _, ren = O.refine(cost, wh.astype(float), wv.astype(float),
                          u0.astype(np.float32).astype(np.float64), iters, P)
    re = O.cont_energy(cost, wh.astype(float), wv.astype(float), ru, P)
    assert np.abs(u - ru).max() <= U_TOL
    assert abs(e - re) <= E_TOL * abs(re)
    # the GPU energy of the oracle's own solution is the oracle's energy
    return u, ru


@pytest.mark.parametrize("H,W,L,iters", [(48, 64, 16, 50), (37, 53, 32, 100), (20, 31, 128, 60),
                                         (1, 40, 16, 30), (30, 1, 16, 30)])
def test_refine_from_labels(dm, H, W, L, iters):
    left, right = _pair(H, W, L, seed=11 + H)
    cost = O.cost_volume(left, right, L)
    u0 = np.argmin(cost, axis=2).astype(np.float64)  # a labelling the oracle computes itself
    _refine_case(dm, H, W, L, iters, u0, seed=11 + H)


@pytest.mark.parametrize("params", [dict(), dict(lambda_r=3.0), dict(alpha=0.5, warps=3),
                                    dict(C=50.0), dict(tau=0.2, sigma=0.5, h=0.5)])
def test_refine_fractional_start_and_params(dm, params):
    H, W, L = 24, 40, 32
    rng = np.random.default_rng(3)
    u0 = rng.uniform(0, L - 1, size=(H, W))
    _refine_case(dm, H, W, L, 40, u0, seed=3, **params)


# --- whole path -------------------------------------------------------------------

def test_solve_small_workload(dm):
    spec = S.SMALL
    sp = S.make_workload(spec, seed=0)
    H, W, L = spec["H"], spec["W"], spec["L"]
    ctx = _ctx(dm, H, W, L)
    u = _np(ctx.solve(sp.left, sp.right, spec["dmm_iters"], spec["pd_iters"])).astype(np.float64)
    labels = dm.labels_u16(ctx.labels())
    lb = ctx.lower_bounds(spec["dmm_iters"])
    e = ctx.energy()
    ref = O.solve(sp.left, sp.right, L, spec["dmm_iters"], spec["pd_iters"])
    assert np.array_equal(labels, ref["labels"])
    assert np.array_equal(lb, ref["lb"])
    assert np.abs(u - ref["u"]).max() <= U_TOL
    assert abs(e - ref["energy"][-1]) <= E_TOL * abs(ref["energy"][-1])


def test_solve_host_buffers(dm):
    import torch
    spec = S.SMALL
    sp = S.make_workload(spec, seed=4)
    H, W, L = spec["H"], spec["W"], spec["L"]
    ctx = _ctx(dm, H, W, L)
    left = torch.from_numpy(sp.left).pin_memory()
    right = torch.from_numpy(sp.right).pin_memory()
    u = torch.empty((H, W), dtype=torch.float32).pin_memory()
    lab = torch.empty((H, W), dtype=torch.int16).pin_memory()
    for _ in range(2):
        ctx.solve_host(left, right, spec["dmm_iters"], spec["pd_iters"], u, lab)
    ref = O.solve(sp.left, sp.right, L, spec["dmm_iters"], spec["pd_iters"])
    assert np.array_equal(lab.numpy().view(np.uint16), ref["labels"])
    assert np.abs(u.numpy().astype(np.float64) - ref["u"]).max() <= U_TOL
