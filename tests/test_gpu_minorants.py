"""Dual MM with the naive and the iterative chain minorant (Sec. 2.3 "Good and
Fast Minorants"; Alg. iterative-minorant) on the GPU against the int64 oracle:
both duals after every pass, the labels and the lower bounds bit-exact, on
ragged shapes and label counts of every register class; sampled chains of the
1242x375x128 frame against the oracle's per-chain minorant.  Label counts that
are multiples of 16 run the staged kernel (inputs copied NS - 1 steps ahead
into shared memory), the others the kernel with one-step-ahead loads; the
shapes cover both.
"""

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


SHAPES = [(12, 20, 16), (1, 37, 8), (23, 1, 8), (9, 13, 33), (7, 19, 64), (5, 11, 100),
          (4, 9, 128), (3, 7, 256)]
KINDS = [("naive", 3, (1, 4)), ("iterative", 3, (1, 4)), ("iterative", 2, (1, 2)),
         ("iterative", 4, (3, 4)), ("iterative", 1, (1, 4))]


def _setup(dm, H, W, L, seed, kind, max_pass, gamma):
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=seed)
    ctx = dm.Context(H, W, L)
    ctx.cost_volume(sp.left, sp.right)
    ctx.set_minorant(kind, max_pass, gamma)
    cost = O.cost_volume(sp.left, sp.right, L)
    wh, wv = O.edge_weights(sp.left)
    return ctx, cost, wh, wv


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind,max_pass,gamma", KINDS)
def test_passes_bit_exact(dm, shape, kind, max_pass, gamma):
    H, W, L = shape
    ctx, cost, wh, wv = _setup(dm, H, W, L, H * 31 + W + L, kind, max_pass, gamma)
    assert ctx.path()[0] == 32
    lam_v = np.zeros(cost.shape, dtype=np.int64)
    for it in range(2):
        for which in (0, 1):
            ctx.discrete_pass(which)
            lam_in = lam_v if which == 0 else lam_h
            ref = O.dmm_pass(cost, wh, wv, which, lam_in, minorant=kind, max_pass=max_pass,
                             gamma=gamma)
            lh, lv = ctx.duals()
            got = (lh if which == 0 else lv).cpu().numpy().astype(np.int64)
            assert np.array_equal(got, ref), (it, which)
            if which == 0:
                lam_h = ref
            else:
                lam_v = ref


@pytest.mark.parametrize("shape", [(12, 20, 16), (9, 13, 33), (6, 17, 128)])
@pytest.mark.parametrize("kind", ["naive", "iterative"])
def test_labels_and_bounds_bit_exact(dm, shape, kind):
    H, W, L = shape
    ctx, cost, wh, wv = _setup(dm, H, W, L, W * 7 + L, kind, 3, (1, 4))
    lb = ctx.discrete(4, lower_bounds=True)
    rl, rlb, _, _ = O.dmm(cost, wh, wv, 4, minorant=kind)
    assert np.array_equal(dm.labels_u16(ctx.labels()), rl)
    assert np.array_equal(lb, rlb)


def test_switching_minorants(dm):
    """Switching resets the duals and the path; back to the hierarchical minorant
    the results are those of a context that never switched."""
    H, W, L = 16, 24, 32
    sp = S.make_pair(H, W, L, planes=3, seed=2)
    ref = dm.Context(H, W, L)
    ref.cost_volume(sp.left, sp.right)
    ref_lb = ref.discrete(3, lower_bounds=True)
    ctx = dm.Context(H, W, L)
    ctx.cost_volume(sp.left, sp.right)
    ctx.set_minorant("naive")
    naive_lb = ctx.discrete(3, lower_bounds=True)
    ctx.set_minorant("hier")
    assert ctx.path()[0] == 8
    lb = ctx.discrete(3, lower_bounds=True)
    assert np.array_equal(lb, ref_lb)
    assert np.array_equal(dm.labels_u16(ctx.labels()), dm.labels_u16(ref.labels()))
    # the naive minorant's bound is far below the hierarchical one's (Sec. 2.3)
    assert naive_lb[-1] < ref_lb[-1]


def test_set_minorant_rejects_bad_arguments(dm):
    ctx = dm.Context(4, 4, 8)
    for args in [("iterative", 0, (1, 4)), ("iterative", 3, (5, 4)), ("iterative", 3, (1, 0)),
                 ("iterative", 65, (1, 4))]:
        with pytest.raises(dm.DMError):
            ctx.set_minorant(*args)


@pytest.mark.parametrize("kind", ["naive", "iterative"])
def test_full_frame_sampled_chains(dm, kind):
    """1242x375x128, one iteration: sampled rows of lambda_h and columns of
    lambda_v against the oracle's minorant of those chains."""
    spec = S.KITTI
    H, W, L = spec["H"], spec["W"], spec["L"]
    pair = S.make_workload(spec, seed=0)
    ctx = dm.Context(H, W, L)
    ctx.cost_volume(pair.left, pair.right)
    ctx.set_minorant(kind)
    c, wh_t, wv_t = ctx.cost()
    cost = c.cpu().numpy().astype(np.int64)
    wh, wv = wh_t.cpu().numpy(), wv_t.cpu().numpy()
    ctx.discrete_pass(0)
    lh, _ = ctx.duals()
    lh = lh.cpu().numpy().astype(np.int64)
    fn = O.naive_minorant if kind == "naive" else O.iterative_minorant
    for y in (0, 1, 187, 374):
        V = np.stack([O.penalty_table(int(wh[y, x]), L) for x in range(W - 1)])
        assert np.array_equal(lh[y], fn(cost[y], V)), y      # lambda_v = 0: mu = lambda_h
    ctx.discrete_pass(1)
    _, lv = ctx.duals()
    lv = lv.cpu().numpy().astype(np.int64)
    for x in (0, 640, 1241):
        V = np.stack([O.penalty_table(int(wv[y, x]), L) for y in range(H - 1)])
        assert np.array_equal(lv[:, x] + lh[:, x], fn(lh[:, x], V)), x


@pytest.mark.parametrize("kind", ["naive", "iterative"])
@pytest.mark.parametrize("L", [40, 48, 128])
def test_uint16_cost_storage(dm, kind, L):
    """The alternatives read uint16 cost volumes too: the same numbers as uint8
    (L = 40 on the one-step-ahead kernel, 48 and 128 on the staged one)."""
    H, W = 11, 23
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=77)
    ctx = dm.Context(H, W, L, dm.default_params(cost_bytes=2))
    ctx.cost_volume(sp.left, sp.right)
    ctx.set_minorant(kind)
    lb = ctx.discrete(3, lower_bounds=True)
    cost = O.cost_volume(sp.left, sp.right, L)
    wh, wv = O.edge_weights(sp.left)
    rl, rlb, _, _ = O.dmm(cost, wh, wv, 3, minorant=kind)
    assert np.array_equal(dm.labels_u16(ctx.labels()), rl) and np.array_equal(lb, rlb)


@pytest.mark.parametrize("kind", ["naive", "iterative"])
@pytest.mark.parametrize("shape", [(6, 9, 2), (1, 12, 3), (12, 1, 3)])
def test_few_labels_and_single_rows(dm, kind, shape):
    H, W, L = shape
    ctx, cost, wh, wv = _setup(dm, H, W, L, H + W + L, kind, 3, (1, 4))
    lb = ctx.discrete(3, lower_bounds=True)
    rl, rlb, _, _ = O.dmm(cost, wh, wv, 3, minorant=kind)
    assert np.array_equal(dm.labels_u16(ctx.labels()), rl) and np.array_equal(lb, rlb)
