"""The batched form: pairs of mixed sizes and label counts through persistent
Dual MM and primal-dual kernels, as one captured CUDA graph.

Small batches are checked against the oracle pair by pair (discrete stage
bit-exact, refined disparity within 1e-3 px); the 32-pair batch of the
batched workload against the single-pair path on the same GPU, which the
other tests tie to the oracle (the same kernels' arithmetic: identical results).
"""

import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_06274_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

U_TOL = 1e-3
SMALL = [(24, 32, 32), (40, 48, 64), (30, 70, 128), (17, 33, 32), (12, 20, 64), (8, 100, 128),
         (10, 30, 40), (1, 50, 32), (45, 1, 64)]


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_06274_gb300 import build, dm as _dm
    build.build()
    return _dm


def _pairs(shapes, seed):
    return [S.make_pair(H, W, L, planes=4, noise_sigma=2.0, seed=seed + k)
            for k, (H, W, L) in enumerate(shapes)]


def _check_against_oracle(dm, batch, pairs, shapes, outs, iters, pd):
    for k, ((H, W, L), sp) in enumerate(zip(shapes, pairs)):
        ref = O.solve(sp.left, sp.right, L, iters, pd)
        pv = batch.pairs[k]
        assert np.array_equal(dm.labels_u16(pv.labels()), ref["labels"]), f"pair {k}"
        assert np.array_equal(pv.lower_bounds(iters), ref["lb"]), f"pair {k}"
        u = outs[k].cpu().numpy().astype(np.float64)
        assert np.abs(u - ref["u"]).max() <= U_TOL, f"pair {k}"


def test_batch_matches_oracle(dm):
    pairs = _pairs(SMALL, 100)
    b = dm.Batch(SMALL)
    outs = b.solve([p.left for p in pairs], [p.right for p in pairs], 5, 50)
    b.sync()
    _check_against_oracle(dm, b, pairs, SMALL, outs, 5, 50)


def test_batch_after_work_still_queued_on_torch_stream(dm):
    """A batch created while work of a freed context is still queued on torch's
    stream: the caching allocator may hand the batch that context's memory, and
    the batch binds it on its own stream only after the queued work."""
    import torch
    sp = S.make_pair(375, 1242, 128, planes=4, seed=3)
    for _ in range(2):
        ctx = dm.Context(375, 1242, 128)
        ctx.solve(sp.left, sp.right, 10, 100)   # left running, not synchronised
        del ctx
        shapes = SMALL[:3]
        pairs = _pairs(shapes, 500)
        b = dm.Batch(shapes)
        outs = b.solve([p.left for p in pairs], [p.right for p in pairs], 3, 20)
        b.sync()
        _check_against_oracle(dm, b, pairs, shapes, outs, 3, 20)
        del b
    torch.cuda.synchronize()


def test_batch_discrete_pass_continues_every_pair(dm):
    """After a 3-iteration solve, one more horizontal pass over the batch gives
    every pair the oracle's next horizontal pass."""
    shapes = SMALL[:5]
    pairs = _pairs(shapes, 600)
    b = dm.Batch(shapes)
    b.solve([p.left for p in pairs], [p.right for p in pairs], 3, 0)
    b.discrete_pass(0)
    b.sync()
    for k, ((H, W, L), sp) in enumerate(zip(shapes, pairs)):
        cost = O.cost_volume(sp.left, sp.right, L)
        wh, wv = O.edge_weights(sp.left)
        _, _, _, lam_v = O.dmm(cost, wh, wv, 3)
        ref = O.dmm_pass(cost, wh, wv, 0, lam_v)
        lh, _ = b.pairs[k].duals()
        assert np.array_equal(lh.cpu().numpy().astype(np.int64), ref), k


def test_batch_with_256_labels(dm):
    """Pairs with 256 labels (the kernel class that runs two CTAs per SM) mixed
    with others, against the oracle."""
    shapes = [(8, 40, 256), (12, 30, 256), (10, 20, 128), (6, 50, 64)]
    pairs = _pairs(shapes, 700)
    b = dm.Batch(shapes)
    outs = b.solve([p.left for p in pairs], [p.right for p in pairs], 3, 20)
    b.sync()
    _check_against_oracle(dm, b, pairs, shapes, outs, 3, 20)


def test_batch_graph_replays_new_inputs(dm):
    import torch
    shapes = SMALL[:6]
    b = dm.Batch(shapes)
    lefts = [torch.zeros((H, W), dtype=torch.uint8, device="cuda") for H, W, _ in shapes]
    rights = [torch.zeros((H, W), dtype=torch.uint8, device="cuda") for H, W, _ in shapes]
    outs = b.outputs()
    b.capture(lefts, rights, 5, 50, outs)
    for seed in (200, 300):
        pairs = _pairs(shapes, seed)
        for k, sp in enumerate(pairs):
            lefts[k].copy_(torch.from_numpy(sp.left))
            rights[k].copy_(torch.from_numpy(sp.right))
        b.replay()
        b.sync()
        _check_against_oracle(dm, b, pairs, shapes, outs, 5, 50)


@pytest.mark.parametrize("choice", [(1, 32, 8, 4, 0), (3, 64, 4, 2, 1), (2, 16, 16, 8, 2),
                                    (2, 32, 16, 1, 96), (1, 64, 8, 64, 0)])
def test_every_launch_shape_gives_the_same_result(dm, choice):
    shapes = SMALL
    pairs = _pairs(shapes, 400)
    ref = dm.Batch(shapes)
    ref_out = ref.solve([p.left for p in pairs], [p.right for p in pairs], 4, 30)
    ref.sync()
    b = dm.Batch(shapes)
    b.set_tuning(choice)
    out = b.solve([p.left for p in pairs], [p.right for p in pairs], 4, 30)
    b.sync()
    for k in range(len(shapes)):
        assert np.array_equal(dm.labels_u16(b.pairs[k].labels()), dm.labels_u16(ref.pairs[k].labels()))
        assert np.array_equal(out[k].cpu().numpy(), ref_out[k].cpu().numpy())


def test_tuner_and_its_cache(dm, tmp_path):
    shapes = SMALL[:5]
    pairs = _pairs(shapes, 500)
    cache = str(tmp_path / "tune.txt")
    b = dm.Batch(shapes)
    choice = b.tune([p.left for p in pairs], [p.right for p in pairs], cache)
    assert b.tuning() == choice
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].split()[1:] == [str(v) for v in choice]
    b2 = dm.Batch(shapes)
    assert b2.tune([p.left for p in pairs], [p.right for p in pairs], cache) == choice
    assert len(open(cache).read().splitlines()) == 1   # read, not tuned again
    out = b2.solve([p.left for p in pairs], [p.right for p in pairs], 5, 50)
    b2.sync()
    _check_against_oracle(dm, b2, pairs, shapes, out, 5, 50)


def test_batch_of_32_mixed_pairs_matches_the_single_pair_path(dm):
    """the batched workload: 32 pairs of 320x240, 640x480 or 1242x375 with 32,
    64 or 128 labels, 5 Dual MM and 50 primal-dual iterations, one graph"""
    import torch
    specs = S.batch_specs(32, seed=0)
    shapes = [(s["H"], s["W"], s["L"]) for s in specs]
    pairs = [S.make_workload(s, seed=s["seed"]) for s in specs]
    b = dm.Batch(shapes)
    lefts = [torch.from_numpy(p.left).cuda() for p in pairs]
    rights = [torch.from_numpy(p.right).cuda() for p in pairs]
    outs = b.outputs()
    b.capture(lefts, rights, 5, 50, outs)
    b.replay()
    b.sync()
    for k, (s, sp) in enumerate(zip(specs, pairs)):
        ctx = dm.Context(s["H"], s["W"], s["L"])
        u = ctx.solve(sp.left, sp.right, 5, 50)
        lb = ctx.lower_bounds(5)
        assert np.array_equal(dm.labels_u16(b.pairs[k].labels()), dm.labels_u16(ctx.labels()))
        assert np.array_equal(b.pairs[k].lower_bounds(5), lb)
        assert np.array_equal(outs[k].cpu().numpy(), u.cpu().numpy())
