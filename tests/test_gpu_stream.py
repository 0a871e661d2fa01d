"""uint16 cost volumes and the warm-started sequence (the streaming form).

Discrete stage bit-exact against the oracle (which takes any integer costs and
a starting lambda_v), continuous stage within 1e-3 px; the 1920x1080x256
workload is checked on sampled cost rows and on invariants that hold at any
size.
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


def _ctx(dm, H, W, L, **params):
    return dm.Context(H, W, L, dm.default_params(cost_bytes=2, **params))


def _np(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("H,W,L", [(48, 64, 16), (13, 29, 2), (9, 21, 33), (5, 11, 128),
                                   (3, 7, 256), (6, 40, 64)])
def test_u16_cost_volume_bit_exact(dm, H, W, L):
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=H + W + L)
    ctx = _ctx(dm, H, W, L)
    ctx.cost_volume(sp.left, sp.right)
    c, wh, wv = ctx.cost()
    assert c.dtype.itemsize == 2
    assert np.array_equal(_np(c).view(np.uint16).astype(np.int32),
                          O.cost_volume(sp.left, sp.right, L))


def _check_passes(ctx, cost, wh, wv, iters, P=O.Params()):
    lam_v = np.zeros(cost.shape, dtype=np.int64)
    for it in range(iters):
        ctx.discrete_pass(0)
        lam_h = O.dmm_pass(cost, wh, wv, 0, lam_v, P)
        lh, _ = ctx.duals()
        assert np.array_equal(_np(lh).astype(np.int64), lam_h), f"lambda_h, iteration {it}"
        ctx.discrete_pass(1)
        lam_v = O.dmm_pass(cost, wh, wv, 1, lam_h, P)
        _, lv = ctx.duals()
        assert np.array_equal(_np(lv).astype(np.int64), lam_v), f"lambda_v, iteration {it}"


@pytest.mark.parametrize("H,W,L", [(48, 64, 16), (17, 31, 48), (7, 19, 64), (5, 11, 128),
                                   (4, 9, 256)])
@pytest.mark.parametrize("path", [0, 1, 2])
def test_u16_census_passes_bit_exact(dm, H, W, L, path):
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=3 * H + W)
    ctx = _ctx(dm, H, W, L, dmm_path=path)
    ctx.cost_volume(sp.left, sp.right)
    cost = O.cost_volume(sp.left, sp.right, L)
    wh, wv = O.edge_weights(sp.left)
    _check_passes(ctx, cost, wh, wv, 2)


@pytest.mark.parametrize("cost_max", [200, 2000, 60000])
@pytest.mark.parametrize("H,W,L", [(9, 14, 16), (6, 30, 64), (12, 8, 128)])
def test_u16_caller_volume_bit_exact(dm, H, W, L, cost_max):
    # 200 and 2000: the packed 16-bit kernel (uint8 / int16 deltas); 60000: int32
    rng = np.random.default_rng(H * W + cost_max)
    cost = rng.integers(0, cost_max + 1, size=(H, W, L)).astype(np.uint16)
    cost[0, 0, :] = cost_max
    wh = np.where(rng.random((H, W)) < 0.5, 8, 4).astype(np.uint8)
    wv = np.where(rng.random((H, W)) < 0.5, 8, 4).astype(np.uint8)
    ctx = _ctx(dm, H, W, L)
    ctx.set_cost_volume_u16(cost, wh, wv, cost_max)
    _check_passes(ctx, cost.astype(np.int32), wh.astype(np.int32), wv.astype(np.int32), 2)


def test_u16_caller_volume_out_of_range_is_refused(dm):
    H, W, L = 4, 20000, 16   # (65535 + 4 * 16) * 20001 >= 2^30
    ctx = _ctx(dm, H, W, L)
    cost = np.zeros((H, W, L), dtype=np.uint16)
    z = np.zeros((H, W), dtype=np.uint8)
    with pytest.raises(dm.DMError) as e:
        ctx.set_cost_volume_u16(cost, z + 4, z + 4, 65535)
    assert e.value.code == dm.DM_ERR_RANGE


def test_u16_refine_matches_oracle(dm):
    H, W, L, iters = 30, 50, 64, 60
    sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=21)
    ctx = _ctx(dm, H, W, L)
    ctx.cost_volume(sp.left, sp.right)
    ctx.discrete(4)
    labels = dm.labels_u16(ctx.labels())
    ctx.refine(iters)
    u = _np(ctx.disparity()).astype(np.float64)
    cost = O.cost_volume(sp.left, sp.right, L)
    wh, wv = O.edge_weights(sp.left)
    rl, _, _, _ = O.dmm(cost, wh, wv, 4)
    assert np.array_equal(labels, rl)
    ru, _, _ = O.refine(cost.astype(float), wh.astype(float), wv.astype(float),
                        rl.astype(float), iters)
    assert np.abs(u - ru).max() <= U_TOL


@pytest.mark.parametrize("H,W,L", [(48, 64, 16), (30, 70, 64)])
@pytest.mark.parametrize("cost_bytes", [1, 2])
@pytest.mark.parametrize("path", [0, 1, 2])
def test_warm_started_sequence_matches_oracle(dm, H, W, L, cost_bytes, path):
    """frame 0 cold, then each frame starts Dual MM from the previous lambda_v"""
    iters, pd = 3, 20
    frames = list(S.make_sequence(H, W, L, 4, planes=4, noise_sigma=2.0, drift=0.5, seed=H))
    ctx = dm.Context(H, W, L, dm.default_params(cost_bytes=cost_bytes, dmm_path=path))
    lam_v = None
    for f, sp in enumerate(frames):
        if f == 0:
            u = ctx.solve(sp.left, sp.right, iters, pd)
        else:
            u = ctx.solve_next(sp.left, sp.right, iters, pd)
        lb = ctx.lower_bounds(iters)
        labels = dm.labels_u16(ctx.labels())
        cost = O.cost_volume(sp.left, sp.right, L)
        wh, wv = O.edge_weights(sp.left)
        rl, rlb, _, lam_v = O.dmm(cost, wh, wv, iters, lam_v0=lam_v)
        assert np.array_equal(lb, rlb), f"frame {f}"
        assert np.array_equal(labels, rl), f"frame {f}"
        ru, _, _ = O.refine(cost.astype(float), wh.astype(float), wv.astype(float),
                            rl.astype(float), pd)
        assert np.abs(_np(u).astype(np.float64) - ru).max() <= U_TOL
        # the bound is a bound for the new frame
        assert lb[-1] <= O.discrete_energy(cost, wh, wv, labels)


def test_warm_start_after_float_cost_is_a_cold_start(dm):
    H, W, L = 12, 20, 16
    frames = list(S.make_sequence(H, W, L, 2, planes=3, seed=5))
    ctx = dm.Context(H, W, L)
    ctx.cost_volume(frames[0].left, frames[0].right)
    ctx.set_cost_volume_f32(np.zeros((H, W, L), np.float32))
    ctx.cost_volume_warm(frames[1].left, frames[1].right)
    lb = ctx.discrete(2, lower_bounds=True)
    cost = O.cost_volume(frames[1].left, frames[1].right, L)
    wh, wv = O.edge_weights(frames[1].left)
    _, rlb, _, _ = O.dmm(cost, wh, wv, 2)
    assert np.array_equal(lb, rlb)


def test_stream_1920x1080x256_invariants(dm):
    """three frames of the streaming workload: sampled cost rows against the
    oracle, monotone bounds within a frame, the refined disparity inside the
    warps' boxes and the label range"""
    spec = S.STREAM
    H, W, L = spec["H"], spec["W"], spec["L"]
    ctx = _ctx(dm, H, W, L)
    frames = S.make_sequence(H, W, L, 3, planes=spec["planes"], noise_sigma=spec["noise_sigma"],
                             drift=spec["drift"], seed=0)
    for f, sp in enumerate(frames):
        solve = ctx.solve if f == 0 else ctx.solve_next
        u = _np(solve(sp.left, sp.right, spec["dmm_iters"], spec["pd_iters"])).astype(np.float64)
        lb = ctx.lower_bounds(spec["dmm_iters"])
        assert np.all(np.diff(lb) >= 0), f"frame {f}"
        labels = dm.labels_u16(ctx.labels()).astype(np.float64)
        assert np.all(u >= 0) and np.all(u <= L - 1)
        assert np.all(np.abs(u - labels) <= 5.0 + 1e-4)
        c, _, _ = ctx.cost()
        rows = slice(500, 504)
        crop = O.cost_volume(sp.left[498:506], sp.right[498:506], L)[2:6]
        assert np.array_equal(_np(c[rows]).view(np.uint16).astype(np.int32), crop)


@pytest.mark.parametrize("warm", [False, True])
def test_stream_1920x1080x256_sampled_chains_bit_exact(dm, warm):
    """One Dual MM iteration on the streaming frame (1920 x 1080, 256 labels,
    uint16 costs) cold (frame 0) and warm-started (frame 1 from frame 0's
    lambda_v): rows 0, 1, 540, 1079 of the horizontal pass and columns 0, 960,
    1919 of the vertical pass against the oracle's hierarchical minorant of
    those chains (App. A), bit for bit."""
    spec = S.STREAM
    H, W, L = spec["H"], spec["W"], spec["L"]
    ctx = _ctx(dm, H, W, L)
    frames = list(S.make_sequence(H, W, L, 2, planes=spec["planes"],
                                  noise_sigma=spec["noise_sigma"], drift=spec["drift"], seed=0))
    if warm:
        ctx.solve(frames[0].left, frames[0].right, spec["dmm_iters"], spec["pd_iters"])
        ctx.cost_volume_warm(frames[1].left, frames[1].right)
    else:
        ctx.cost_volume(frames[0].left, frames[0].right)
    assert ctx.path()[0] == 8
    c, wh_t, wv_t = ctx.cost()
    wh, wv = _np(wh_t), _np(wv_t)
    rows, cols = (0, 1, 540, 1079), (0, 960, 1919)
    _, lv = ctx.duals()
    lv_in = {y: _np(lv[y]).astype(np.int64) for y in rows}   # zero for the cold frame
    c_rows = {y: _np(c[y]).view(np.uint16).astype(np.int64) for y in rows}
    ctx.discrete_pass(0)
    lh, _ = ctx.duals()
    for y in rows:
        V = np.stack([O.penalty_table(int(wh[y, x]), L) for x in range(W - 1)])
        mu = O.hier_minorant(c_rows[y] + lv_in[y], V)
        assert np.array_equal(_np(lh[y]).astype(np.int64) + lv_in[y], mu), f"row {y}"
    lh_cols = {x: _np(lh[:, x]).astype(np.int64) for x in cols}
    ctx.discrete_pass(1)
    _, lv = ctx.duals()
    for x in cols:
        V = np.stack([O.penalty_table(int(wv[y, x]), L) for y in range(H - 1)])
        nu = O.hier_minorant(lh_cols[x], V)
        assert np.array_equal(_np(lv[:, x]).astype(np.int64) + lh_cols[x], nu), f"column {x}"
    if not warm:
        assert not any(np.any(v) for v in lv_in.values())
