"""Optical flow on the GPU against the oracle (Sec. 2.2 "Flow"; the appendix's
quadratic data model): the decoupled cost volumes bit-exact, each layer's
Dual MM labels and bounds bit-exact, the two-component refinement within
1e-3 px of the FP64 oracle started from the same labels; at 640x480 with
64x64 displacements, sampled pixels of the cost volumes and accuracy against
the synthetic ground truth.
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


CASES = [(24, 40, -4, 8, -3, 6), (17, 33, -2, 5, -1, 3), (12, 50, -10, 33, -2, 4),
         (9, 70, -20, 64, 0, 2), (30, 20, -3, 7, -8, 16), (6, 40, -5, 256, -1, 3),
         (1, 30, -3, 6, 0, 2), (25, 1, 0, 2, -4, 9)]


def _pair(H, W, lo1, K1, lo2, K2, seed):
    return S.make_flow_pair(H, W, lo1, K1, lo2, K2, objects=2, noise_sigma=2.0, seed=seed)


@pytest.mark.parametrize("case", CASES)
def test_cost_volumes_bit_exact(dm, case):
    H, W, lo1, K1, lo2, K2 = case
    fp = _pair(*case, seed=H + W)
    f = dm.Flow(H, W, lo1, K1, lo2, K2)
    f.cost_volumes(fp.img1, fp.img2)
    fl = O.Flow(fp.img1, fp.img2, lo1, K1, lo2, K2)
    p1, p2 = fl.projected_costs()
    c1, wh1, wv1 = f.layer1.cost()
    c2, wh2, wv2 = f.layer2.cost()
    assert np.array_equal(c1.cpu().numpy().astype(np.int32), p1)
    assert np.array_equal(c2.cpu().numpy().astype(np.int32), p2)
    wh, wv = O.edge_weights(fp.img1)
    for a, b in ((wh1, wh), (wv1, wv), (wh2, wh), (wv2, wv)):
        assert np.array_equal(a.cpu().numpy().astype(np.int32), b)


@pytest.mark.parametrize("case", CASES[:5])
def test_layers_and_refinement_against_oracle(dm, case):
    H, W, lo1, K1, lo2, K2 = case
    fp = _pair(*case, seed=7 * H + W)
    f = dm.Flow(H, W, lo1, K1, lo2, K2)
    f.cost_volumes(fp.img1, fp.img2)
    lb1, lb2 = f.discrete(4, lower_bounds=True)
    d1, d2 = f.refine(40)
    f.sync()
    fl = O.Flow(fp.img1, fp.img2, lo1, K1, lo2, K2)
    p1, p2 = fl.projected_costs()
    wh, wv = O.edge_weights(fp.img1)
    r1, rb1, _, _ = O.dmm(p1, wh, wv, 4)
    r2, rb2, _, _ = O.dmm(p2, wh, wv, 4)
    g1, g2 = dm.labels_u16(f.layer1.labels()), dm.labels_u16(f.layer2.labels())
    assert np.array_equal(g1, r1) and np.array_equal(lb1, rb1)
    assert np.array_equal(g2, r2) and np.array_equal(lb2, rb2)
    u1, u2, _, _ = fl.refine(r1.astype(np.float64), r2.astype(np.float64), wh, wv, 40)
    assert np.abs(d1.cpu().numpy() - (lo1 + u1)).max() <= U_TOL
    assert np.abs(d2.cpu().numpy() - (lo2 + u2)).max() <= U_TOL


def test_refinement_without_labels_is_a_state_error(dm):
    f = dm.Flow(8, 12, -2, 5, -2, 5)
    fp = _pair(8, 12, -2, 5, -2, 5, seed=1)
    f.cost_volumes(fp.img1, fp.img2)
    with pytest.raises(dm.DMError):
        f.refine(10)


def test_full_size_flow(dm):
    """640x480, displacements in [-32, 32)^2: sampled pixels of both cost volumes
    against the oracle's data term; the refined flow stays within the boxes of
    the warps around the labels and matches most of the ground truth."""
    spec = S.FLOW
    fp = S.make_flow_workload(spec, seed=0)
    H, W = spec["H"], spec["W"]
    lo1, K1, lo2, K2 = spec["lo1"], spec["K1"], spec["lo2"], spec["K2"]
    f = dm.Flow(H, W, lo1, K1, lo2, K2)
    f.cost_volumes(fp.img1, fp.img2)
    c1 = f.layer1.cost()[0].cpu().numpy()
    c2 = f.layer2.cost()[0].cpu().numpy()
    fl = O.Flow(fp.img1, fp.img2, lo1, K1, lo2, K2)
    rng = np.random.default_rng(0)
    for y, x in [(0, 0), (H - 1, W - 1), (240, 320)] + [tuple(v) for v in
                                                        rng.integers(0, [H, W], size=(5, 2))]:
        D = np.array([[fl.D(y, x, a, b) for b in range(K2)] for a in range(K1)])
        assert np.array_equal(c1[y, x], D.min(axis=1)) and np.array_equal(c2[y, x], D.min(axis=0))
    f.discrete(spec["dmm_iters"])
    d1, d2 = f.refine(spec["pd_iters"])
    f.sync()
    d1, d2 = d1.cpu().numpy(), d2.cpu().numpy()
    l1 = lo1 + dm.labels_u16(f.layer1.labels()).astype(np.float64)
    l2 = lo2 + dm.labels_u16(f.layer2.labels()).astype(np.float64)
    warps = dm.default_params().warps
    assert np.all(np.isfinite(d1)) and np.all(np.isfinite(d2))
    assert np.abs(d1 - l1).max() <= warps + 1e-4 and np.abs(d2 - l2).max() <= warps + 1e-4
    inner = np.s_[40:H - 40, 40:W - 40]
    # six moving rectangles with displacements up to 32 px: occlusions and their
    # borders are wrong, most of the frame is right
    assert np.mean(np.abs(d1 - fp.gt1)[inner] < 1.0) > 0.7
    assert np.mean(np.abs(d2 - fp.gt2)[inner] < 1.0) > 0.7


@pytest.mark.parametrize("case", [(10, 14, -1, 2, 0, 2), (8, 12, -100, 4, 50, 3)])
def test_flow_minimal_and_out_of_image_ranges(dm, case):
    """Two displacements per component; and ranges that leave the image, where
    every cost is the out-of-image cost."""
    H, W, lo1, K1, lo2, K2 = case
    fp = S.make_flow_pair(H, W, max(lo1, -3), 2, 0, 2, objects=1, seed=3)
    f = dm.Flow(H, W, lo1, K1, lo2, K2)
    f.cost_volumes(fp.img1, fp.img2)
    lb1, lb2 = f.discrete(2, lower_bounds=True)
    d1, d2 = f.refine(10)
    f.sync()
    fl = O.Flow(fp.img1, fp.img2, lo1, K1, lo2, K2)
    p1, p2 = fl.projected_costs()
    assert np.array_equal(f.layer1.cost()[0].cpu().numpy().astype(np.int32), p1)
    assert np.array_equal(f.layer2.cost()[0].cpu().numpy().astype(np.int32), p2)
    wh, wv = O.edge_weights(fp.img1)
    r1, rb1, _, _ = O.dmm(p1, wh, wv, 2)
    r2, rb2, _, _ = O.dmm(p2, wh, wv, 2)
    assert np.array_equal(lb1, rb1) and np.array_equal(lb2, rb2)
    u1, u2, _, _ = fl.refine(r1.astype(np.float64), r2.astype(np.float64), wh, wv, 10)
    assert np.abs(d1.cpu().numpy() - (lo1 + u1)).max() <= U_TOL
    assert np.abs(d2.cpu().numpy() - (lo2 + u2)).max() <= U_TOL
