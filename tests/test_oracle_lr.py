"""Pins of the oracle's two-sided consistency check (Sec. 4.1.1) and of its
right-view problem, against brute force, scene geometry and the mirror
symmetry of the census cost.

The right view's cost is written from its definition (the right image as
reference, label l matching the left image's pixel x + l); the two-view path
instead solves the mirrored pair.  The first pins tie the two together; the
check itself is pinned on disparity fields whose consistent and occluded
pixels follow from the geometry of the scene, not from the check's formula.
"""

import numpy as np
import pytest

import bruteforce as B
from oracle import oracle as O
from paper_1601_06274_gb300 import synthetic as S


# --- right view's cost -----------------------------------------------------------

@pytest.mark.parametrize("win", [3, 5])
def test_right_cost_bruteforce(win):
    rng = np.random.default_rng(11)
    left = rng.integers(0, 256, size=(6, 13), dtype=np.uint8)
    right = rng.integers(0, 256, size=(6, 13), dtype=np.uint8)
    right[3, 2:7] = 90  # ties in the census comparisons
    L = 7
    cost = O.cost_volume_right(left, right, L, win)
    cl, cr = B.census_ref(left, win), B.census_ref(right, win)
    for y in range(6):
        for x in range(13):
            for l in range(L):
                # the right pixel x sees the scene point that the left image has at x + l
                ref = B.hamming(cr[y, x], cl[y, x + l]) if x + l < 13 else win * win - 1
                assert cost[y, x, l] == ref


@pytest.mark.parametrize("shape", [(5, 17, 8), (9, 31, 16), (1, 12, 12)])
def test_mirrored_pair_is_the_right_view(shape):
    """The mirrored pair's left-reference cost is the right-view cost with its
    columns reversed, bit for bit (census bits of a mirrored window are the
    same permutation on both sides; clamp-to-edge is mirror symmetric)."""
    H, W, L = shape
    sp = S.make_pair(H, W, L, planes=2, seed=H * W)
    direct = O.cost_volume_right(sp.left, sp.right, L)
    mirrored = O.cost_volume(np.ascontiguousarray(sp.right[:, ::-1]),
                             np.ascontiguousarray(sp.left[:, ::-1]), L)
    assert np.array_equal(mirrored[:, ::-1, :], direct)
    # the edge weights of the mirrored reference are those of the right image,
    # with the horizontal edge (x, x+1) of the mirror at (W-2-x, W-1-x)
    whm, wvm = O.edge_weights(np.ascontiguousarray(sp.right[:, ::-1]))
    whr, wvr = O.edge_weights(sp.right)
    assert np.array_equal(wvm, wvr[:, ::-1])
    assert np.array_equal(whm[:, :W - 1], whr[:, W - 2::-1])
    assert np.all(whm[:, W - 1] == 0)


def test_two_view_path_on_a_fronto_parallel_scene():
    """A textured plane at integer disparity 3, no noise: both views find it,
    and every pixel whose counterpart is visible passes the check."""
    rng = np.random.default_rng(5)
    H, W, L, d0 = 10, 48, 8, 3
    scene = rng.integers(0, 256, size=(H, W + d0), dtype=np.uint8)
    left = np.ascontiguousarray(scene[:, :W])       # left pixel x shows scene column x
    right = np.ascontiguousarray(scene[:, d0:])     # right pixel x - d0 shows it too
    r = O.solve_lr(left, right, L, 4, 20)
    inner = np.s_[:, d0 + 2:W - 2]
    assert np.abs(r["u_left"][inner] - d0).max() < 0.05
    assert np.abs(r["u_right"][:, 2:W - d0 - 2] - d0).max() < 0.05
    assert r["ok"][inner].all()
    assert np.array_equal(r["u"][inner], r["u_left"][inner])
    # pixels with no counterpart in the image (x - d < 0) fail
    assert not r["ok"][:, 0].any() and (r["u"][:, 0] == -1).all()


# --- the check -------------------------------------------------------------------

def test_check_constant_disparity():
    H, W, d0 = 3, 20, 4
    ul = np.full((H, W), d0, np.float32)
    ur = np.full((H, W), d0, np.float32)
    ok, out = O.lr_check(ul, ur)
    x = np.arange(W)
    assert np.array_equal(ok, np.broadcast_to((x >= d0).astype(np.uint8), (H, W)))
    assert np.array_equal(out[ok == 1], ul[ok == 1]) and np.all(out[ok == 0] == -1)


def test_check_two_planes_with_occlusion():
    """Background at disparity 2, a foreground strip at disparity 6 over left
    columns [10, 16).  Drawn from the scene: the right view sees the strip over
    columns [4, 10) and the background elsewhere, so the background that the
    left view shows at columns [6, 10) is hidden in the right view, and the
    left columns 0, 1 have no counterpart in the image."""
    W = 30
    xs = np.arange(W)
    ul = np.where((xs >= 10) & (xs < 16), 6.0, 2.0).astype(np.float32)[None, :]
    ur = np.where((xs >= 4) & (xs < 10), 6.0, 2.0).astype(np.float32)[None, :]
    ok, out = O.lr_check(ul, ur, 1.0)
    expect = np.ones(W, np.uint8)
    expect[0:2] = 0
    expect[6:10] = 0
    assert np.array_equal(ok[0], expect)


def test_check_rounds_half_to_even():
    """The counterpart of d = 2.5 at x = 5 is column 3 (rint 2.5 = 2) and that of
    d = 3.5 at x = 9 is column 5 (rint 3.5 = 4): only those columns agree."""
    ul = np.zeros((1, 12), np.float32)
    ur = np.full((1, 12), 50.0, np.float32)
    ul[0, 5], ur[0, 3] = 2.5, 2.5
    ul[0, 9], ur[0, 5] = 3.5, 3.5
    ok, _ = O.lr_check(ul, ur, 0.25)
    assert ok[0, 5] == 1 and ok[0, 9] == 1
    # the neighbouring columns that other roundings would pick disagree
    ur2 = ur.copy()
    ur2[0, 3] = ur2[0, 5] = 50.0
    ur2[0, 2] = 2.5
    ur2[0, 6] = 3.5
    ok2, _ = O.lr_check(ul, ur2, 0.25)
    assert ok2[0, 5] == 0 and ok2[0, 9] == 0


def test_check_threshold_is_inclusive_and_symmetric():
    # d = 2 at x = 4..7: the counterparts are the columns x - 2
    ul = np.full((1, 8), 0.0, np.float32)
    ur = np.full((1, 8), 0.0, np.float32)
    ul[0, 4] = 2.0; ur[0, 2] = 3.0       # difference exactly 1: passes
    ul[0, 5] = 2.0; ur[0, 3] = 1.0       # -1: passes
    ul[0, 6] = 2.0; ur[0, 4] = 3.0625    # just above: fails
    ul[0, 7] = 2.0; ur[0, 5] = 0.9375    # just below -1: fails
    ok, out = O.lr_check(ul, ur, 1.0)
    assert ok[0, 4:].tolist() == [1, 1, 0, 0]
    assert out[0, 4:].tolist() == [2.0, 2.0, -1.0, -1.0]


def test_check_borders_and_non_finite():
    ul = np.array([[0.0, 2.0, -1.0, np.nan, np.inf, 0.0]], np.float32)
    ur = np.zeros((1, 6), np.float32)
    ul[0, 2] = -1.0     # x=2, d=-1: counterpart column 3, inside: |-1 - 0| <= 1 passes
    ul[0, 5] = -1.0     # x=5, d=-1: counterpart column 6 = W: outside, fails
    ok, out = O.lr_check(ul, ur, 1.0)
    assert ok[0].tolist() == [1, 0, 1, 0, 0, 0]   # x=1, d=2: column -1, outside
    assert out[0, 3] == -1 and out[0, 4] == -1


def test_check_rejects_bad_arguments():
    with pytest.raises(RuntimeError):
        O.lr_check(np.zeros((2, 2), np.float32), np.zeros((2, 2), np.float32), -1.0)
