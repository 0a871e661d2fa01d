"""Pins of the oracle's optical-flow path (Sec. 2.2 "Flow": decoupled layers
with min-projected costs; the appendix's quadratic data model and its prox).

* Decoupled costs and the data term D against brute force over census codes.
* The quadratic fit is exact on quadratics; the PSD part equals the
  eigenvalue clamp of numpy.linalg.eigh.
* The prox satisfies its optimality condition inside the box, and equals a
  brute-force minimisation when Q is diagonal.
* Without the regulariser the refinement reaches each pixel's Newton point
  u0 - Q^-1 L; transposing both images swaps the two components; a pure
  translation is recovered with its signs.
"""

import numpy as np
import pytest

import bruteforce as B
from oracle import oracle as O


def _imgs(H, W, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 256, size=(H, W), dtype=np.uint8),
            rng.integers(0, 256, size=(H, W), dtype=np.uint8))


def _D_brute(c1, c2, y, x, d1, d2, maxc=24):
    H, W = c1.shape
    yy, xx = y + d2, x + d1
    if not (0 <= yy < H and 0 <= xx < W):
        return maxc
    return B.hamming(c1[y, x], c2[yy, xx])


@pytest.mark.parametrize("lo1,K1,lo2,K2", [(-2, 5, -1, 3), (0, 4, 0, 1), (-3, 2, 1, 4)])
def test_projected_costs_bruteforce(lo1, K1, lo2, K2):
    a, b = _imgs(7, 9, K1 * 10 + K2)
    fl = O.Flow(a, b, lo1, K1, lo2, K2)
    p1, p2 = fl.projected_costs()
    c1, c2 = B.census_ref(a, 5), B.census_ref(b, 5)
    for y in range(7):
        for x in range(9):
            D = np.array([[_D_brute(c1, c2, y, x, lo1 + i, lo2 + j) for j in range(K2)]
                          for i in range(K1)])
            assert np.array_equal(p1[y, x], D.min(axis=1))
            assert np.array_equal(p2[y, x], D.min(axis=0))


def test_data_term_is_bilinear_in_the_labels():
    a, b = _imgs(8, 10, 3)
    fl = O.Flow(a, b, -2, 5, -1, 4)
    c1, c2 = B.census_ref(a, 5), B.census_ref(b, 5)
    y, x = 4, 5
    Dint = lambda i, j: _D_brute(c1, c2, y, x, -2 + i, -1 + j)
    for i in range(5):
        for j in range(4):
            assert fl.D(y, x, i, j) == Dint(i, j)
    t, s = 0.3, 0.75
    ref = ((1 - t) * (1 - s) * Dint(1, 2) + t * (1 - s) * Dint(2, 2) + (1 - t) * s * Dint(1, 3)
           + t * s * Dint(2, 3))
    assert abs(fl.D(y, x, 1 + t, 2 + s) - ref) < 1e-12
    # arguments are clamped to the label ranges
    assert fl.D(y, x, -3.0, 9.0) == Dint(0, 3)
    assert fl.D(y, x, 4.0, 3.0) == Dint(4, 3)


@pytest.mark.parametrize("h", [1.0, 0.5])
def test_fit_is_exact_on_quadratics(h):
    rng = np.random.default_rng(int(h * 10))
    for _ in range(10):
        g = rng.normal(size=2)
        M = rng.normal(size=(2, 2))
        A = M + M.T
        c = rng.normal()
        f = lambda v: c + g @ v + 0.5 * v @ A @ v
        S = np.array([[f(np.array([(i - 1) * h, (j - 1) * h])) for i in range(3)]
                      for j in range(3)])
        L, Q = O.flow_fit_samples(S, h)
        assert np.allclose(L, g, atol=1e-12)
        assert np.allclose(Q, [A[0, 0], A[0, 1], A[1, 1]], atol=1e-12)


def test_psd_part_is_the_eigenvalue_clamp():
    rng = np.random.default_rng(5)
    cases = [rng.normal(size=3) * 3 for _ in range(40)]
    cases += [np.array([2.0, 0.0, -1.0]), np.array([-1.0, 0.0, 3.0]), np.array([-1, 0.0, -2]),
              np.array([1.0, 1.0, 1.0]), np.array([0.0, 0.0, 0.0])]
    for q in cases:
        A = np.array([[q[0], q[1]], [q[1], q[2]]])
        w, V = np.linalg.eigh(A)
        ref = V @ np.diag(np.maximum(w, 0)) @ V.T
        got = O.psd2(q)
        assert np.allclose([ref[0, 0], ref[0, 1], ref[1, 1]], got, atol=1e-12), q
        assert np.allclose(O.psd2(got), got, atol=1e-12)   # idempotent


def test_prox_optimality_inside_the_box():
    rng = np.random.default_rng(7)
    for _ in range(20):
        M = rng.normal(size=(2, 2))
        Qm = M @ M.T
        Q = np.array([Qm[0, 0], Qm[0, 1], Qm[1, 1]])
        L = rng.normal(size=2)
        u0 = rng.uniform(5, 10, size=2)
        uh = u0 + rng.normal(scale=0.2, size=2)
        box = np.array([u0[0] - 100, u0[0] + 100, u0[1] - 100, u0[1] + 100])
        tau = 0.35
        u = O.flow_prox(uh, u0, L, Q, box, tau)
        grad = (u - uh) / tau + L + Qm @ (u - u0)
        assert np.allclose(grad, 0, atol=1e-10)


def test_prox_with_diagonal_q_is_the_box_constrained_minimiser():
    rng = np.random.default_rng(9)
    for _ in range(10):
        Q = np.array([rng.uniform(0, 3), 0.0, rng.uniform(0, 3)])
        L = rng.normal(scale=3, size=2)
        u0 = np.array([4.0, 6.0])
        uh = u0 + rng.normal(scale=1.0, size=2)
        box = np.array([3.0, 5.0, 5.0, 7.0])
        tau = 0.35
        u = O.flow_prox(uh, u0, L, Q, box, tau)
        g1 = np.linspace(box[0], box[1], 2001)
        g2 = np.linspace(box[2], box[3], 2001)
        obj = lambda v, k: (0.5 * (v - uh[k]) ** 2 / tau + L[k] * (v - u0[k])
                            + 0.5 * Q[2 * k] * (v - u0[k]) ** 2)
        ref = np.array([g1[np.argmin(obj(g1, 0))], g2[np.argmin(obj(g2, 1))]])
        assert np.allclose(u, ref, atol=2e-3)


def test_refine_without_regulariser_reaches_the_newton_point():
    a, b = _imgs(6, 8, 11)
    fl = O.Flow(a, b, -3, 7, -3, 7)
    P = O.Params(lambda_r=0.0, warps=1)
    rng = np.random.default_rng(2)
    u1 = rng.integers(2, 5, size=(6, 8)).astype(np.float64)
    u2 = rng.integers(2, 5, size=(6, 8)).astype(np.float64)
    wh, wv = O.edge_weights(a)
    r1, r2, D, _ = fl.refine(u1, u2, wh, wv, 3000, P)
    assert np.all(D == 0)
    checked = 0
    for y in range(6):
        for x in range(8):
            L, Q, box = fl.linearise_px(y, x, u1[y, x], u2[y, x])
            Qm = np.array([[Q[0], Q[1]], [Q[1], Q[2]]])
            if np.linalg.eigvalsh(Qm).min() < 0.5:
                continue
            newton = np.array([u1[y, x], u2[y, x]]) - np.linalg.solve(Qm, L)
            if not (box[0] < newton[0] < box[1] and box[2] < newton[1] < box[3]):
                continue
            assert np.allclose([r1[y, x], r2[y, x]], newton, atol=1e-6)
            checked += 1
    assert checked >= 3


def test_transposed_images_swap_the_components():
    a, b = _imgs(7, 9, 13)
    rng = np.random.default_rng(4)
    u1 = rng.integers(0, 5, size=(7, 9)).astype(np.float64)
    u2 = rng.integers(0, 4, size=(7, 9)).astype(np.float64)
    fl = O.Flow(a, b, -2, 5, -1, 4)
    wh, wv = O.edge_weights(a)
    r1, r2, _, en = fl.refine(u1, u2, wh, wv, 40)
    at, bt = a.T.copy(), b.T.copy()
    ft = O.Flow(at, bt, -1, 4, -2, 5)
    wht, wvt = O.edge_weights(at)
    assert np.array_equal(wht, wv.T) and np.array_equal(wvt, wh.T)
    t1, t2, _, ent = ft.refine(u2.T, u1.T, wht, wvt, 40)
    assert np.allclose(t1, r2.T, atol=1e-9) and np.allclose(t2, r1.T, atol=1e-9)
    assert np.allclose(en, ent, rtol=1e-12)
    p1, p2 = fl.projected_costs()
    q1, q2 = ft.projected_costs()
    assert np.array_equal(q1, p2.transpose(1, 0, 2)) and np.array_equal(q2, p1.transpose(1, 0, 2))


def test_translation_is_recovered():
    """I2 is I1 moved by (+3, -2): the labels of both layers find it."""
    rng = np.random.default_rng(21)
    scene = rng.integers(0, 256, size=(40, 60), dtype=np.uint8)
    H, W, u, v = 16, 24, 3, -2
    Y0, X0 = 10, 10
    img1 = scene[Y0:Y0 + H, X0:X0 + W].copy()
    img2 = scene[Y0 - v:Y0 - v + H, X0 - u:X0 - u + W].copy()   # I2(y + v, x + u) = I1(y, x)
    r = O.solve_flow(img1, img2, -4, 8, -4, 8, 3, 20)
    # pixels whose census windows, here and at the displaced position, are interior
    inner = np.s_[5:H - 3, 3:W - 6]
    l1, l2 = r["labels1"].astype(np.int64) - 4, r["labels2"].astype(np.int64) - 4
    assert np.all(l1[inner] == u) and np.all(l2[inner] == v)
    # the refinement follows the quadratic model of the V-shaped census cost: it
    # stays within the linearisation box (h = 1) and mostly at the true flow
    for got, true in ((r["u1"], u + 4), (r["u2"], v + 4)):
        err = np.abs(got[inner] - true)
        assert err.max() < 1.0 and np.median(err) < 0.1
