"""Pins of the oracle's continuous stage (Sec. 2.4, 3.1) against the mathematics.

Proximal maps and conjugates are checked against numeric minimisation and
numeric suprema of their definitions; the whole primal-dual iteration is
checked on the convex special case (C -> infinity) where the primal-dual gap
must close, and on zero pairwise weights where it must reach the per-pixel
minimiser; the continuous energy at integer labels must equal the discrete
energy (Sec. 2.4: the same energy in both stages).
"""

import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_06274_gb300 import synthetic as S


def _grid_argmin(f, lo, hi, n=200001):
    xs = np.linspace(lo, hi, n)
    v = f(xs)
    k = int(np.argmin(v))
    return xs[k], (hi - lo) / (n - 1)


def test_interpolation():
    c = np.array([3.0, 7.0, 1.0, 1.0, 9.0])
    for k in range(5):
        assert O.interp(c, k) == c[k]
    assert O.interp(c, 0.25) == pytest.approx(4.0)
    assert O.interp(c, 1.5) == pytest.approx(4.0)
    assert O.interp(c, -2.0) == 3.0 and O.interp(c, 7.5) == 9.0


def test_linearisation_slopes_and_box():
    c = np.array([5.0, 2.0, 4.0, 10.0, 11.0, 0.0])
    # at u0 = 2: s1 = D(2) - D(1) = 2, s2 = D(3) - D(2) = 6
    assert O.linearise_px(c, 1.0, 2.0, 1.0) == pytest.approx((2.0, 6.0, 1.0, 3.0))
    # at u0 = 1: s1 = -3, s2 = 2
    assert O.linearise_px(c, 2.0, 1.0, 1.0) == pytest.approx((-6.0, 4.0, 0.0, 2.0))
    # at u0 = 4: s1 = 1, s2 = -11 < s1 -> both the mean -5
    assert O.linearise_px(c, 1.0, 4.0, 1.0) == pytest.approx((-5.0, -5.0, 3.0, 5.0))
    # at the label range ends the argument is clamped: D(-1) = D(0)
    assert O.linearise_px(c, 1.0, 0.0, 1.0) == pytest.approx((-1.5, -1.5, 0.0, 1.0))
    assert O.linearise_px(c, 1.0, 0.5, 1.0)[2:] == pytest.approx((0.0, 1.5))


def test_data_prox_is_argmin():
    rng = np.random.default_rng(0)
    for _ in range(200):
        u0 = rng.uniform(2, 8)
        s1, s2 = sorted(rng.uniform(-6, 6, size=2))
        lo, hi = u0 - rng.uniform(0, 1.5), u0 + rng.uniform(0, 1.5)
        tau = rng.uniform(0.05, 1.0)
        uh = u0 + rng.uniform(-4, 4)

        def obj(u):
            d = np.where(u <= u0, s1 * (u - u0), s2 * (u - u0))
            return d + (u - uh) ** 2 / (2 * tau)
        ref, dx = _grid_argmin(obj, lo, hi)
        assert O.prox_data(uh, u0, s1, s2, lo, hi, tau) == pytest.approx(ref, abs=2 * dx)


@pytest.mark.parametrize("a,b", [(0.25, 1.0), (0.0, 2.75), (0.5, 2.0)])
def test_conjugate_is_numeric_sup(a, b):
    omega = 6.0
    ts = np.linspace(-200, 200, 400001)
    rt = omega * np.where(np.abs(ts) <= b, a * np.abs(ts), np.abs(ts) - b * (1 - a))
    for s in np.linspace(-omega, omega, 41):
        assert O.conj(s, omega, a, b) == pytest.approx(np.max(s * ts - rt), abs=1e-6)
    assert O.conj(omega * 1.01, omega, a, b) == np.inf


@pytest.mark.parametrize("a,b", [(0.25, 1.0), (0.0, 2.75), (0.5, 2.0)])
def test_conjugate_prox_is_argmin(a, b):
    rng = np.random.default_rng(1)
    omega = 5.0
    for _ in range(100):
        t = rng.uniform(-12, 12)
        step = rng.uniform(0.05, 2.0)

        def obj(s):
            g = b * np.maximum(0.0, np.abs(s) - omega * a)
            return step * g + (s - t) ** 2 / 2

        ref, dx = _grid_argmin(obj, -omega, omega)
        assert O.prox_conj(t, omega, a, b, step) == pytest.approx(ref, abs=2 * dx)


def test_continuous_energy_at_labels_equals_discrete_energy():
    sp = S.make_workload(S.SMALL, seed=1)
    cost = O.cost_volume(sp.left, sp.right, 16)
    wh, wv = O.edge_weights(sp.left)
    rng = np.random.default_rng(2)
    for _ in range(3):
        labels = rng.integers(0, 16, size=cost.shape[:2]).astype(np.uint16)
        e_d = O.discrete_energy(cost, wh, wv, labels)
        e_c = O.cont_energy(cost.astype(float), wh.astype(float), wv.astype(float),
                            labels.astype(float))
        assert e_c == pytest.approx(e_d, abs=1e-9)


def _small_problem(seed=3):
    sp = S.make_pair(12, 16, 16, planes=3, seed=seed)
    cost = O.cost_volume(sp.left, sp.right, 16).astype(float)
    wh, wv = O.edge_weights(sp.left)
    u0 = np.random.default_rng(seed).uniform(0, 15, size=(12, 16))
    return cost, wh.astype(float), wv.astype(float), u0


def test_convex_case_gap_closes():
    # C -> infinity removes R- (q stays 0): min_u D~(u) + R+(Au) is convex and the
    # primal-dual gap of Eq. (cont_nonlin_pd) must vanish
    cost, wh, wv, u0 = _small_problem()
    for lam_r in (1.0, 4.0):
        P = O.Params(C=1e7, warps=1, lambda_r=lam_r)
        u, (ph, pv, qh, qv), _ = O.refine(cost, wh, wv, u0, 20000, P)
        assert np.all(qh == 0) and np.all(qv == 0)
        pr, du = O.convex_gap(cost, wh, wv, u0, u, ph, pv, P)
        assert abs(pr - du) <= 1e-9 * abs(pr)


def test_zero_weights_reach_pixelwise_minimiser():
    cost, wh, wv, u0 = _small_problem(4)
    P = O.Params(warps=1)
    u, _, _ = O.refine(cost, 0 * wh, 0 * wv, u0, 200, P)
    for y in range(12):
        for x in range(16):
            s1, s2, lo, hi = O.linearise_px(cost[y, x], 1.0, u0[y, x], 1.0)
            ref = u0[y, x] if s1 <= 0 <= s2 else (lo if s1 > 0 else hi)
            assert u[y, x] == pytest.approx(ref, abs=1e-12)


def test_dual_feasibility_and_box():
    sp = S.make_workload(S.SMALL, seed=2)
    cost = O.cost_volume(sp.left, sp.right, 16)
    wh, wv = O.edge_weights(sp.left)
    labels, _, _, _ = O.dmm(cost, wh, wv, 3)
    P = O.Params(lambda_r=1.5)
    u, (ph, pv, qh, qv), en = O.refine(cost.astype(float), wh.astype(float), wv.astype(float),
                                       labels.astype(float), 50, P)
    for arr, w in ((ph, wh), (pv, wv), (qh, wh), (qv, wv)):
        assert np.all(np.abs(arr) <= 1.5 * w + 1e-12)
    assert np.all(u >= 0) and np.all(u <= 15)
    # 5 warps of half-width 1 around the labels
    assert np.all(np.abs(u - labels) <= 5.0 + 1e-12)


# --- planted mistakes: each must be caught by the convex-gap pin -------------

MUTATIONS = [
    ("sign of A^T in the primal step", "u[p] - tau * div", "u[p] + tau * div"),
    ("no extrapolation in the dual step",
     "double ext = (2.0 * un[p] - u[p]) - (2.0 * un[p + 1] - u[p + 1]);",
     "double ext = un[p] - un[p + 1];"),
    ("data prox middle case returns the input", "else v = u0;", "else v = uh;"),
    ("dual prox without the clamp", "if (tp > omega) tp = omega;", "(void)0;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS)
def test_pins_catch_planted_mistakes(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(O.__file__), "dm_oracle.c")).read()
    assert old in src, name
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(mut), "-lm"],
                   check=True)
    lib = ctypes.CDLL(str(so))
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.or_refine.argtypes = ([ctypes.c_int] * 3 + [f64p] * 4 + [ctypes.c_int,
                              ctypes.POINTER(O.ContParams)] + [f64p] * 5 + [ctypes.c_int, f64p])
    cost, wh, wv, u0 = _small_problem()
    H, W, L = cost.shape
    P = O.Params(C=1e7, warps=1, lambda_r=4.0)
    u = u0.copy()
    st = [np.zeros((H, W)) for _ in range(4)]
    en = np.zeros(1)
    cp = P.cont()
    p = lambda a: a.ctypes.data_as(f64p)
    lib.or_refine(H, W, L, p(cost), None, p(wh), p(wv), 20000, ctypes.byref(cp), p(u),
                  *[p(s) for s in st], 1, p(en))
    pr, du = O.convex_gap(cost, wh, wv, u0, u, st[0], st[1], P)
    assert not (np.isfinite(pr) and abs(pr - du) <= 1e-9 * abs(pr)), f"not caught: {name}"


# --- reverse mode of the refinement (the differentiable form) -----------------

def _adjoint_problem(seed=2):
    H, W, L = 12, 16, 16
    sp = S.make_pair(H, W, L, planes=3, seed=seed)
    rng = np.random.default_rng(seed)
    cost = O.cost_volume(sp.left, sp.right, L).astype(float) + rng.uniform(0, 1, (H, W, L))
    wh, wv = O.edge_weights(sp.left)
    u0 = np.argmin(cost, -1).astype(float)
    alpha = rng.uniform(0.5, 1.5, (H, W))
    return cost, wh.astype(float), wv.astype(float), u0, alpha, sp.gt


def _fd_directions(gradfn, lossfn, cost, alpha, lam, n, seed, h=1e-6):
    """(finite difference, adjoint) pairs on random joint directions; a direction
    whose difference quotients at h and h/2 disagree straddles a kink and is skipped."""
    gc, ga, gl = gradfn
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        vc, va, vl = rng.normal(size=cost.shape), rng.normal(size=alpha.shape), rng.normal()
        def q(hh):
            return (lossfn(cost + hh * vc, alpha + hh * va, lam + hh * vl)
                    - lossfn(cost - hh * vc, alpha - hh * va, lam - hh * vl)) / (2 * hh)
        f1, f2 = q(h), q(h / 2)
        if abs(f1 - f2) > 1e-6 * max(1.0, abs(f1)):
            continue
        out.append((f1, float((gc * vc).sum() + (ga * va).sum() + gl * vl)))
    return out


def test_refine_gradient_matches_finite_differences():
    cost, wh, wv, u0, alpha, gt = _adjoint_problem()
    iters, lam = 30, 1.2
    P = O.Params(warps=3, lambda_r=lam)
    u, loss, gc, ga, gl = O.refine_grad(cost, wh, wv, u0, iters, gt, P, alpha)
    ur, _, _ = O.refine(cost, wh, wv, u0, iters, P, alpha)
    assert np.array_equal(u, ur) and loss == pytest.approx(np.abs(ur - gt).mean(), rel=1e-15)

    def lossfn(c, a, l):
        uu, _, _ = O.refine(c, wh, wv, u0, iters, O.Params(warps=3, lambda_r=l), a)
        return np.abs(uu - gt).mean()
    pairs = _fd_directions((gc, ga, gl), lossfn, cost, alpha, lam, 16, seed=3)
    assert len(pairs) >= 12
    for fd, an in pairs:
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9)


def _half_integer_start(labels, L):
    return np.clip(labels, 4, L - 6) + 0.5


def _u0_fd_errors(grad_u0, cost, wh, wv, u0, alpha, gt, iters, lam, n=12, seed=5, h=1e-6):
    """relative errors of g_u0 . v against central differences in the start u0,
    on directions whose quotients at h and h/2 agree"""
    def lossfn(uu):
        u, _, _ = O.refine(cost, wh, wv, uu, iters, O.Params(warps=3, lambda_r=lam), alpha)
        return np.abs(u - gt).mean()
    rng = np.random.default_rng(seed)
    errs = []
    for _ in range(n):
        v = rng.normal(size=u0.shape)
        q = lambda hh: (lossfn(u0 + hh * v) - lossfn(u0 - hh * v)) / (2 * hh)
        f1, f2 = q(h), q(h / 2)
        if abs(f1 - f2) > 1e-6 * max(1.0, abs(f1)):
            continue
        errs.append(abs(float((grad_u0 * v).sum()) - f1) / max(abs(f1), 1e-9))
    return errs


def test_refine_gradient_in_the_start_matches_finite_differences():
    # the start is the argmin labelling moved to the half-integers and kept 4
    # labels inside the range: the clamped interpolation has its kinks at the
    # integers, and three warps of half-width 1 then never reach the ends of
    # the range.  Neighbours with equal labels put the q prox (a = 0) exactly at
    # t = 0 in the first iteration, where the map is constant around t (its
    # derivative is 0).
    # (after a few iterations equal neighbours meet further exact ties, kinks at
    # the base point that central differences average over; 4 iterations stay
    # clear of them)
    cost, wh, wv, u0, alpha, gt = _adjoint_problem(seed=4)
    u0 = _half_integer_start(u0, cost.shape[2])
    iters, lam = 4, 1.2
    P = O.Params(warps=3, lambda_r=lam)
    _, _, _, _, _, g0 = O.refine_grad(cost, wh, wv, u0, iters, gt, P, alpha, want_u0=True)
    errs = _u0_fd_errors(g0, cost, wh, wv, u0, alpha, gt, iters, lam)
    assert len(errs) >= 8 and max(errs) <= 1e-6


def test_start_gradient_pin_catches_the_wrong_tie_of_the_dual_prox(tmp_path):
    src = open(os.path.join(os.path.dirname(O.__file__), "dm_oracle.c")).read()
    old, new = "if (fabs(t) < a * omega) {", "if (fabs(t) <= a * omega) {"
    assert old in src
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(mut), "-lm"],
                   check=True)
    lib = ctypes.CDLL(str(so))
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.or_refine_grad.argtypes = ([ctypes.c_int] * 3 + [f64p] * 5 + [ctypes.c_int,
                                   ctypes.POINTER(O.ContParams)] + [f64p] * 7)
    cost, wh, wv, u0, alpha, gt = _adjoint_problem(seed=4)
    u0 = _half_integer_start(u0, cost.shape[2])
    H, W, L = cost.shape
    iters, lam = 4, 1.2
    cp = O.Params(warps=3, lambda_r=lam).cont()
    out = [np.zeros((H, W)), np.zeros(1), np.zeros((H, W, L)), np.zeros((H, W)), np.zeros(1),
           np.zeros((H, W))]
    p = lambda a: np.ascontiguousarray(a).ctypes.data_as(f64p)
    lib.or_refine_grad(H, W, L, p(cost), p(alpha), p(wh), p(wv), p(u0), iters, ctypes.byref(cp),
                       p(gt), *[p(o) for o in out])
    errs = _u0_fd_errors(out[5], cost, wh, wv, u0, alpha, gt, iters, lam)
    assert max(errs) > 1e-3


ADJ_MUTATIONS = [
    ("extrapolation factor dropped", "double unb = ub[p] + 2.0 * wbar;", "double unb = ub[p] + wbar;"),
    ("data slope sign", "s2b[p] -= tau * unb;", "s2b[p] += tau * unb;"),
    ("convexity fix not reversed", "if (s2r < s1r) { double m = 0.5 * (b1 + b2); b1 = m; b2 = m; }", "(void)0;"),
]


@pytest.mark.parametrize("name,old,new", ADJ_MUTATIONS)
def test_adjoint_pin_catches_planted_mistakes(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(O.__file__), "dm_oracle.c")).read()
    assert old in src, name
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(mut), "-lm"],
                   check=True)
    lib = ctypes.CDLL(str(so))
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.or_refine_grad.argtypes = ([ctypes.c_int] * 3 + [f64p] * 5 + [ctypes.c_int,
                                   ctypes.POINTER(O.ContParams)] + [f64p] * 7)
    cost, wh, wv, u0, alpha, gt = _adjoint_problem()
    H, W, L = cost.shape
    iters, lam = 30, 1.2
    cp = O.Params(warps=3, lambda_r=lam).cont()
    u, loss, gc, ga, gl = np.zeros((H, W)), np.zeros(1), np.zeros((H, W, L)), np.zeros((H, W)), np.zeros(1)
    p = lambda a: np.ascontiguousarray(a).ctypes.data_as(f64p)
    lib.or_refine_grad(H, W, L, p(cost), p(alpha), p(wh), p(wv), p(u0), iters, ctypes.byref(cp),
                       p(gt), p(u), p(loss), p(gc), p(ga), p(gl), None)

    def lossfn(c, a, l):
        uu, _, _ = O.refine(c, wh, wv, u0, iters, O.Params(warps=3, lambda_r=l), a)
        return np.abs(uu - gt).mean()
    pairs = _fd_directions((gc, ga, float(gl[0])), lossfn, cost, alpha, lam, 16, seed=3)
    assert any(abs(an - fd) > 1e-6 * max(abs(fd), 1e-3) for fd, an in pairs), f"not caught: {name}"


def test_unrolled_refinement_is_kinked_at_the_1e3_scale_after_many_iterations():
    """Central differences of the exact (FP64) unrolled refinement along random
    unit directions in (cost, alpha, lambda_r): after 30 iterations the
    quotients at h = 1e-3 and h/2 agree to ~1e-8 (the loss is linear at that
    scale); after 200 iterations they disagree by several percent or more along
    every direction: the piecewise-linear iteration amplifies perturbations, so
    finite differences at h = 1e-3 cannot confirm a gradient there."""
    H, W, L = 32, 64, 96
    sp = S.make_pair(H, W, L, planes=4, noise_sigma=2.0, seed=0)
    rng = np.random.default_rng(1)
    cost = O.cost_volume(sp.left, sp.right, L) + rng.uniform(0, 1, (H, W, L))
    wh, wv = (w.astype(float) for w in O.edge_weights(sp.left))
    alpha = rng.uniform(0.5, 1.5, (H, W))
    u0 = np.clip(np.argmin(cost, 2) + rng.uniform(-0.3, 0.3, (H, W)), 0, L - 1)
    spread = {}
    for iters in (30, 200):
        def lossf(c, a, lam):
            u = O.refine(c, wh, wv, u0, iters, O.Params(lambda_r=lam), a)[0]
            return np.abs(u - sp.gt).mean()
        drng = np.random.default_rng(2)
        out = []
        for _ in range(12):
            v = drng.standard_normal(cost.size + alpha.size + 1)
            v /= np.linalg.norm(v)
            vc, va, vl = v[:cost.size].reshape(cost.shape), v[cost.size:-1].reshape(alpha.shape), v[-1]

            def q(h):
                return (lossf(cost + h * vc, alpha + h * va, 1 + h * vl)
                        - lossf(cost - h * vc, alpha - h * va, 1 - h * vl)) / (2 * h)
            a, b = q(1e-3), q(5e-4)
            out.append(abs(a - b) / abs(a))
        spread[iters] = np.array(out)
    assert np.median(spread[30]) < 1e-6
    assert np.sum(spread[200] > 1e-2) >= 10
