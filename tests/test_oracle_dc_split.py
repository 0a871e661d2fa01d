"""Pins of the oracle's refinement on its non-convex half: the q step of the
difference-of-convex split (Sec. 2.4, Eq. r-decompose, Eq. cont_problem and
the iterates of Eq. cont_iterates with the gradient of the operator A(x)).

Two facts that hold independently of how the oracle writes the step:

* Critical point.  A fixed point (u, p, q) of the iterates satisfies, edge by
  edge with t = (Au)_e and w = lambda_R omega_e,
      q_e in dR-(t)     (R- = w r_{0, C + delta - eps delta}),
      p_e in dR+(t)     (R+ = w r_{eps, delta}),
  and, pixel by pixel, -(A^T (p - q))_i in the subdifferential of the
  linearised data term (slopes s1, s2 at the linearisation point, box).
  These are the optimality conditions of the three proximal steps, written
  with the subdifferentials of the convex pieces of Sec. 2.4 and 3.1; they do
  not depend on the step sizes.  Started from a Dual MM labelling (how the
  method uses the refinement), the iteration reaches its fixed point exactly
  on these small problems.
* Structure of one iteration.  In Eq. cont_iterates the primal block
  x = (u, q) moves with step tau from x^k and y^k only: the q-block of
  grad A(x)^T y is -A u^k (times the dummy d = 1), so q^{k+1} depends on
  neither p^k nor sigma, nor on the u^{k+1} computed in the same iteration.

Neither pin calls the reverse mode of the oracle.  The planted mistakes at the
end (the sign of the q step, sigma in place of tau, the new u in place of the
old one) are each caught by at least one of them.
"""

import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_06274_gb300 import synthetic as S

TOL = 1e-9


def _dmm_start(seed, H=12, W=16, L=16, planes=4, frac=0.0):
    """a small pair, its Dual MM labelling as the start (optionally moved off
    the integers by up to frac/2), and float copies of cost and weights"""
    sp = S.make_pair(H, W, L, planes=planes, seed=seed)
    cost = O.cost_volume(sp.left, sp.right, L)
    wh, wv = O.edge_weights(sp.left)
    labels, _, _, _ = O.dmm(cost.astype(np.int32), wh, wv, 5)
    u0 = labels.astype(float)
    if frac:
        u0 = np.clip(u0 + frac * np.random.default_rng(seed).uniform(-0.5, 0.5, u0.shape), 0, L - 1)
    return cost.astype(float), wh.astype(float), wv.astype(float), u0


def _edges(u, ph, pv, qh, qv, wh, wv):
    """(t = Au, p, q, omega) over all horizontal then vertical edges"""
    t = np.concatenate([(u[:, :-1] - u[:, 1:]).ravel(), (u[:-1] - u[1:]).ravel()])
    p = np.concatenate([ph[:, :-1].ravel(), pv[:-1].ravel()])
    q = np.concatenate([qh[:, :-1].ravel(), qv[:-1].ravel()])
    w = np.concatenate([wh[:, :-1].ravel(), wv[:-1].ravel()])
    return t, p, q, w


def in_dR_minus(t, q, w, beta):
    """q in the subdifferential of w * r_{0,beta} at t (r_{0,beta}(t) = max(0, |t| - beta))"""
    a, s = np.abs(t), np.sign(t)
    return np.where(a < beta - TOL, np.abs(q) <= TOL,
                    np.where(a > beta + TOL, np.abs(q - w * s) <= TOL,
                             (q * s >= -TOL) & (np.abs(q) <= w + TOL)))


def in_dR_plus(t, p, w, eps, delta):
    """p in the subdifferential of w * r_{eps,delta} at t (slope w eps inside
    |t| <= delta, slope w outside)"""
    a, s = np.abs(t), np.sign(t)
    inner = np.where(a <= TOL, np.abs(p) <= eps * w + TOL, np.abs(p - eps * w * s) <= TOL)
    outer = np.abs(p - w * s) <= TOL
    kink = (p * s >= eps * w - TOL) & (np.abs(p) <= w + TOL)
    return np.where(a < delta - TOL, inner, np.where(a > delta + TOL, outer, kink))


def data_violations(cost, u0, u, ph, pv, qh, qv, P):
    """pixels where g = -(A^T (p - q))_i is outside the subdifferential of the
    linearised data term D~_i(v) = max(s1 (v - u0), s2 (v - u0)) on [lo, hi]"""
    H, W, _ = cost.shape
    yh, yv = ph - qh, pv - qv
    div = np.zeros((H, W))
    div[:, :-1] += yh[:, :-1]
    div[:, 1:] -= yh[:, :-1]
    div[:-1] += yv[:-1]
    div[1:] -= yv[:-1]
    g = -div
    bad = 0
    for y in range(H):
        for x in range(W):
            s1, s2, lo, hi = O.linearise_px(cost[y, x], 1.0, u0[y, x], P.h)
            v, c = u[y, x], u0[y, x]
            if abs(v - c) <= TOL:
                dl, dr = s1, s2
            elif v < c:
                dl = dr = s1
            else:
                dl = dr = s2
            low = -np.inf if v <= lo + TOL else dl
            high = np.inf if v >= hi - TOL else dr
            bad += not (low - 1e-7 <= g[y, x] <= high + 1e-7)
    return bad


CASES = [(11, 0.35, 0.35), (3, 0.25, 0.45), (11, 0.45, 0.25), (5, 0.25, 0.45)]


@pytest.mark.parametrize("seed,tau,sigma", CASES)
def test_fixed_point_is_a_critical_point_of_the_dc_split(seed, tau, sigma):
    cost, wh, wv, u0 = _dmm_start(seed)
    P = O.Params(warps=1, tau=tau, sigma=sigma)
    u, st, _ = O.refine(cost, wh, wv, u0, 3000, P)
    u2, st2, _ = O.refine(cost, wh, wv, u0, 3500, P)
    change = max(np.abs(u2 - u).max(), *(np.abs(a - b).max() for a, b in zip(st, st2)))
    assert change <= 1e-9, f"no fixed point reached (change {change})"
    assert np.abs(u - u0).max() > 0.1  # the refinement moved the labelling
    t, p, q, w = _edges(u, *st, wh, wv)
    w = P.lambda_r * w
    beta = P.C + P.delta - P.eps * P.delta
    a = np.abs(t)
    # every branch of both subdifferentials is exercised
    assert (a > beta + TOL).sum() >= 3
    assert ((a > P.delta + TOL) & (a < beta - TOL)).sum() >= 3
    assert ((a > TOL) & (a < P.delta - TOL)).sum() >= 3
    assert (a <= TOL).sum() >= 3
    assert in_dR_minus(t, q, w, beta).all()
    assert in_dR_plus(t, p, w, P.eps, P.delta).all()
    assert data_violations(cost, u0, u, *st, P) == 0


def _random_state(cost, wh, wv, P, seed):
    H, W, _ = cost.shape
    rng = np.random.default_rng(seed)
    ph = rng.uniform(-1, 1, (H, W)) * P.lambda_r * wh
    pv = rng.uniform(-1, 1, (H, W)) * P.lambda_r * wv
    qh = rng.uniform(-1, 1, (H, W)) * P.lambda_r * wh
    qv = rng.uniform(-1, 1, (H, W)) * P.lambda_r * wv
    for a in (ph, qh):
        a[:, -1] = 0.0
    for a in (pv, qv):
        a[-1] = 0.0
    return ph, pv, qh, qv


def test_q_step_moves_from_the_old_iterate_with_step_tau():
    cost, wh, wv, u0 = _dmm_start(5, frac=0.6)
    P = O.Params(warps=1, tau=0.3, sigma=0.4)
    ph, pv, qh, qv = _random_state(cost, wh, wv, P, 1)
    ph2, pv2, _, _ = _random_state(cost, wh, wv, P, 2)
    u_a, (pha, pva, qha, qva), _ = O.refine(cost, wh, wv, u0, 1, P, state=(ph, pv, qh, qv))
    # another p^k: u^{k+1} changes, q^{k+1} must not
    u_b, (_, _, qhb, qvb), _ = O.refine(cost, wh, wv, u0, 1, P, state=(ph2, pv2, qh, qv))
    assert np.abs(u_a - u_b).max() > 1e-3
    assert np.array_equal(qha, qhb) and np.array_equal(qva, qvb)
    # another sigma: p^{k+1} changes, q^{k+1} must not
    P2 = O.Params(warps=1, tau=0.3, sigma=0.2)
    _, (phc, pvc, qhc, qvc), _ = O.refine(cost, wh, wv, u0, 1, P2, state=(ph, pv, qh, qv))
    assert np.abs(pha - phc).max() > 1e-3
    assert np.array_equal(qha, qhc) and np.array_equal(qva, qvc)
    # and the step tau does move it
    P3 = O.Params(warps=1, tau=0.2, sigma=0.4)
    _, (_, _, qhd, _), _ = O.refine(cost, wh, wv, u0, 1, P3, state=(ph, pv, qh, qv))
    assert np.abs(qha - qhd).max() > 1e-3


PINS = [lambda c=c: test_fixed_point_is_a_critical_point_of_the_dc_split(*c) for c in CASES] + [
    test_q_step_moves_from_the_old_iterate_with_step_tau]

# (name, [(old, new), ...]); the strings are in the forward refinement only,
# and the reverse mode is left as it is
MUTATIONS = [
    ("q step with the sign of A u flipped",
     [("qh[p] = or_prox_conj(qh[p] + tau * au,", "qh[p] = or_prox_conj(qh[p] - tau * au,"),
      ("qv[p] = or_prox_conj(qv[p] + tau * au,", "qv[p] = or_prox_conj(qv[p] - tau * au,")]),
    ("q prox with step sigma",
     [("qh[p] = or_prox_conj(qh[p] + tau * au, om, 0.0, bq, tau);",
       "qh[p] = or_prox_conj(qh[p] + tau * au, om, 0.0, bq, sigma);"),
      ("qv[p] = or_prox_conj(qv[p] + tau * au, om, 0.0, bq, tau);",
       "qv[p] = or_prox_conj(qv[p] + tau * au, om, 0.0, bq, sigma);")]),
    ("q step from the new u",
     [("double au = u[p] - u[p + 1];", "double au = un[p] - un[p + 1];"),
      ("double au = u[p] - u[p + W];", "double au = un[p] - un[p + W];")]),
    ("q threshold without the eps delta term",
     [("const double bq = P->C + P->delta - P->eps * P->delta;",
       "const double bq = P->C + P->delta;")]),
]


@pytest.mark.parametrize("name,edits", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistakes_in_the_q_step(tmp_path, monkeypatch, name, edits):
    src = open(O._SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    mut = tmp_path / "mut.c"
    mut.write_text(src)
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(mut), "-lm"],
                   check=True)
    monkeypatch.setattr(O, "_lib", O.load(str(so)))
    caught = 0
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught > 0, f"planted mistake not caught: {name}"
