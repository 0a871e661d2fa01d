"""Pins of the oracle's discrete stage against the paper and brute force.

Each test checks the oracle against something other than itself: values the
paper prints (the worked example of App. A), exhaustive enumeration on tiny
inputs, closed forms and the propositions the paper proves.
"""

import itertools
import os
import shutil
import subprocess
import ctypes

import numpy as np
import pytest

import bruteforce as B
from oracle import oracle as O
from paper_1601_06274_gb300 import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")


def _we():
    g = B.read_golden(GOLDEN)
    U = g["unary"]
    theta = np.array([[int(U[l][k]) for l in range(3)] for k in range(6)], dtype=np.int64)
    return g, theta


# --- penalty r (Eq. r-decompose) --------------------------------------------

def test_penalty_dc_split_is_truncated_linear():
    # r = r_{eps,delta} - r_{0,C+delta-eps delta} is the truncated norm of Fig. 2:
    # eps|t| up to delta, then slope 1, truncated at C.
    for eps, delta, C in [(0.25, 1.0, 2.0), (0.5, 1.0, 3.0), (0.25, 2.0, 4.0), (0.0, 1.0, 1.0)]:
        P = O.Params(eps=eps, delta=delta, C=C)
        for t in np.linspace(-9, 9, 181):
            at = abs(t)
            closed = eps * at if at <= delta else min(C, at - delta + eps * delta)
            assert O.r(t, P) == pytest.approx(closed, abs=1e-12)
        # both parts convex (midpoint test)
        for a, b in [(eps, delta), (0.0, C + delta - eps * delta)]:
            ts = np.linspace(-9, 9, 73)
            f = np.array([O.lib().or_r_ab(float(t), a, b) for t in ts])
            assert np.all(f[1:-1] <= 0.5 * (f[:-2] + f[2:]) + 1e-12)


def test_penalty_table_values():
    # omega = 8 with eps = 1/4, delta = 1, C = 2: {0, 2, 10, 16, 16, ...}
    assert O.penalty_table(8, 6).tolist() == [0, 2, 10, 16, 16, 16]
    assert O.penalty_table(4, 5).tolist() == [0, 1, 5, 8, 8]
    assert O.penalty_table(0, 4).tolist() == [0, 0, 0, 0]
    with pytest.raises(RuntimeError):
        O.penalty_table(3, 4)  # 3 * 1/4 is not an integer


# --- Msg and min-marginals (App. A) ------------------------------------------

def test_msg_is_min_convolution():
    rng = np.random.default_rng(0)
    for _ in range(50):
        K = int(rng.integers(1, 9))
        a = rng.integers(-20, 20, size=K)
        V = np.sort(rng.integers(0, 15, size=K))
        V[0] = 0
        out = O.msg(a, V)
        ref = [min(int(a[x]) + int(V[abs(x - xp)]) for x in range(K)) for xp in range(K)]
        assert out.tolist() == ref


def test_min_marginals_worked_example_w5():
    g, theta = _we()
    V = np.tile(np.array([0, 5, 5], dtype=np.int64), (5, 1))
    mm = O.min_marginals(theta, V)
    fstar = mm.min()
    printed = np.array(g["w5_min_marginals"], dtype=np.int64)  # rows = labels
    assert (mm - fstar).T.tolist() == printed.tolist()


def test_min_marginals_bruteforce():
    rng = np.random.default_rng(1)
    for _ in range(60):
        n, K = int(rng.integers(1, 6)), int(rng.integers(1, 4))
        theta = rng.integers(-5, 10, size=(n, K))
        V = np.zeros((max(n - 1, 1), K), dtype=np.int64)
        for k in range(n - 1):
            V[k] = O.penalty_table(4 * int(rng.integers(0, 3)), K)
        mm = O.min_marginals(theta, V)
        ref = B.min_marginals(theta.tolist(), V.tolist())
        assert mm.tolist() == ref


def test_uniform_minorant_reading_matches_printed_example():
    # pins the meaning of "minorant" (unaries indexed [label][node], built on the
    # chain normalised by its minimum) used throughout the oracle's invariants
    g, theta = _we()
    for w, key_first, key_final in [(1, "w1_first_minorant", "w1_final_minorant"),
                                    (5, None, "w5_final_minorant")]:
        V = [[0, w, w]] * 5
        hist = B.uniform_minorant(theta.tolist(), V)
        final = [[hist[-1][k][l] for k in range(6)] for l in range(3)]
        assert final == g[key_final]
        if key_first:
            first = [[hist[0][k][l] for k in range(6)] for l in range(3)]
            assert first == g[key_first]
        # Lemma: the uniform minorant dominates m/n (n = 6)
        mm = B.min_marginals(theta.tolist(), V)
        fs = B.chain_min(theta.tolist(), V)
        for k in range(6):
            for l in range(3):
                assert hist[-1][k][l] >= B.Fraction(mm[k][l] - fs, 6)


# --- hierarchical minorant (App. A, Alg. Handshake) --------------------------

def _random_chain(rng, n, K, kind):
    theta = rng.integers(-4, 12, size=(n, K))
    V = np.zeros((max(n - 1, 1), K), dtype=np.int64)
    for k in range(n - 1):
        w = int(rng.integers(0, 8))
        if kind == 0:
            V[k] = [0] + [w] * (K - 1)
        elif kind == 1:
            V[k] = O.penalty_table(4 * int(rng.integers(0, 3)), K)
        else:
            V[k] = np.minimum(np.arange(K) * w, 3 * w)
    return theta, V


def test_hier_minorant_valid_and_exact():
    # validity: lam(x) <= f(x) for every labelling (Prop. P:dual-minorant needs a
    # minorant); exactness: sum_i min lam_i = min f (tight at the optimum)
    rng = np.random.default_rng(2)
    for trial in range(240):
        n, K = int(rng.integers(1, 7)), int(rng.integers(1, 4))
        theta, V = _random_chain(rng, n, K, trial % 3)
        lam = O.hier_minorant(theta, V)
        fmin = None
        for x in itertools.product(range(K), repeat=n):
            f = B.chain_energy(theta.tolist(), V.tolist(), x)
            assert sum(int(lam[k, x[k]]) for k in range(n)) <= f
            fmin = f if fmin is None else min(fmin, f)
        assert int(lam.min(axis=1).sum()) == fmin


def test_hier_minorant_matches_enumerated_messages():
    # the oracle's messages come from dynamic programming; here every message is
    # the min-marginal of its definition, computed by enumeration
    rng = np.random.default_rng(12)
    for trial in range(150):
        n, K = int(rng.integers(1, 7)), int(rng.integers(1, 4))
        theta, V = _random_chain(rng, n, K, trial % 3)
        lam = O.hier_minorant(theta, V)
        assert lam.tolist() == B.hier_minorant_enum(theta.tolist(), V.tolist())


def test_hier_minorant_is_maximal():
    # Lemma (App. A): for a maximal minorant all min-marginals of f - lam vanish
    rng = np.random.default_rng(13)
    for trial in range(120):
        n, K = int(rng.integers(1, 6)), int(rng.integers(1, 4))
        theta, V = _random_chain(rng, n, K, trial % 3)
        lam = O.hier_minorant(theta, V)
        mm = B.min_marginals((theta - lam).tolist(), V.tolist())
        assert all(v == 0 for row in mm for v in row)


def test_hier_minorant_worked_example_valid_exact():
    _, theta = _we()
    for w in (1, 5):
        V = np.tile(np.array([0, w, w], dtype=np.int64), (5, 1))
        lam = O.hier_minorant(theta, V)
        fs = B.chain_min(theta.tolist(), V.tolist())
        assert int(lam.min(axis=1).sum()) == fs
        for x in itertools.product(range(3), repeat=6):
            assert sum(int(lam[k, x[k]]) for k in range(6)) <= B.chain_energy(theta.tolist(), V.tolist(), x)


def _two_node_procedure(th1, th2, F, half):
    """The four bullet points of App. A for a chain of length two, written with
    explicit minimisations over the full pairwise table F[a][b]."""
    K = len(th1)
    m1 = [min(th1[a] + F[a][b] + th2[b] for b in range(K)) for a in range(K)]
    lam1 = [half(m) for m in m1]                              # a half of the min-marginal
    phi12 = [min(th1[a] - lam1[a] + F[a][b] for a in range(K)) for b in range(K)]
    lam2 = [phi12[b] + th2[b] for b in range(K)]              # the whole remaining min-marginal
    phi21 = [min(th2[b] - lam2[b] + F[a][b] for b in range(K)) for a in range(K)]
    lam1 = [lam1[a] + (th1[a] - lam1[a] + phi21[a]) for a in range(K)]
    return lam1, lam2


def test_hier_minorant_two_nodes_matches_paper_procedure():
    rng = np.random.default_rng(3)
    for _ in range(100):
        K = int(rng.integers(1, 5))
        w = int(rng.integers(0, 3)) * 4
        Vt = O.penalty_table(w, K)
        # (a) even data: m_1 is even, no rounding, the paper's procedure exactly
        th1 = (2 * rng.integers(-6, 10, size=K)).tolist()
        th2 = (2 * rng.integers(-6, 10, size=K)).tolist()
        F = [[2 * int(Vt[abs(a - b)]) for b in range(K)] for a in range(K)]
        lam = O.hier_minorant(np.array([th1, th2]), np.array([2 * Vt]))
        lam1, lam2 = _two_node_procedure(th1, th2, F, lambda m: B.Fraction(m, 2))
        assert lam[0].tolist() == lam1 and lam[1].tolist() == lam2
        # (b) any integers: Alg. Handshake shares floor(m/2) - phi_21 to the right,
        # i.e. the first node keeps ceil(m_1/2)
        th1 = rng.integers(-6, 10, size=K).tolist()
        th2 = rng.integers(-6, 10, size=K).tolist()
        F = [[int(Vt[abs(a - b)]) for b in range(K)] for a in range(K)]
        lam = O.hier_minorant(np.array([th1, th2]), np.array([Vt]))
        lam1, lam2 = _two_node_procedure(th1, th2, F, lambda m: -((-m) // 2))
        assert lam[0].tolist() == lam1 and lam[1].tolist() == lam2


def test_hier_minorant_zero_pairwise_keeps_unaries():
    # with zero pairwise terms every message is a constant, so each node keeps
    # its unary up to a constant, and the constants cancel over the chain
    rng = np.random.default_rng(4)
    for n in (1, 2, 3, 7, 16, 33):
        theta = rng.integers(-50, 50, size=(n, 5))
        lam = O.hier_minorant(theta, np.zeros((max(n - 1, 1), 5), dtype=np.int64))
        shift = lam - theta
        assert np.all(shift == shift[:, :1])
        assert int(shift[:, 0].sum()) == 0


def test_hier_minorant_long_chain_exact_vs_viterbi():
    rng = np.random.default_rng(5)
    for n in (17, 40, 101):
        theta, V = _random_chain(rng, n, 4, 1)
        lam = O.hier_minorant(theta, V)
        assert int(lam.min(axis=1).sum()) == B.viterbi_min(theta.tolist(), V.tolist())


# --- census and cost volume (Sec. 3.1) ---------------------------------------

@pytest.mark.parametrize("win", [3, 5])
def test_census_and_cost_bruteforce(win):
    rng = np.random.default_rng(6)
    left = rng.integers(0, 256, size=(7, 11), dtype=np.uint8)
    right = rng.integers(0, 256, size=(7, 11), dtype=np.uint8)
    left[2, 3:6] = 100  # ties
    cl = O.census(left, win)
    assert np.array_equal(cl, B.census_ref(left, win))
    L = 6
    cost = O.cost_volume(left, right, L, win)
    cr = B.census_ref(right, win)
    for y in range(7):
        for x in range(11):
            for l in range(L):
                ref = B.hamming(cl[y, x], cr[y, x - l]) if x - l >= 0 else win * win - 1
                assert cost[y, x, l] == ref


def test_edge_weights_definition():
    img = np.array([[0, 15, 31, 31], [16, 15, 100, 60]], dtype=np.uint8)
    wh, wv = O.edge_weights(img)
    assert wh.tolist() == [[8, 4, 8, 0], [8, 4, 4, 0]]
    assert wv.tolist() == [[4, 8, 4, 4], [0, 0, 0, 0]]


# --- Dual MM (Alg. Dual_MM) ---------------------------------------------------

def _tables(K):
    cache = {}

    def table_of(w):
        if w not in cache:
            cache[w] = O.penalty_table(w, K).tolist()
        return cache[w]
    return table_of


def test_dmm_weak_duality_bruteforce_grids():
    # LB <= min E <= E(output labels) on grids small enough to enumerate
    rng = np.random.default_rng(7)
    for trial in range(12):
        H, W, K = [(2, 3, 3), (3, 3, 2), (3, 4, 2), (2, 2, 3)][trial % 4]
        cost = rng.integers(0, 10, size=(H, W, K)).astype(np.int32)
        wh = (rng.integers(0, 3, size=(H, W)) * 4).astype(np.int32)
        wv = (rng.integers(0, 3, size=(H, W)) * 4).astype(np.int32)
        wh[:, -1] = 0
        wv[-1, :] = 0
        labels, lb, _, _ = O.dmm(cost, wh, wv, 4)
        emin = B.grid_min(cost, wh, wv, _tables(K))
        e = O.discrete_energy(cost, wh, wv, labels)
        assert e == B.grid_energy(cost, wh, wv, _tables(K), labels.tolist())
        assert np.all(lb <= emin) and emin <= e
        assert np.all(np.diff(lb) >= 0)


def test_dmm_lb_monotone_and_below_energy():
    sp = S.make_workload(S.SMALL, seed=0)
    cost = O.cost_volume(sp.left, sp.right, 16)
    wh, wv = O.edge_weights(sp.left)
    labels, lb, lam_h, lam_v = O.dmm(cost, wh, wv, 5)
    assert np.all(np.diff(lb) >= 0)
    assert lb[-1] <= O.discrete_energy(cost, wh, wv, labels)
    l2, b2 = O.dmm_outputs(lam_h, lam_v)
    assert np.array_equal(l2, labels) and b2 == lb[-1]


def test_dmm_passes_are_exact_chain_minima():
    # after the horizontal pass, lam_h + lam_v is the hierarchical minorant of
    # every row chain (c + lam_v), so its per-row bound is the row's Viterbi
    # minimum; likewise for the vertical pass with unaries lam_h
    rng = np.random.default_rng(8)
    H, W, L = 5, 7, 4
    cost = rng.integers(0, 9, size=(H, W, L)).astype(np.int32)
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    wh, wv = O.edge_weights(img)
    lam_v = np.zeros((H, W, L), dtype=np.int64)
    for it in range(3):
        lam_h = O.dmm_pass(cost, wh, wv, 0, lam_v)
        tot = lam_h + lam_v
        for y in range(H):
            theta = (cost[y] + lam_v[y]).tolist()
            V = [O.penalty_table(int(wh[y, x]), L).tolist() for x in range(W - 1)]
            assert int(tot[y].min(axis=1).sum()) == B.viterbi_min(theta, V)
        lam_v = O.dmm_pass(cost, wh, wv, 1, lam_h)
        tot = lam_h + lam_v
        for x in range(W):
            theta = lam_h[:, x].tolist()
            V = [O.penalty_table(int(wv[y, x]), L).tolist() for y in range(H - 1)]
            assert int(tot[:, x].min(axis=1).sum()) == B.viterbi_min(theta, V)


def test_dmm_single_row_is_exact():
    rng = np.random.default_rng(9)
    cost = rng.integers(0, 25, size=(1, 30, 6)).astype(np.int32)
    img = rng.integers(0, 256, size=(1, 30), dtype=np.uint8)
    wh, wv = O.edge_weights(img)
    labels, lb, lam_h, lam_v = O.dmm(cost, wh, wv, 1)
    theta = cost[0].tolist()
    V = [O.penalty_table(int(wh[0, x]), 6).tolist() for x in range(29)]
    assert lb[0] == B.viterbi_min(theta, V)
    assert np.all(lam_v == 0)


def test_dmm_zero_pairwise_is_winner_take_all():
    rng = np.random.default_rng(10)
    cost = rng.integers(0, 25, size=(6, 9, 7)).astype(np.int32)
    z = np.zeros((6, 9), dtype=np.int32)
    labels, lb, _, _ = O.dmm(cost, z, z, 2)
    assert np.array_equal(labels, np.argmin(cost, axis=2))
    assert lb[-1] == int(cost.min(axis=2).sum())


# --- planted mistakes: each must be caught by a pin above ---------------------

MUTATIONS = [
    ("no halving in the Handshake", "tmp[l] = floor_half(m_i[l]) - phi_ji[l];",
     "tmp[l] = m_i[l] - phi_ji[l];"),
    ("no bounce-back", "or_msg(K, tmp, V + (i64)i * K, phi_ji);                  /* bounce back",
     "(void)0;                  /* bounce back"),
    ("wrong edge table in the backward sweep", "or_msg(K, tmp, V + (i64)(k - 1) * K, Rm);",
     "or_msg(K, tmp, V + (i64)(k - 2 < 0 ? 0 : k - 2) * K, Rm);"),
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
    lib.or_hier_minorant.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int64)] * 3
    p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))

    def mut_hier(theta, V):
        theta = np.ascontiguousarray(theta, dtype=np.int64)
        V = np.ascontiguousarray(V, dtype=np.int64)
        lam = np.zeros_like(theta)
        lib.or_hier_minorant(theta.shape[0], theta.shape[1], p(theta), p(V), p(lam))
        return lam

    rng = np.random.default_rng(11)
    caught = False
    # the two-node procedure of App. A
    for _ in range(50):
        K = int(rng.integers(2, 5))
        Vt = O.penalty_table(4 * int(rng.integers(1, 3)), K)
        th1 = rng.integers(-6, 10, size=K).tolist()
        th2 = rng.integers(-6, 10, size=K).tolist()
        F = [[int(Vt[abs(a - b)]) for b in range(K)] for a in range(K)]
        lam = mut_hier(np.array([th1, th2]), np.array([Vt]))
        lam1, lam2 = _two_node_procedure(th1, th2, F, lambda m: -((-m) // 2))
        if lam[0].tolist() != lam1 or lam[1].tolist() != lam2:
            caught = True
            break
    # validity, exactness and the enumerated-message restatement on random chains
    for trial in range(200):
        if caught:
            break
        n, K = int(rng.integers(2, 6)), int(rng.integers(2, 4))
        theta, V = _random_chain(rng, n, K, trial % 3)
        lam = mut_hier(theta, V)
        if lam.tolist() != B.hier_minorant_enum(theta.tolist(), V.tolist()):
            caught = True
            break
        if int(lam.min(axis=1).sum()) != B.chain_min(theta.tolist(), V.tolist()):
            caught = True
            break
        for x in itertools.product(range(K), repeat=n):
            if sum(int(lam[k, x[k]]) for k in range(n)) > B.chain_energy(theta.tolist(), V.tolist(), x):
                caught = True
                break
    assert caught, f"planted mistake not caught: {name}"
