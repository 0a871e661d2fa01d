"""Pins of the oracle's CPU research baselines (App. A and Sec. 2.3):

* the maximal uniform minorant (Alg. uniform-minorant, minimum ratios by
  Dinkelbach's form of Lawler's method) against the exact rational
  enumeration of the test helpers, its maximality, validity and the paper's
  lemma lambda >= m / n;
* Primal_MM (Alg. Primal_MM): primal monotone, never below the grid minimum,
  and a global minimiser is a fixed point.
"""

import numpy as np
import pytest

import bruteforce as B
from oracle import oracle as O


def _chain(rng, n, K, lo=0, hi=12):
    theta = rng.integers(lo, hi, size=(n, K)).astype(np.int64)
    V = np.zeros((max(n - 1, 1), K), dtype=np.int64)
    for k in range(n - 1):
        V[k] = O.penalty_table(4 * int(rng.integers(0, 3)), K)
    return theta, V


@pytest.mark.parametrize("n,K", [(1, 3), (2, 2), (3, 3), (4, 3), (5, 2)])
def test_uniform_minorant_matches_exact_enumeration(n, K):
    rng = np.random.default_rng(n * 7 + K)
    for _ in range(4):
        theta, V = _chain(rng, n, K)
        lam, _ = O.uniform_minorant(theta, V)
        hist = B.uniform_minorant(theta.tolist(), V.tolist())
        fstar = B.chain_min(theta.tolist(), V.tolist())
        ref = np.zeros((n, K)) if not hist else np.array(
            [[float(v) for v in row] for row in hist[-1]])
        # the algorithm starts from lam = 0: its first round spreads f* evenly
        assert np.allclose(lam, ref + fstar / n, atol=1e-9)


@pytest.mark.parametrize("n,K", [(3, 3), (4, 3), (6, 2)])
def test_uniform_minorant_is_maximal_valid_and_above_m_over_n(n, K):
    rng = np.random.default_rng(n + 100 * K)
    for _ in range(4):
        theta, V = _chain(rng, n, K)
        lam, _ = O.uniform_minorant(theta, V)
        vals = {x: B.chain_energy(theta.tolist(), V.tolist(), x)
                for x in B.all_labellings(n, K)}
        for x, fx in vals.items():
            assert sum(lam[i, x[i]] for i in range(n)) <= fx + 1e-9
        mm_rem = np.full((n, K), np.inf)
        for x, fx in vals.items():
            r = fx - sum(lam[i, x[i]] for i in range(n))
            for i in range(n):
                mm_rem[i, x[i]] = min(mm_rem[i, x[i]], r)
        assert np.allclose(mm_rem, 0, atol=1e-8)                 # maximal
        m = np.array(B.min_marginals(theta.tolist(), V.tolist()), dtype=np.float64)
        assert np.all(lam >= m / n - 1e-9)                       # lambda >= m / n


def _grid(rng, H, W, K):
    cost = rng.integers(0, 10, size=(H, W, K)).astype(np.int32)
    wh = (rng.integers(0, 3, size=(H, W)) * 4).astype(np.int32)
    wv = (rng.integers(0, 3, size=(H, W)) * 4).astype(np.int32)
    wh[:, -1] = 0
    wv[-1, :] = 0
    return cost, wh, wv


def _tables(K):
    cache = {}

    def table_of(w):
        if w not in cache:
            cache[w] = O.penalty_table(w, K).tolist()
        return cache[w]
    return table_of


def test_primal_mm_majorant_is_above_and_exact():
    """For each family of chains the modular majorant is >= the family's energy
    at every labelling (enumeration) and equal at the labelling it is built at."""
    import itertools
    rng = np.random.default_rng(41)
    for trial in range(6):
        H, W, K = [(2, 3, 3), (3, 2, 3), (2, 2, 4)][trial % 3]
        cost, wh, wv = _grid(rng, H, W, K)
        at = rng.integers(0, K, size=(H, W)).astype(np.uint16)
        tab = _tables(K)
        for half in (0, 1):
            bar = O.pmm_majorant(cost, wh, wv, half, at)

            def family(lab):
                e = 0
                for y in range(H):
                    for x in range(W):
                        if half == 0:
                            e += int(cost[y, x, lab[y][x]])
                            if x + 1 < W:
                                e += tab(int(wh[y, x]))[abs(lab[y][x] - lab[y][x + 1])]
                        elif y + 1 < H:
                            e += tab(int(wv[y, x]))[abs(lab[y][x] - lab[y + 1][x])]
                return e
            for flat in itertools.product(range(K), repeat=H * W):
                lab = [flat[y * W:(y + 1) * W] for y in range(H)]
                m = sum(bar[y, x, lab[y][x]] for y in range(H) for x in range(W))
                assert m >= family(lab) - 1e-9
            m0 = sum(bar[y, x, at[y, x]] for y in range(H) for x in range(W))
            assert abs(m0 - family(at.tolist())) < 1e-9


def test_primal_mm_is_monotone_and_above_the_minimum():
    rng = np.random.default_rng(31)
    for trial in range(8):
        H, W, K = [(2, 3, 3), (3, 3, 2), (3, 4, 2), (2, 2, 3)][trial % 4]
        cost, wh, wv = _grid(rng, H, W, K)
        start = rng.integers(0, K, size=(H, W)).astype(np.uint16)
        e0 = O.discrete_energy(cost, wh, wv, start)
        labels, en = O.primal_mm(cost, wh, wv, 5, start)
        assert en[0] <= e0 and np.all(np.diff(en) <= 0)
        assert en[-1] == O.discrete_energy(cost, wh, wv, labels)
        assert en[-1] >= B.grid_min(cost, wh, wv, _tables(K))


def test_primal_mm_keeps_a_global_minimiser():
    import itertools
    rng = np.random.default_rng(5)
    H, W, K = 2, 3, 3
    cost, wh, wv = _grid(rng, H, W, K)
    best, arg = None, None
    for flat in itertools.product(range(K), repeat=H * W):
        lab = np.array(flat, dtype=np.uint16).reshape(H, W)
        e = O.discrete_energy(cost, wh, wv, lab)
        if best is None or e < best:
            best, arg = e, lab
    labels, en = O.primal_mm(cost, wh, wv, 3, arg)
    assert np.all(en == best)


def test_primal_mm_on_a_synthetic_frame_reaches_a_low_energy():
    """From the per-pixel argmin of the data cost, Primal_MM lowers the energy
    every iteration; Dual MM's labels on the same frame serve as a yardstick."""
    from paper_1601_06274_gb300 import synthetic as S
    sp = S.make_pair(16, 24, 8, planes=2, noise_sigma=2.0, seed=4)
    cost = O.cost_volume(sp.left, sp.right, 8)
    wh, wv = O.edge_weights(sp.left)
    start = cost.argmin(axis=2).astype(np.uint16)
    labels, en = O.primal_mm(cost, wh, wv, 6, start)
    assert np.all(np.diff(en) <= 0) and en[-1] < O.discrete_energy(cost, wh, wv, start)
    dl, lb, _, _ = O.dmm(cost, wh, wv, 6)
    assert lb[-1] <= en[-1]          # Dual MM's bound stays below every labelling's energy
