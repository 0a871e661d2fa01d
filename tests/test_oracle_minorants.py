"""Pins of the oracle's other chain minorants (Sec. 2.3 "Good and Fast
Minorants", App. A): the naive minorant (min-marginals divided by the chain
length) and the iterative minorant (Alg. iterative-minorant).

* The naive minorant against min-marginals by enumeration.
* The iterative minorant against a restatement that recomputes, at every node
  visit, the min-marginals of the remainder from scratch (by enumeration, or by
  the oracle's own min-marginal routine on longer chains), so that the oracle's
  reuse of messages between passes is checked against the plain definition.
* Validity (lambda(x) <= f(x) for every labelling) of both; maximality (all
  min-marginals of f - lambda vanish) after a last pass with gamma = 1.
* Dual MM with either minorant: the lower bound stays below the grid minimum.
"""

import itertools

import numpy as np
import pytest

import bruteforce as B
from oracle import oracle as O


def _random_chain(rng, n, K, lo=-4, hi=12):
    theta = rng.integers(lo, hi, size=(n, K)).astype(np.int64)
    V = np.zeros((max(n - 1, 1), K), dtype=np.int64)
    for k in range(n - 1):
        V[k] = O.penalty_table(4 * int(rng.integers(0, 3)), K)
    return theta, V


def _chain_values(theta, V):
    n, K = theta.shape
    return {x: B.chain_energy(theta.tolist(), V.tolist(), x) for x in B.all_labellings(n, K)}


def _valid(theta, V, lam):
    n = theta.shape[0]
    for x, fx in _chain_values(theta, V).items():
        if sum(int(lam[i, x[i]]) for i in range(n)) > fx:
            return False
    return True


def _mm_enum(theta, V):
    return np.array(B.min_marginals(theta.tolist(), V.tolist()), dtype=np.int64)


def _iterative_by_definition(theta, V, max_pass, gamma, mm_of):
    n, K = theta.shape
    lam = np.zeros((n, K), dtype=np.int64)
    for s in range(1, max_pass + 1):
        num, den = (1, 1) if s == max_pass else gamma
        order = range(n) if s % 2 == 1 else range(n - 1, -1, -1)
        for i in order:
            mm = mm_of(theta - lam, V)            # min-marginals of the remainder f - lam
            lam[i] += (mm[i] * num) // den        # floor(gamma m_i)
    return lam


# --- naive -------------------------------------------------------------------------

@pytest.mark.parametrize("n,K", [(1, 3), (2, 2), (3, 3), (4, 2), (5, 3)])
def test_naive_is_min_marginals_over_n(n, K):
    rng = np.random.default_rng(n * 10 + K)
    for _ in range(4):
        theta, V = _random_chain(rng, n, K)
        lam = O.naive_minorant(theta, V)
        mm = _mm_enum(theta, V)
        assert np.array_equal(lam, mm // n)       # floor division, negatives included
        assert _valid(theta, V, lam)


def test_naive_single_node_keeps_its_unary():
    theta = np.array([[3, -2, 7]], np.int64)
    assert np.array_equal(O.naive_minorant(theta, np.zeros((1, 3), np.int64)), theta)


# --- iterative ---------------------------------------------------------------------

@pytest.mark.parametrize("max_pass,gamma", [(1, (1, 4)), (2, (1, 4)), (3, (1, 4)), (3, (1, 2)),
                                            (4, (3, 4))])
@pytest.mark.parametrize("n,K", [(1, 3), (2, 3), (4, 2), (5, 3)])
def test_iterative_matches_its_definition_by_enumeration(max_pass, gamma, n, K):
    rng = np.random.default_rng(max_pass * 100 + n * 10 + K)
    for _ in range(3):
        theta, V = _random_chain(rng, n, K)
        lam = O.iterative_minorant(theta, V, max_pass, gamma)
        ref = _iterative_by_definition(theta, V, max_pass, gamma, _mm_enum)
        assert np.array_equal(lam, ref)


@pytest.mark.parametrize("n,K", [(12, 5), (20, 8)])
def test_iterative_matches_its_definition_on_longer_chains(n, K):
    rng = np.random.default_rng(n + K)
    theta, V = _random_chain(rng, n, K, -20, 40)
    lam = O.iterative_minorant(theta, V, 3, (1, 4))
    ref = _iterative_by_definition(theta, V, 3, (1, 4), O.min_marginals)
    assert np.array_equal(lam, ref)


@pytest.mark.parametrize("max_pass,gamma", [(1, (1, 4)), (3, (1, 4)), (2, (1, 2))])
def test_iterative_is_valid_and_maximal(max_pass, gamma):
    """gamma = 1 on the last pass drains every min-marginal of the remainder."""
    rng = np.random.default_rng(max_pass)
    for n, K in [(3, 3), (4, 3), (5, 2), (6, 2)]:
        theta, V = _random_chain(rng, n, K)
        lam = O.iterative_minorant(theta, V, max_pass, gamma)
        assert _valid(theta, V, lam)
        assert np.all(_mm_enum(theta - lam, V) == 0)


def test_iterative_early_passes_leave_slack():
    """With max_pass = 2 the first pass drains a quarter only: the minorant
    differs from the one-pass (gamma = 1) minorant, and both are maximal."""
    rng = np.random.default_rng(3)
    theta, V = _random_chain(rng, 5, 3, 0, 30)
    one = O.iterative_minorant(theta, V, 1, (1, 4))
    two = O.iterative_minorant(theta, V, 2, (1, 4))
    assert not np.array_equal(one, two)
    for lam in (one, two):
        assert _valid(theta, V, lam) and np.all(_mm_enum(theta - lam, V) == 0)


def test_iterative_rejects_bad_arguments():
    theta = np.zeros((3, 2), np.int64)
    V = np.zeros((2, 2), np.int64)
    for mp, g in [(0, (1, 4)), (3, (5, 4)), (3, (1, 0)), (3, (-1, 4))]:
        with pytest.raises(RuntimeError):
            O.iterative_minorant(theta, V, mp, g)


# --- Dual MM with the other minorants ------------------------------------------------

def _tables(K):
    cache = {}

    def table_of(w):
        if w not in cache:
            cache[w] = O.penalty_table(w, K).tolist()
        return cache[w]
    return table_of


@pytest.mark.parametrize("minorant", ["naive", "iterative"])
def test_dmm_weak_duality_with_other_minorants(minorant):
    rng = np.random.default_rng(17)
    for trial in range(8):
        H, W, K = [(2, 3, 3), (3, 3, 2), (3, 4, 2), (2, 2, 3)][trial % 4]
        cost = rng.integers(0, 10, size=(H, W, K)).astype(np.int32)
        wh = (rng.integers(0, 3, size=(H, W)) * 4).astype(np.int32)
        wv = (rng.integers(0, 3, size=(H, W)) * 4).astype(np.int32)
        wh[:, -1] = 0
        wv[-1, :] = 0
        labels, lb, lam_h, lam_v = O.dmm(cost, wh, wv, 4, minorant=minorant)
        emin = B.grid_min(cost, wh, wv, _tables(K))
        assert np.all(lb <= emin)
        assert emin <= O.discrete_energy(cost, wh, wv, labels)


@pytest.mark.parametrize("minorant", ["naive", "iterative"])
def test_dmm_pass_uses_the_chosen_minorant_per_chain(minorant):
    """One horizontal pass: every row's lam_h + lam_v is the chosen minorant of
    that row's chain with unaries c + lam_v."""
    rng = np.random.default_rng(23)
    H, W, K = 3, 7, 4
    cost = rng.integers(0, 12, size=(H, W, K)).astype(np.int32)
    wh = (rng.integers(1, 3, size=(H, W)) * 4).astype(np.int32)
    wv = (rng.integers(1, 3, size=(H, W)) * 4).astype(np.int32)
    wh[:, -1] = 0
    wv[-1, :] = 0
    lam_v = rng.integers(-5, 5, size=(H, W, K)).astype(np.int64)
    lam_h = O.dmm_pass(cost, wh, wv, 0, lam_v, minorant=minorant)
    for y in range(H):
        theta = cost[y].astype(np.int64) + lam_v[y]
        V = np.stack([O.penalty_table(int(wh[y, x]), K) for x in range(W - 1)])
        ref = O.naive_minorant(theta, V) if minorant == "naive" else O.iterative_minorant(theta, V)
        assert np.array_equal(lam_h[y] + lam_v[y], ref)
