"""Independent brute-force references used to pin the oracle (pure Python).

Everything here is written from the mathematical definitions with explicit
enumeration, so it shares nothing with the oracle's dynamic programming.
Only small inputs are feasible.
"""

from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def chain_energy(theta, V, x):
    """f(x) = sum_k theta_k(x_k) + sum_k V_k(|x_k - x_{k+1}|)."""
    e = 0
    for k in range(len(x)):
        e += theta[k][x[k]]
    for k in range(len(x) - 1):
        e += V[k][abs(x[k] - x[k + 1])]
    return e


def chain_pair_energy(theta, F, x):
    """Same with full pairwise matrices F[k][a][b]."""
    e = sum(theta[k][x[k]] for k in range(len(x)))
    e += sum(F[k][x[k]][x[k + 1]] for k in range(len(x) - 1))
    return e


def all_labellings(n, K):
    return itertools.product(range(K), repeat=n)


def min_marginals(theta, V):
    """m_i(l) = min over labellings with x_i = l of f(x), by enumeration."""
    n, K = len(theta), len(theta[0])
    mm = [[None] * K for _ in range(n)]
    for x in all_labellings(n, K):
        e = chain_energy(theta, V, x)
        for i in range(n):
            if mm[i][x[i]] is None or e < mm[i][x[i]]:
                mm[i][x[i]] = e
    return mm


def chain_min(theta, V):
    return min(chain_energy(theta, V, x) for x in all_labellings(len(theta), len(theta[0])))


def uniform_minorant(theta, V):
    """Alg. A:uniform-minorant on the chain normalised by its minimum f*.

    The maximisation of epsilon is done by enumerating labellings (exact, in
    rationals) instead of Lawler's minimum-ratio cycle.  Returns the list of
    minorants after each iteration.
    """
    n, K = len(theta), len(theta[0])
    labs = list(all_labellings(n, K))
    fvals = {x: Fraction(chain_energy(theta, V, x)) for x in labs}
    fstar = min(fvals.values())
    lam = [[Fraction(0)] * K for _ in range(n)]
    history = []
    for _ in range(64):
        rem = {x: fvals[x] - fstar - sum(lam[i][x[i]] for i in range(n)) for x in labs}
        mm = [[min(rem[x] for x in labs if x[i] == l) for l in range(K)] for i in range(n)]
        if all(mm[i][l] == 0 for i in range(n) for l in range(K)):
            break
        O = [[1 if mm[i][l] == 0 else 0 for l in range(K)] for i in range(n)]
        best = None
        for x in labs:
            cnt = sum(1 - O[i][x[i]] for i in range(n))
            if cnt > 0:
                r = rem[x] / cnt
                best = r if best is None or r < best else best
        lam = [[lam[i][l] + best * (1 - O[i][l]) for l in range(K)] for i in range(n)]
        history.append([row[:] for row in lam])
    return history


def viterbi_min(theta, V):
    """Minimum chain energy by a plain forward recursion over full tables."""
    n, K = len(theta), len(theta[0])
    best = [theta[0][l] for l in range(K)]
    for k in range(1, n):
        best = [min(best[a] + V[k - 1][abs(a - b)] for a in range(K)) + theta[k][b]
                for b in range(K)]
    return min(best)


def grid_energy(cost, wh, wv, table_of, labels):
    H, W, _ = cost.shape
    e = 0
    for y in range(H):
        for x in range(W):
            e += int(cost[y, x, labels[y][x]])
            if x + 1 < W:
                e += int(table_of(int(wh[y, x]))[abs(labels[y][x] - labels[y][x + 1])])
            if y + 1 < H:
                e += int(table_of(int(wv[y, x]))[abs(labels[y][x] - labels[y + 1][x])])
    return e


def grid_min(cost, wh, wv, table_of):
    H, W, K = cost.shape
    best = None
    for flat in itertools.product(range(K), repeat=H * W):
        labels = [flat[y * W:(y + 1) * W] for y in range(H)]
        e = grid_energy(cost, wh, wv, table_of, labels)
        best = e if best is None or e < best else best
    return best


def census_ref(img, win):
    """Census transform written directly from its definition (pure Python)."""
    H, W = img.shape
    r = win // 2
    out = np.zeros((H, W), dtype=np.uint32)
    for y in range(H):
        for x in range(W):
            code, bit = 0, 0
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    if dy == 0 and dx == 0:
                        continue
                    yy = min(max(y + dy, 0), H - 1)
                    xx = min(max(x + dx, 0), W - 1)
                    if int(img[yy, xx]) < int(img[y, x]):
                        code |= 1 << bit
                    bit += 1
            out[y, x] = code
    return out


def hamming(a: int, b: int) -> int:
    return bin(int(a) ^ int(b)).count("1")


def read_golden(path):
    """Parse a sectioned text fixture: '[name]' headers, rows of numbers."""
    out, cur = {}, None
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                out[cur] = []
                continue
            out[cur].append([Fraction(t) for t in line.split()])
    return out


def _left_message(theta, V, a, i, Lin, K):
    """phi_{i-1,i}(x_i): min over x_a..x_{i-1} of the sub-chain a..i-1 energy,
    the boundary message Lin at a and the edge (i-1, i), by enumeration."""
    out = []
    for xi in range(K):
        best = None
        for xs in itertools.product(range(K), repeat=i - a):
            x = list(xs) + [xi]
            e = Lin[x[0]]
            for k in range(i - a):
                e += theta[a + k][x[k]] + V[a + k][abs(x[k] - x[k + 1])]
            best = e if best is None or e < best else best
        out.append(best)
    return out


def _right_message(theta, V, j, b, Rin, K):
    """phi_{j+1,j}(x_j) by enumeration of x_{j+1}..x_b (mirror of _left_message)."""
    out = []
    for xj in range(K):
        best = None
        for xs in itertools.product(range(K), repeat=b - j):
            x = [xj] + list(xs)
            e = Rin[x[-1]]
            for k in range(1, b - j + 1):
                e += theta[j + k][x[k]] + V[j + k - 1][abs(x[k - 1] - x[k])]
            best = e if best is None or e < best else best
        out.append(best)
    return out


def hier_minorant_enum(theta, V):
    """Hierarchical minorant (App. A) with every min-marginal message obtained by
    enumeration from its definition instead of dynamic programming.  Split rule
    and rounding follow the readings: the left part keeps ceil(n/2) nodes and
    the Handshake shares floor(m_i/2) - phi_ji."""
    n, K = len(theta), len(theta[0])
    lam = [[0] * K for _ in range(n)]

    def msg(a, table):
        return [min(a[x] + table[abs(x - xp)] for x in range(K)) for xp in range(K)]

    def rec(a, b, Lin, Rin):
        if a == b:
            lam[a] = [theta[a][l] + Lin[l] + Rin[l] for l in range(K)]
            return
        i = a + (b - a + 2) // 2 - 1
        j = i + 1
        Lm = _left_message(theta, V, a, i, Lin, K) if i > a else list(Lin)
        Rm = _right_message(theta, V, j, b, Rin, K) if b > j else list(Rin)
        phi_ji = msg([theta[j][l] + Rm[l] for l in range(K)], V[i])
        m_i = [Lm[l] + theta[i][l] + phi_ji[l] for l in range(K)]
        phi_ij = msg([m_i[l] // 2 - phi_ji[l] for l in range(K)], V[i])
        phi_ji = msg([-phi_ij[l] for l in range(K)], V[i])
        rec(a, i, Lin, phi_ji)
        rec(j, b, phi_ij, Rin)

    rec(0, n - 1, [0] * K, [0] * K)
    return lam
