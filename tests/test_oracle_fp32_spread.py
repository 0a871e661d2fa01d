"""Pins of the oracle's float32 noise model of the refinement
(oracle.refine_perturbed, oracle.fp32_spread).

The model is the double-precision refinement (Sec. 2.4, Eq. cont_iterates)
with the state (u, p, q) multiplied by 1 + noise * U after every iteration, U
uniform in [-1, 1) from splitmix64 (Steele, Lea and Flood, OOPSLA 2014).  The
full-frame GPU check uses its spread as the part of the oracle's answer that
float32 does not determine, so the pins fix that the noise is exactly the
stated generator at the stated counter, that zero noise is the refinement
itself, and that the spread is small where the iteration settles at an
attracting fixed point.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_06274_gb300 import synthetic as S

from test_oracle_dc_split import CASES, _dmm_start

M64 = (1 << 64) - 1


def splitmix64(seed, n):
    """the n-th output (from 0) of splitmix64 started at state `seed`"""
    z = (seed + (n + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def unit(seed, n):
    return (splitmix64(seed, n) >> 11) * (2.0 / 2 ** 53) - 1.0


def test_splitmix64_restatement_gives_the_published_outputs():
    # the first three outputs of splitmix64 from state 0, as published with the
    # generator's reference implementation
    assert [splitmix64(0, n) for n in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_noise_is_the_stated_generator_at_the_stated_counter():
    """Zero cost, u = c everywhere, zero duals: one iteration leaves the state
    where it is (A u = 0, zero slopes: the data prox returns u0), so after it
    u = c (1 + noise U) with U at counter (0 * 5 + 0) * N + pixel."""
    H, W, L, c, noise, seed = 5, 7, 8, 3.0, 2.0 ** -10, 12345
    cost = np.zeros((H, W, L))
    w = np.full((H, W), 4.0)
    u = O.refine_perturbed(cost, w, w, np.full((H, W), c), 1, noise, seed, O.Params(warps=1))
    got = (u / c - 1.0) / noise
    want = np.array([unit(seed, p) for p in range(H * W)]).reshape(H, W)
    assert np.abs(got - want).max() <= 1e-9
    assert got.min() >= -1.0 and got.max() < 1.0


def test_zero_noise_is_the_refinement():
    sp = S.make_pair(24, 40, 32, planes=4, noise_sigma=2.0, seed=7)
    cost = O.cost_volume(sp.left, sp.right, 32).astype(float)
    wh, wv = O.edge_weights(sp.left)
    u0 = O.dmm(cost.astype(np.int32), wh, wv, 3)[0].astype(float)
    u = O.refine(cost, wh, wv, u0, 60)[0]
    assert np.array_equal(O.refine_perturbed(cost, wh, wv, u0, 60, 0.0, 3), u)
    a = O.refine_perturbed(cost, wh, wv, u0, 60, 2.0 ** -24, 3)
    assert np.array_equal(a, O.refine_perturbed(cost, wh, wv, u0, 60, 2.0 ** -24, 3))
    assert not np.array_equal(a, O.refine_perturbed(cost, wh, wv, u0, 60, 2.0 ** -24, 4))
    assert 0 < np.abs(a - u).max()


@pytest.mark.parametrize("seed,tau,sigma", CASES)
def test_spread_is_small_at_an_attracting_fixed_point(seed, tau, sigma):
    """Where the iteration reaches a fixed point (the critical-point cases of
    the DC split), float32-sized noise moves the result by little: a random
    walk of steps of about 2^-24 |u| along the directions the iteration does
    not contract."""
    cost, wh, wv, u0 = _dmm_start(seed)
    P = O.Params(warps=1, tau=tau, sigma=sigma)
    spread = O.fp32_spread(cost, wh, wv, u0, 3000, P, seeds=range(4))
    assert spread.max() <= 2e-4
