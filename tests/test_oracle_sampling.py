"""Pins for the oracle's samplers: the chain rule reproduces |det|^2
exactly (summed over pick orders), sample frequencies match the exact
distributions, and the inverse CDF agrees with a direct scan.  CPU only."""

import itertools
import math

import numpy as np

import oracle
from paper_2605_03123_gb300 import inputs


def test_chain_rule_sums_to_determinant_probability():
    g = inputs.rng(1400)
    N, occ = 5, [0, 2, 3]
    U = inputs.haar_unitary(N, g)
    total = 0.0
    for I in itertools.combinations(range(N), len(occ)):
        p = sum(oracle.chain_rule_probability(U, occ, order) for order in itertools.permutations(I))
        exact = abs(np.linalg.det(U[np.ix_(I, occ)])) ** 2
        assert abs(p - exact) < 1e-12
        total += p
    assert abs(total - 1) < 1e-12


def test_slater_sample_frequencies_match_determinants():
    g = inputs.rng(1410)
    N, occ = 5, [1, 3]
    U = inputs.haar_unitary(N, g)
    shots = 40000
    masks = oracle.sample_slater_spin(U, occ, g.random((shots, len(occ))))
    tv = 0.0
    for I in itertools.combinations(range(N), len(occ)):
        m = sum(1 << p for p in I)
        exact = abs(np.linalg.det(U[np.ix_(I, occ)])) ** 2
        tv += abs(np.mean(masks == m) - exact)
    assert 0.5 * tv < 0.012
    assert all(bin(int(m)).count("1") == len(occ) for m in masks)


def test_state_sampler_is_inverse_cdf():
    g = inputs.rng(1420)
    v = inputs.random_state(4, (2, 1), g)
    p = np.abs(v.ravel()) ** 2
    u = g.random(2000)
    got = oracle.sample_state(v, u)
    for uk, k in zip(u, got):
        below = p[:k].sum()
        assert below <= uk <= below + p[k] + 1e-15
    freq = np.bincount(oracle.sample_state(v, g.random(60000)), minlength=p.size) / 60000
    assert 0.5 * np.abs(freq - p).sum() < 0.02


def test_slater_samples_match_state_amplitudes():
    """The closed form of §2.4 ties the two samplers: a Slater state's
    amplitudes are determinants, so each configuration's frequency under
    the Slater sampler matches |psi|^2 of the explicit state."""
    g = inputs.rng(1430)
    N, nelec = 4, (2, 1)
    Ua, Ub = inputs.haar_unitary(N, g), inputs.haar_unitary(N, g)
    psi = oracle.slater_from_hf(Ua, Ub, N, nelec)
    shots = 30000
    ma = oracle.sample_slater_spin(Ua, [0, 1], g.random((shots, 2)))
    mb = oracle.sample_slater_spin(Ub, [0], g.random((shots, 1)))
    sa, sb = oracle.strings(N, 2), oracle.strings(N, 1)
    ia = {int(m): k for k, m in enumerate(sa)}
    ib = {int(m): k for k, m in enumerate(sb)}
    freq = np.zeros((len(sa), len(sb)))
    for a, b in zip(ma, mb):
        freq[ia[int(a)], ib[int(b)]] += 1 / shots
    assert 0.5 * np.abs(freq - np.abs(psi) ** 2).sum() < 0.02
    assert math.isclose(np.sum(np.abs(psi) ** 2), 1.0, rel_tol=1e-12)
