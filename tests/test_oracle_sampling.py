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


def _check_slater_frequencies(sampler, U, occ, g, shots=40000):
    """Pin: every sample has len(occ) orbitals and the sample frequencies
    match |det U[I, occ]|^2 (total variation below 0.012)."""
    N = U.shape[0]
    masks = sampler(U, occ, g.random((shots, len(occ))))
    assert all(bin(int(m)).count("1") == len(occ) for m in masks)
    tv = 0.0
    for I in itertools.combinations(range(N), len(occ)):
        m = sum(1 << p for p in I)
        exact = abs(np.linalg.det(U[np.ix_(I, occ)])) ** 2
        tv += abs(np.mean(masks == m) - exact)
    assert 0.5 * tv < 0.012


def _check_inverse_cdf(sampler, v, g):
    """Pin: on an unnormalised state with zero amplitudes, every sample k
    has p_k > 0 and sum_{k' < k} p_k' <= u ||v||^2 <= sum_{k' <= k} p_k'
    (u = 0 included), and frequencies match |v|^2 / ||v||^2."""
    p = np.abs(v.ravel()) ** 2
    tot = p.sum()
    u = np.concatenate([[0.0], g.random(2000)])
    got = sampler(v, u)
    for uk, k in zip(u, got):
        below = p[:k].sum()
        assert p[k] > 0
        assert below <= uk * tot * (1 + 1e-12) and uk * tot <= (below + p[k]) * (1 + 1e-12)
    freq = np.bincount(sampler(v, g.random(60000)), minlength=p.size) / 60000
    assert 0.5 * np.abs(freq - p / tot).sum() < 0.02


def _sparse_unnormalised(g):
    v = 3.7 * inputs.random_state(4, (2, 1), g)
    v.reshape(-1)[[0, 1, 5]] = 0
    return v


def test_slater_sample_frequencies_match_determinants():
    g = inputs.rng(1410)
    U = inputs.haar_unitary(5, g)
    _check_slater_frequencies(oracle.sample_slater_spin, U, [1, 3], g)


def test_state_sampler_is_inverse_cdf():
    g = inputs.rng(1420)
    _check_inverse_cdf(oracle.sample_state, _sparse_unnormalised(g), g)


def test_sampling_pins_catch_planted_mistakes():
    """Plausible mistakes planted in copies of the samplers each fail a pin:
    the uniform not scaled by the total, |v| in place of |v|^2, ties sent to
    the left (a zero-probability configuration for u = 0), no projection
    after a pick, rows in place of columns, an unnormalised projection."""
    import pytest

    def state_with(prob, scale_total, side):
        def sampler(vec, uniforms):
            pp = prob(np.asarray(vec, dtype=complex).ravel())
            c = np.cumsum(pp)
            x = np.asarray(uniforms) * (c[-1] if scale_total else 1.0)
            return np.minimum(np.searchsorted(c, x, side=side), len(c) - 1)
        return sampler

    sq = lambda z: np.abs(z) ** 2
    for bad in (state_with(sq, False, "right"), state_with(np.abs, True, "right"),
                state_with(sq, True, "left")):
        g = inputs.rng(1420)
        with pytest.raises(AssertionError):
            _check_inverse_cdf(bad, _sparse_unnormalised(g), g)

    def slater_with(project, columns, normalise):
        def sampler(U, occ, uniforms):
            out = []
            for us in np.atleast_2d(uniforms):
                V = (U[:, occ] if columns else U[occ, :].T).copy()
                mask = 0
                for i in range(len(occ)):
                    w = np.sum(np.abs(V) ** 2, axis=1)
                    c = np.cumsum(w)
                    p = min(int(np.searchsorted(c, us[i] * c[-1], side="right")), len(c) - 1)
                    mask |= 1 << p
                    if project:
                        e = V[p] / (np.linalg.norm(V[p]) if normalise else 1.0)
                        V = V - np.outer(V @ e.conj(), e)
                out.append(mask)
            return np.array(out, dtype=object)
        return sampler

    for bad in (slater_with(False, True, True), slater_with(True, False, True),
                slater_with(True, True, False)):
        g = inputs.rng(1410)
        U = inputs.haar_unitary(5, g)
        with pytest.raises(AssertionError):
            _check_slater_frequencies(bad, U, [1, 3], g, shots=20000)
    # the faithful copy passes the same pins
    g = inputs.rng(1410)
    U = inputs.haar_unitary(5, g)
    _check_slater_frequencies(slater_with(True, True, True), U, [1, 3], g, shots=20000)
    g = inputs.rng(1420)
    _check_inverse_cdf(state_with(sq, True, "right"), _sparse_unnormalised(g), g)


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
