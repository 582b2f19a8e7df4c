"""Pins for the oracle's Table-1 gates and Trotter-Suzuki evolution: dense
Jordan-Wigner matrices with expm on tiny systems, the convergence order of
each product formula, exactness when the terms commute.  CPU only."""

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import bruteforce as bf
from paper_2605_03123_gb300 import inputs


@pytest.fixture(scope="module")
def fock3():
    return bf.FockSpace(3)


def _hermitian(n, g, s=1.0):
    A = g.normal(0, s, (n, n)) + 1j * g.normal(0, s, (n, n))
    return (A + A.conj().T) / 2


def _apply(fs, G, v, nelec):
    return fs.extract(G @ fs.embed(v, nelec), nelec)


SECTORS3 = [(1, 2), (2, 1), (2, 2), (1, 1), (3, 1)]


@pytest.mark.parametrize("nelec", SECTORS3)
def test_table1_gates_match_jordan_wigner(fock3, nelec):
    fs, N = fock3, 3
    g = inputs.rng(700 + 10 * nelec[0] + nelec[1])
    v = inputs.random_state(N, nelec, g)
    theta = 0.61
    n = lambda s, p: fs.number(s * N + p)
    hop = lambda s, p, q: fs.cdag[s * N + p] @ fs.c[s * N + q]
    for spins in [(0,), (1,), (0, 1)]:
        H = sum(n(s, 1) for s in spins)
        ref = _apply(fs, scipy.linalg.expm(1j * theta * H), v, nelec)
        assert np.max(np.abs(oracle.apply_num_interaction(v, theta, 1, spins, N, nelec) - ref)) < 1e-12
        for p, q in [(0, 2), (2, 0), (1, 2)]:
            H = sum(hop(s, p, q) - hop(s, q, p) for s in spins)
            ref = _apply(fs, scipy.linalg.expm(theta * H), v, nelec)
            got = oracle.apply_givens_rotation(v, theta, p, q, spins, N, nelec)
            assert np.max(np.abs(got - ref)) < 1e-12
            H = sum(hop(s, p, q) + hop(s, q, p) for s in spins)
            ref = _apply(fs, scipy.linalg.expm(1j * theta * H), v, nelec)
            got = oracle.apply_tunneling_interaction(v, theta, p, q, spins, N, nelec)
            assert np.max(np.abs(got - ref)) < 1e-12
    for p, sigma, q, tau in [(0, 0, 2, 0), (1, 1, 1, 1), (0, 0, 2, 1), (2, 1, 0, 0), (1, 0, 1, 1)]:
        H = n(sigma, p) @ n(tau, q)
        ref = _apply(fs, scipy.linalg.expm(1j * theta * H), v, nelec)
        got = oracle.apply_num_num_interaction(v, theta, p, sigma, q, tau, N, nelec)
        assert np.max(np.abs(got - ref)) < 1e-12
    Ma, Mb = _hermitian(N, g), _hermitian(N, g)
    ref = _apply(fs, scipy.linalg.expm(-0.8j * fs.one_body(Ma, Mb)), v, nelec)
    got = oracle.apply_quad_ham_evolution(v, Ma, Mb, 0.8, N, nelec)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_product_formula_structure():
    """Each term's times add up to t; S_1 is a palindrome; S_2 has 5 copies
    of S_1 with u_2 = 1/(4 - 4^(1/3))."""
    for L in (1, 2, 4):
        for order in range(4):
            seq = oracle.product_formula(L, 0.9, order)
            for j in range(L):
                assert abs(sum(t for k, t in seq if k == j) - 0.9) < 1e-14
            if order >= 1:
                assert seq == seq[::-1]
    s2 = oracle.product_formula(3, 1.0, 2)
    u = 1 / (4 - 4 ** (1 / 3))
    assert len(s2) == 5 * 6 and abs(s2[0][1] - u / 2) < 1e-15
    assert abs(s2[12][1] - (1 - 4 * u) / 2) < 1e-15


def _dc_hamiltonian(fs, h, J_aa, J_ab, J_bb):
    N = fs.norb
    H = fs.one_body(h).astype(complex)
    blocks = {(0, 0): J_aa, (0, 1): J_ab, (1, 0): J_ab.T, (1, 1): J_bb}
    for (s, u), J in blocks.items():
        for p in range(N):
            for q in range(N):
                H = H + 0.5 * J[p, q] * (fs.number(s * N + p) @ fs.number(u * N + q))
    return H


def _df_hamiltonian(fs, h, Js, Us):
    N = fs.norb
    H = fs.one_body(h).astype(complex)
    for J, U in zip(Js, Us):
        # n^(t)_{p sigma} = sum_ij U_ip conj(U_jp) a^dag_{i sigma} a_{j sigma}
        nt = [fs.one_body(np.outer(U[:, p], U[:, p].conj()), np.zeros((N, N)))
              for p in range(N)]
        nt += [fs.one_body(np.zeros((N, N)), np.outer(U[:, p], U[:, p].conj()))
               for p in range(N)]
        for p in range(N):
            for q in range(N):
                for s in (0, 1):
                    for u in (0, 1):
                        H = H + 0.5 * J[p, q] * (nt[s * N + p] @ nt[u * N + q])
    return H


def _order_estimate(errs):
    return np.log2(errs[0] / errs[1])


@pytest.mark.parametrize("nelec", [(1, 2), (2, 2)])
def test_trotter_diag_coulomb_converges_at_each_order(fock3, nelec):
    """||S_k(T/r)^r psi - exp(-iHT) psi|| falls as r^-p with p = 1, 2, 4 for
    orders 0, 1, 2 (the S_k definition); order 2 at r = 16 is near exact."""
    fs, N = fock3, 3
    g = inputs.rng(720 + nelec[0])
    h = _hermitian(N, g, 0.6)
    J_aa, J_ab, J_bb = (inputs.random_symmetric(N, 0.7, g) for _ in range(3))
    v = inputs.random_state(N, nelec, g)
    T = 0.8
    exact = _apply(fs, scipy.linalg.expm(-1j * T * _dc_hamiltonian(fs, h, J_aa, J_ab, J_bb)),
                   v, nelec)
    for order, p in [(0, 1), (1, 2), (2, 4)]:
        errs = [np.linalg.norm(oracle.simulate_trotter_diag_coulomb(
            v, h, J_aa, J_ab, J_bb, T, N, nelec, r, order) - exact) for r in (4, 8)]
        assert abs(_order_estimate(errs) - p) < 0.35, (order, errs)
    e = np.linalg.norm(oracle.simulate_trotter_diag_coulomb(v, h, J_aa, J_ab, J_bb, T, N, nelec,
                                                            16, 2) - exact)
    assert e < 1e-7


@pytest.mark.parametrize("nelec", [(1, 2), (2, 1)])
def test_trotter_double_factorized_converges_at_each_order(fock3, nelec):
    fs, N = fock3, 3
    g = inputs.rng(740 + nelec[0])
    h = _hermitian(N, g, 0.6)
    Js = [inputs.random_symmetric(N, 0.7, g) for _ in range(2)]
    Us = [inputs.haar_unitary(N, g) for _ in range(2)]
    v = inputs.random_state(N, nelec, g)
    T = 0.7
    exact = _apply(fs, scipy.linalg.expm(-1j * T * _df_hamiltonian(fs, h, Js, Us)), v, nelec)
    for order, p in [(0, 1), (1, 2), (2, 4)]:
        errs = [np.linalg.norm(oracle.simulate_trotter_double_factorized(
            v, h, Js, Us, T, N, nelec, r, order) - exact) for r in (4, 8)]
        assert abs(_order_estimate(errs) - p) < 0.35, (order, errs)


def test_trotter_exact_when_terms_commute(fock3):
    """A diagonal one-body term commutes with the diagonal-Coulomb term: every
    order is exact at one step."""
    fs, N, nelec = fock3, 3, (2, 1)
    g = inputs.rng(760)
    h = np.diag(g.normal(0, 1, N)).astype(complex)
    J_aa, J_ab = inputs.random_symmetric(N, 0.7, g), inputs.random_symmetric(N, 0.7, g)
    v = inputs.random_state(N, nelec, g)
    exact = _apply(fs, scipy.linalg.expm(-1.3j * _dc_hamiltonian(fs, h, J_aa, J_ab, J_aa)), v,
                   nelec)
    for order in range(3):
        got = oracle.simulate_trotter_diag_coulomb(v, h, J_aa, J_ab, None, 1.3, N, nelec, 1, order)
        assert np.max(np.abs(got - exact)) < 1e-12


def test_convergence_pin_catches_planted_mistakes(fock3, monkeypatch):
    """The order test above fails for a wrong u_k, for an S_1 whose second
    half is not reversed, and for a DF term applied as U^dag DC U."""
    import oracle.trotter as ot
    fs, N, nelec = fock3, 3, (1, 2)
    g = inputs.rng(780)
    h = _hermitian(N, g, 0.6)
    J_aa, J_ab, J_bb = (inputs.random_symmetric(N, 0.7, g) for _ in range(3))
    v = inputs.random_state(N, nelec, g)
    T = 0.8
    exact = _apply(fs, scipy.linalg.expm(-1j * T * _dc_hamiltonian(fs, h, J_aa, J_ab, J_bb)),
                   v, nelec)
    good = ot.product_formula

    def order_of(order):
        errs = [np.linalg.norm(ot.simulate_trotter_diag_coulomb(
            v, h, J_aa, J_ab, J_bb, T, N, nelec, r, order) - exact) for r in (4, 8)]
        return _order_estimate(errs)

    def wrong_u(L, t, order):
        if order < 2:
            return good(L, t, order)
        u = 1.0 / (4.0 - 4.0 ** (1.0 / (2 * order)))
        outer, inner = wrong_u(L, u * t, order - 1), wrong_u(L, (1 - 4 * u) * t, order - 1)
        return outer + outer + inner + outer + outer

    def unreversed(L, t, order):
        if order == 1:
            return [(j, t / 2) for j in range(L)] * 2
        return good(L, t, order)

    monkeypatch.setattr(ot, "product_formula", wrong_u)
    assert abs(order_of(2) - 4) > 0.35
    monkeypatch.setattr(ot, "product_formula", unreversed)
    assert abs(order_of(1) - 2) > 0.35
    monkeypatch.setattr(ot, "product_formula", good)
    # DF term with the rotation on the wrong side
    Js = [inputs.random_symmetric(N, 0.7, g)]
    Us = [inputs.haar_unitary(N, g)]
    exact_df = _apply(fs, scipy.linalg.expm(-1j * T * _df_hamiltonian(fs, h, Js, Us)), v, nelec)
    swapped = [U.conj().T for U in Us]
    err = np.linalg.norm(ot.simulate_trotter_double_factorized(v, h, Js, swapped, T, N, nelec, 16,
                                                               2) - exact_df)
    assert err > 1e-3
