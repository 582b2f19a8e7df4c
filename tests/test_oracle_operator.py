"""Pins for the oracle's molecular-Hamiltonian action: dense Jordan-Wigner
matrices on tiny systems, and the time derivative of the (independently
written) quadratic-Hamiltonian evolution.  CPU only."""

import numpy as np
import pytest

import oracle
from oracle import bruteforce as bf
from paper_2605_03123_gb300 import inputs


@pytest.fixture(scope="module")
def fock3():
    return bf.FockSpace(3)


def _tensors(N, g, complex_=False):
    h1 = g.normal(0, 1, (N, N)) + (1j * g.normal(0, 1, (N, N)) if complex_ else 0)
    h2 = g.normal(0, 1, (N, N, N, N)) + (1j * g.normal(0, 1, (N, N, N, N)) if complex_ else 0)
    return h1, h2


def _dense(fs, h1, h2, const):
    N = fs.norb
    dim = 1 << (2 * N)
    H = const * np.eye(dim, dtype=complex)
    cd, c = fs.cdag, fs.c
    for s in (0, 1):
        for p in range(N):
            for q in range(N):
                H = H + h1[p, q] * (cd[s * N + p] @ c[s * N + q])
    for s in (0, 1):
        for t in (0, 1):
            for p in range(N):
                for q in range(N):
                    for r in range(N):
                        for u in range(N):
                            if h2[p, q, r, u] == 0:
                                continue
                            H = H + 0.5 * h2[p, q, r, u] * (
                                cd[s * N + p] @ cd[t * N + r] @ c[t * N + u] @ c[s * N + q])
    return H


@pytest.mark.parametrize("nelec", [(1, 2), (2, 2), (3, 1), (2, 0)])
@pytest.mark.parametrize("complex_", [False, True])
def test_molecular_hamiltonian_matches_jordan_wigner(fock3, nelec, complex_):
    fs, N = fock3, 3
    g = inputs.rng(1100 + 10 * nelec[0] + nelec[1] + 100 * complex_)
    h1, h2 = _tensors(N, g, complex_)
    v = inputs.random_state(N, nelec, g)
    ref = fs.extract(_dense(fs, h1, h2, 0.3) @ fs.embed(v, nelec), nelec)
    got = oracle.apply_molecular_hamiltonian(v, h1, h2, N, nelec, constant=0.3)
    assert np.max(np.abs(got - ref)) < 1e-11


def test_one_body_part_is_derivative_of_quadratic_evolution():
    """With h_pqrs = 0, H psi = i d/dt exp(-i h t) psi at t = 0 (Table 1's
    quadratic-Hamiltonian evolution, a separate oracle routine)."""
    N, nelec = 5, (2, 3)
    g = inputs.rng(1150)
    A = g.normal(0, 1, (N, N)) + 1j * g.normal(0, 1, (N, N))
    h = (A + A.conj().T) / 2
    v = inputs.random_state(N, nelec, g)
    eps = 1e-5
    fd = 1j * (oracle.apply_quad_ham_evolution(v, h, None, eps, N, nelec)
               - oracle.apply_quad_ham_evolution(v, h, None, -eps, N, nelec)) / (2 * eps)
    got = oracle.apply_molecular_hamiltonian(v, h, np.zeros((N, N, N, N)), N, nelec)
    assert np.max(np.abs(got - fd)) < 1e-8


def test_hermitian_tensors_give_a_hermitian_operator():
    N, nelec = 4, (2, 2)
    g = inputs.rng(1160)
    A = g.normal(0, 1, (N, N))
    h1 = A + A.T
    B = g.normal(0, 1, (N, N, N, N))
    h2 = B + B.transpose(1, 0, 3, 2) + B.transpose(2, 3, 0, 1) + B.transpose(3, 2, 1, 0)
    u, w = inputs.random_state(N, nelec, g), inputs.random_state(N, nelec, g)
    lhs = np.vdot(u, oracle.apply_molecular_hamiltonian(w, h1, h2, N, nelec))
    rhs = np.vdot(oracle.apply_molecular_hamiltonian(u, h1, h2, N, nelec), w)
    assert abs(lhs - rhs) < 1e-11


def test_jordan_wigner_pin_catches_planted_mistakes(fock3, monkeypatch):
    """Mistakes planted in the oracle's operator strings fail the dense
    Jordan-Wigner pin: the fermionic signs dropped, and the two annihilators
    of the two-body term applied in the wrong order."""
    import oracle.operator as oo
    fs, N, nelec = fock3, 3, (2, 2)
    g = inputs.rng(1190)
    h1, h2 = _tensors(N, g)
    v = inputs.random_state(N, nelec, g)
    ref = fs.extract(_dense(fs, h1, h2, 0.0) @ fs.embed(v, nelec), nelec)
    orig = oo._spin_map

    def no_signs(norb, nocc, ops):
        src, dst, sgn = orig(norb, nocc, ops)
        return src, dst, np.abs(sgn)

    def swapped(norb, nocc, ops):
        if len(ops) == 4:
            ops = [ops[0], ops[1], ops[3], ops[2]]
        return orig(norb, nocc, ops)

    for bad in (no_signs, swapped):
        monkeypatch.setattr(oo, "_spin_map", bad)
        got = oo.apply_molecular_hamiltonian(v, h1, h2, N, nelec)
        assert np.max(np.abs(got - ref)) > 1e-3
        monkeypatch.undo()
    got = oo.apply_molecular_hamiltonian(v, h1, h2, N, nelec)
    assert np.max(np.abs(got - ref)) < 1e-11
