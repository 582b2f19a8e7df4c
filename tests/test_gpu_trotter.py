"""Remaining Table-1 gates and Trotter-Suzuki evolution on the GPU against
the oracle, element by element."""

import os

import numpy as np
import pytest

import oracle
from paper_2605_03123_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2605_03123_gb300 import build, fsgpu
    if not os.path.exists(build.lib_path()):
        build.build()
    fsgpu.load_library()
    return fsgpu


def dev(v, dt):
    return torch.from_numpy(np.ascontiguousarray(v)).to(
        "cuda", torch.complex128 if dt == "c128" else torch.complex64)


def host(t):
    return t.cpu().numpy().astype(np.complex128)


def _hermitian(n, g, s=1.0):
    A = g.normal(0, s, (n, n)) + 1j * g.normal(0, s, (n, n))
    return (A + A.conj().T) / 2


SPIN = {(0,): "alpha", (1,): "beta", (0, 1): "both"}


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec", [(6, (3, 2)), (8, (4, 4)), (9, (2, 5))])
def test_table1_gates(lib, dt, norb, nelec):
    g = inputs.rng(800 + norb)
    v = inputs.random_state(norb, nelec, g)
    theta = 0.43
    for spins, name in SPIN.items():
        x = dev(v, dt)
        lib.apply_num_interaction_(x, theta, 2, norb, nelec, spin=name)
        ref = oracle.apply_num_interaction(v, theta, 2, spins, norb, nelec)
        assert np.max(np.abs(host(x) - ref)) < TOL[dt]
        for p, q in [(0, norb - 1), (3, 1)]:
            x = dev(v, dt)
            lib.apply_givens_rotation_(x, theta, p, q, norb, nelec, spin=name)
            ref = oracle.apply_givens_rotation(v, theta, p, q, spins, norb, nelec)
            assert np.max(np.abs(host(x) - ref)) < TOL[dt]
            x = dev(v, dt)
            lib.apply_tunneling_interaction_(x, theta, p, q, norb, nelec, spin=name)
            ref = oracle.apply_tunneling_interaction(v, theta, p, q, spins, norb, nelec)
            assert np.max(np.abs(host(x) - ref)) < TOL[dt]
    for p, sigma, q, tau in [(0, 0, 4, 0), (2, 1, 2, 1), (1, 0, 3, 1), (5, 1, 0, 0), (2, 0, 2, 1)]:
        x = dev(v, dt)
        lib.apply_num_num_interaction_(x, theta, p, q, norb, nelec, spins=(sigma, tau))
        ref = oracle.apply_num_num_interaction(v, theta, p, sigma, q, tau, norb, nelec)
        assert np.max(np.abs(host(x) - ref)) < TOL[dt]
    Ma, Mb = _hermitian(norb, g), _hermitian(norb, g)
    x = dev(v, dt)
    lib.apply_quad_ham_evolution_(x, Ma, 0.7, norb, nelec, M_b=Mb)
    ref = oracle.apply_quad_ham_evolution(v, Ma, Mb, 0.7, norb, nelec)
    assert np.max(np.abs(host(x) - ref)) < TOL[dt]


def test_table1_argument_errors(lib):
    x = dev(inputs.random_state(6, (3, 3), inputs.rng(1)), "c128")
    with pytest.raises(lib.FsError):
        lib.apply_givens_rotation_(x, 0.1, 2, 2, 6, (3, 3))
    with pytest.raises(lib.FsError):
        lib.apply_num_interaction_(x, 0.1, 6, 6, (3, 3))
    with pytest.raises(lib.FsError):
        lib.apply_quad_ham_evolution_(x, np.triu(np.ones((6, 6))), 0.1, 6, (3, 3))


def _df(norb, n_terms, g):
    h = _hermitian(norb, g, 0.5)
    Js = np.array([inputs.random_symmetric(norb, 0.5, g) for _ in range(n_terms)])
    Us = np.array([inputs.haar_unitary(norb, g) for _ in range(n_terms)])
    return h, Js, Us


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec,n_terms,n_steps,order", [
    (6, (3, 2), 2, 1, 0), (8, (4, 4), 3, 2, 1), (8, (3, 5), 1, 1, 2), (10, (5, 5), 2, 2, 0),
    (7, (3, 3), 0, 3, 1)])
def test_trotter_double_factorized(lib, dt, norb, nelec, n_terms, n_steps, order):
    g = inputs.rng(900 + norb + 10 * order)
    h, Js, Us = _df(norb, n_terms, g)
    v = inputs.random_state(norb, nelec, g)
    ref = oracle.simulate_trotter_double_factorized(v, h, list(Js), list(Us), 0.9, norb, nelec,
                                                    n_steps, order)
    x = dev(v, dt)
    lib.simulate_trotter_double_factorized_(x, h, Js, Us, 0.9, norb, nelec, n_steps=n_steps,
                                            order=order)
    assert np.max(np.abs(host(x) - ref)) < TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec,n_steps,order,same_spin", [
    (6, (2, 3), 1, 0, False), (8, (4, 4), 3, 1, True), (9, (4, 3), 2, 2, False)])
def test_trotter_diag_coulomb(lib, dt, norb, nelec, n_steps, order, same_spin):
    g = inputs.rng(950 + norb + order)
    h = _hermitian(norb, g, 0.5)
    J_aa, J_ab, J_bb = (inputs.random_symmetric(norb, 0.5, g) for _ in range(3))
    if same_spin:
        J_bb = None
    v = inputs.random_state(norb, nelec, g)
    ref = oracle.simulate_trotter_diag_coulomb(v, h, J_aa, J_ab, J_bb, 1.1, norb, nelec, n_steps,
                                               order)
    x = dev(v, dt)
    lib.simulate_trotter_diag_coulomb_(x, h, J_aa, J_ab, 1.1, norb, nelec, n_steps=n_steps,
                                       order=order, J_bb=J_bb)
    assert np.max(np.abs(host(x) - ref)) < TOL[dt]


def test_trotter_full_size_norm_and_c64_vs_c128(lib):
    """N=16 (8,8): three order-0 steps of a double-factorized Hamiltonian with
    three two-body terms keep the norm, and complex64 follows complex128."""
    norb, nelec = 16, (8, 8)
    g = inputs.rng(990)
    h, Js, Us = _df(norb, 3, g)
    res = {}
    v0 = inputs.device_state(norb, nelec, 77, torch.complex128)
    for dt in (torch.complex64, torch.complex128):
        x = v0.to(dt)
        lib.simulate_trotter_double_factorized_(x, h, Js, Us, 1.0, norb, nelec, n_steps=3,
                                                order=0)
        assert abs(float(torch.linalg.vector_norm(x).item()) - 1) < 1e-4
        res[dt] = x[:256].clone()
        del x
    d = (res[torch.complex64].to(torch.complex128) - res[torch.complex128]).abs().max()
    assert float(d.item()) < 2e-5
