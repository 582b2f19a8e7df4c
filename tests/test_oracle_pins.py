"""Pins for the oracle: checks against things other than the oracle itself
(dense Jordan-Wigner matrices with expm, closed forms, group identities, the
sizes printed in the paper, finite differences).  CPU only."""

import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import bruteforce as bf
from paper_2605_03123_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def _rs(seed):
    return inputs.rng(seed)


def _sectors(norb):
    return [(a, b) for a in range(norb + 1) for b in range(norb + 1)]


# ---------------------------------------------------------------- strings
@pytest.mark.parametrize("norb", range(0, 11))
def test_string_addresses_are_colex_ranks(norb):
    """Ascending-mask order coincides with the combinatorial number system:
    address(I) = sum_k C(o_k, k+1) over the occupied o_0 < o_1 < ..."""
    for n in range(norb + 1):
        s = oracle.strings(norb, n)
        assert len(s) == math.comb(norb, n)
        assert np.all(np.diff(s) > 0)
        for k, m in enumerate(s):
            occ = [p for p in range(norb) if (int(m) >> p) & 1]
            assert len(occ) == n
            assert sum(math.comb(o, i + 1) for i, o in enumerate(occ)) == k


def test_state_sizes_printed_in_paper():
    """The sector dimension C(N, n_a) C(N, n_b) at 16 bytes per amplitude
    reproduces every state size the paper prints."""
    cases = json.load(open(os.path.join(HERE, "golden", "state_sizes.json")))["cases"]
    for c in cases:
        da, db = oracle.dims(c["norb"], tuple(c["nelec"]))
        size = da * db * 16 / {"GiB": 2**30, "MiB": 2**20}[c["unit"]]
        assert round(size, c["digits"]) == c["printed"], c


def test_hf_is_address_zero():
    for norb, nelec in [(4, (2, 1)), (6, (3, 3)), (5, (0, 2))]:
        hf = oracle.hartree_fock(norb, nelec)
        assert hf[0, 0] == 1 and np.count_nonzero(hf) == 1
        sa = oracle.strings(norb, nelec[0])
        assert sa[0] == (1 << nelec[0]) - 1


# ------------------------------------------------------- brute force (JW)
@pytest.fixture(scope="module")
def fock3():
    return bf.FockSpace(3)


@pytest.fixture(scope="module")
def fock4():
    return bf.FockSpace(4)


@pytest.mark.parametrize("route", ["minors", "givens"])
def test_rotation_matches_jordan_wigner(fock3, fock4, route):
    for fs in (fock3, fock4):
        norb = fs.norb
        for k, nelec in enumerate(_sectors(norb)):
            g = _rs(17 + 31 * k + norb)
            Ua = inputs.haar_unitary(norb, g)
            Ub = inputs.haar_unitary(norb, g)
            v = inputs.random_state(norb, nelec, g)
            ref = bf.orbital_rotation(fs, Ua, Ub, v, nelec)
            got = oracle.apply_orbital_rotation(v, Ua, Ub, norb, nelec, route=route)
            assert np.max(np.abs(got - ref)) < 1e-12, (nelec, route)


def test_rotation_matches_jordan_wigner_n5():
    fs = bf.FockSpace(5)
    for nelec in [(2, 3), (3, 1), (5, 2)]:
        g = _rs(555 + nelec[0] * 7 + nelec[1])
        U = inputs.haar_unitary(5, g)
        v = inputs.random_state(5, nelec, g)
        ref = bf.orbital_rotation(fs, U, None, v, nelec)
        for route in ("minors", "givens"):
            got = oracle.apply_orbital_rotation(v, U, None, 5, nelec, route=route)
            assert np.max(np.abs(got - ref)) < 1e-12


def test_diag_coulomb_matches_jordan_wigner(fock3, fock4):
    for fs in (fock3, fock4):
        norb = fs.norb
        for k, nelec in enumerate(_sectors(norb)):
            g = _rs(900 + 13 * k + norb)
            Jaa = inputs.random_symmetric(norb, 1.0, g)
            Jab = g.normal(0, 1, (norb, norb))        # not symmetric on purpose
            Jbb = inputs.random_symmetric(norb, 1.0, g)
            v = inputs.random_state(norb, nelec, g)
            t = 0.7
            ref = bf.diag_coulomb(fs, Jaa, Jab, Jbb, t, v, nelec)
            got = oracle.apply_diag_coulomb_evolution(v, Jaa, Jab, Jbb, t, norb, nelec)
            assert np.max(np.abs(got - ref)) < 1e-12, nelec


def test_num_op_sum_matches_jordan_wigner(fock4):
    fs = fock4
    for k, nelec in enumerate(_sectors(4)):
        g = _rs(1300 + k)
        la, lb = g.normal(0, 1, 4), g.normal(0, 1, 4)
        v = inputs.random_state(4, nelec, g)
        ref = bf.num_op_sum(fs, la, lb, 0.9, v, nelec)
        got = oracle.apply_num_op_sum_evolution(v, la, lb, 0.9, 4, nelec)
        assert np.max(np.abs(got - ref)) < 1e-12


def test_givens_gate_is_table1_generator(fock4):
    """Table 1: Givens rotation exp(theta (a^dag_p a_q - a^dag_q a_p)) for a
    non-adjacent pair equals the oracle's Givens update with
    G = expm(theta (e_pq - e_qp)) = [[cos, sin], [-sin, cos]] on (p, q)."""
    fs = fock4
    theta, p, q = 0.37, 0, 3
    for nelec in [(2, 2), (3, 1), (1, 3)]:
        v = inputs.random_state(4, nelec, _rs(40 + nelec[0]))
        N = 4
        H = np.zeros((256, 256))
        for s in (0, 1):
            H += fs.cdag[s * N + p] @ fs.c[s * N + q] - fs.cdag[s * N + q] @ fs.c[s * N + p]
        ref = fs.extract(scipy.linalg.expm(theta * H) @ fs.embed(v, nelec), nelec)
        got = v
        for spin in (0, 1):
            got = oracle.apply_givens(got, math.cos(theta), math.sin(theta), p, q,
                                      spin, N, nelec)
        assert np.max(np.abs(got - ref)) < 1e-12


def test_transition_one_body_matches_jordan_wigner(fock3):
    fs = fock3
    for nelec in [(1, 2), (2, 2), (3, 1)]:
        g = _rs(77 + nelec[0])
        psi = inputs.random_state(3, nelec, g)
        gv = inputs.random_state(3, nelec, g)
        T = oracle.transition_one_body(gv, psi, 3, nelec)
        fp, fg = fs.embed(psi, nelec), fs.embed(gv, nelec)
        for p in range(3):
            for q in range(3):
                E = fs.cdag[p] @ fs.c[q] + fs.cdag[3 + p] @ fs.c[3 + q]
                assert abs(T[p, q] - np.vdot(fg, E @ fp)) < 1e-13


# ----------------------------------------------------------- closed forms
@pytest.mark.parametrize("route", ["minors", "givens"])
def test_rotation_of_hartree_fock_is_rank_one_minors(route):
    """§2.4: U|HF> has amplitudes det(U_a[I_a, 0..n_a-1]) det(U_b[I_b, 0..n_b-1])."""
    norb, nelec = 8, (4, 4)
    w = inputs.plain_small()
    U = w["U"]
    got = oracle.apply_orbital_rotation(oracle.hartree_fock(norb, nelec), U, U,
                                        norb, nelec, route=route)
    va = np.array([np.linalg.det(U[np.ix_([p for p in range(norb) if (int(m) >> p) & 1],
                                          range(4))]) for m in oracle.strings(norb, 4)])
    ref = np.outer(va, va)
    assert np.max(np.abs(got - ref)) < 1e-12
    assert np.linalg.matrix_rank(got, tol=1e-10) == 1


def test_one_electron_sector_is_plain_matrix_vector():
    g = _rs(5)
    U = inputs.haar_unitary(6, g)
    v = inputs.random_state(6, (1, 0), g)
    for route in ("minors", "givens"):
        got = oracle.apply_orbital_rotation(v, U, None, 6, (1, 0), route=route)
        assert np.max(np.abs(got[:, 0] - U @ v[:, 0])) < 1e-13


def test_extreme_fillings():
    """n = 0: the operator leaves the string alone; n = N: it multiplies by det U."""
    g = _rs(6)
    U = inputs.haar_unitary(5, g)
    v = inputs.random_state(5, (0, 5), g)
    for route in ("minors", "givens"):
        got = oracle.apply_orbital_rotation(v, U, None, 5, (0, 5), route=route)
        assert abs(got[0, 0] - np.linalg.det(U) * v[0, 0]) < 1e-13


# ------------------------------------------------------------- invariants
def test_homomorphism_and_adjoint():
    """§2.3: U(UV) = U(U)U(V) and U(U^dag) = U(U)^dag; norms are preserved."""
    norb, nelec = 6, (3, 2)
    g = _rs(9)
    U1, U2 = inputs.haar_unitary(norb, g), inputs.haar_unitary(norb, g)
    v, w = inputs.random_state(norb, nelec, g), inputs.random_state(norb, nelec, g)
    rot = lambda x, U: oracle.apply_orbital_rotation(x, U, None, norb, nelec, route="givens")
    a = rot(rot(v, U1), U2)
    b = oracle.apply_orbital_rotation(v, U2 @ U1, None, norb, nelec, route="minors")
    assert np.max(np.abs(a - b)) < 1e-12
    lhs = np.vdot(w, rot(v, U1))
    rhs = np.vdot(rot(w, U1.conj().T), v)
    assert abs(lhs - rhs) < 1e-12
    assert abs(np.linalg.norm(a) - 1) < 1e-12


def test_num_op_sum_is_orbital_rotation_by_diagonal():
    """After Table 1: number-operator-sum evolution is the orbital rotation
    with U = diag(exp(-i t lambda))."""
    norb, nelec = 6, (2, 3)
    g = _rs(10)
    lam = g.normal(0, 1, norb)
    v = inputs.random_state(norb, nelec, g)
    a = oracle.apply_num_op_sum_evolution(v, lam, None, 0.4, norb, nelec)
    b = oracle.apply_orbital_rotation(v, np.diag(np.exp(-0.4j * lam)), None, norb,
                                      nelec, route="givens")
    assert np.max(np.abs(a - b)) < 1e-13


def test_minor_and_givens_routes_agree():
    for norb, nelec in [(7, (3, 4)), (8, (4, 4)), (8, (2, 6)), (6, (6, 0))]:
        g = _rs(11 + norb + nelec[0])
        Ua, Ub = inputs.haar_unitary(norb, g), inputs.haar_unitary(norb, g)
        v = inputs.random_state(norb, nelec, g)
        a = oracle.apply_orbital_rotation(v, Ua, Ub, norb, nelec, route="minors")
        b = oracle.apply_orbital_rotation(v, Ua, Ub, norb, nelec, route="givens")
        assert np.max(np.abs(a - b)) < 1e-12


def test_diagonal_gates_commute_and_spin_swap_symmetry():
    norb, nelec = 6, (3, 3)
    g = _rs(12)
    J = inputs.random_symmetric(norb, 1.0, g)
    Jab = inputs.random_symmetric(norb, 1.0, g)
    lam = g.normal(0, 1, norb)
    U = inputs.haar_unitary(norb, g)
    v = inputs.random_state(norb, nelec, g)
    dc = lambda x: oracle.apply_diag_coulomb_evolution(x, J, Jab, None, 0.3, norb, nelec)
    no = lambda x: oracle.apply_num_op_sum_evolution(x, lam, None, 0.3, norb, nelec)
    assert np.max(np.abs(dc(no(v)) - no(dc(v)))) < 1e-13
    rot = lambda x: oracle.apply_orbital_rotation(x, U, None, norb, nelec, route="givens")
    # alpha <-> beta exchange (transpose) commutes with spin-symmetric gates
    assert np.max(np.abs(dc(rot(v)).T - dc(rot(v.T)))) < 1e-12


# --------------------------------------------------------------- gradient
def test_expm_frechet_adjoint_by_finite_differences():
    g = _rs(13)
    K = inputs.random_antihermitian(4, 0.5, g)
    H = g.normal(0, 1, (4, 4)) + 1j * g.normal(0, 1, (4, 4))
    E = g.normal(0, 1, (4, 4)) + 1j * g.normal(0, 1, (4, 4))
    h = 1e-6
    dexp = (scipy.linalg.expm(K + h * E) - scipy.linalg.expm(K - h * E)) / (2 * h)
    lhs = np.real(np.vdot(H, dexp))
    rhs = np.real(np.vdot(oracle.expm_frechet_adjoint(K, H), E))
    assert abs(lhs - rhs) < 1e-8


@pytest.mark.parametrize("from_hf", [True, False])
def test_lucj_gradient_by_central_differences(from_hf):
    norb, nelec, n_reps = 4, (2, 1), 2
    g = _rs(14 + from_hf)
    K = np.array([inputs.random_antihermitian(norb, 0.4, g) for _ in range(n_reps)])
    Jaa = np.array([inputs.random_symmetric(norb, 0.5, g) for _ in range(n_reps)])
    Jab = np.array([g.normal(0, 0.5, (norb, norb)) for _ in range(n_reps)])
    v0 = None if from_hf else inputs.random_state(norb, nelec, g)
    cot = inputs.random_state(norb, nelec, g)
    dK, dJaa, dJab, dv = oracle.lucj_vjp(K, Jaa, Jab, cot, norb, nelec, vec=v0)

    def loss(K_, Jaa_, Jab_, v_):
        out = oracle.lucj_forward(K_, Jaa_, Jab_, norb, nelec, vec=v_)
        return np.real(np.vdot(cot, out))

    h = 1e-6
    for (k, p, q) in [(0, 0, 1), (1, 2, 3), (1, 1, 1), (0, 3, 0)]:
        for unit in (1.0, 1j):
            Kp, Km = K.copy(), K.copy()
            Kp[k, p, q] += h * unit
            Km[k, p, q] -= h * unit
            fd = (loss(Kp, Jaa, Jab, v0) - loss(Km, Jaa, Jab, v0)) / (2 * h)
            an = dK[k, p, q].real if unit == 1.0 else dK[k, p, q].imag
            assert abs(fd - an) < 1e-7, (k, p, q, unit, fd, an)
        for J, dJ, which in ((Jaa, dJaa, 0), (Jab, dJab, 1)):
            Jp, Jm = J.copy(), J.copy()
            Jp[k, p, q] += h
            Jm[k, p, q] -= h
            args_p = (K, Jp, Jab) if which == 0 else (K, Jaa, Jp)
            args_m = (K, Jm, Jab) if which == 0 else (K, Jaa, Jm)
            fd = (loss(*args_p, v0) - loss(*args_m, v0)) / (2 * h)
            assert abs(fd - dJ[k, p, q]) < 1e-7, (which, k, p, q)
    if not from_hf:
        for idx in [(0, 0), (2, 1), (5, 3)]:
            for unit in (1.0, 1j):
                vp, vm = v0.copy(), v0.copy()
                vp[idx] += h * unit
                vm[idx] -= h * unit
                fd = (loss(K, Jaa, Jab, vp) - loss(K, Jaa, Jab, vm)) / (2 * h)
                an = dv[idx].real if unit == 1.0 else dv[idx].imag
                assert abs(fd - an) < 1e-7


# ---------------------------------------- single rows and single amplitudes
def _minor_sectors():
    return [(5, 0), (5, 1), (5, 2), (6, 3), (7, 4), (8, 1), (8, 4), (8, 7), (8, 8)]


@pytest.mark.parametrize("norb,nocc", _minor_sectors())
def test_minor_matrix_row_is_a_row_of_the_minor_matrix(norb, nocc):
    """Every row of minor_matrix_row equals the corresponding row of the full
    minor matrix, itself pinned to dense Jordan-Wigner evolution above."""
    g = _rs(4100 + 17 * norb + nocc)
    U = inputs.haar_unitary(norb, g)
    M = oracle.minor_matrix(U, norb, nocc)
    for a in range(M.shape[0]):
        row = oracle.minor_matrix_row(U, norb, nocc, a)
        assert np.max(np.abs(row - M[a])) < 1e-13, (norb, nocc, a)


def test_minor_matrix_row_closed_forms():
    """One electron: strings are single orbitals in order, so row a of the
    minor matrix is row a of U (c' = U c).  A full shell has one string
    whose amplitude is multiplied by det U.  No electrons: the vacuum is
    left unchanged."""
    g = _rs(4200)
    for norb in (1, 3, 8):
        U = inputs.haar_unitary(norb, g)
        for a in range(norb):
            assert np.max(np.abs(oracle.minor_matrix_row(U, norb, 1, a) - U[a])) < 1e-15
        full = oracle.minor_matrix_row(U, norb, norb, 0)
        assert full.shape == (1,) and abs(full[0] - np.linalg.det(U)) < 1e-13
        assert np.array_equal(oracle.minor_matrix_row(U, norb, 0, 0), np.ones(1))


def test_rotated_amplitude_matches_jordan_wigner(fock3, fock4):
    """Single amplitudes of the rotated state against dense Jordan-Wigner
    evolution with expm (§2.3), every sector at N = 3 and 4."""
    for fs in (fock3, fock4):
        norb = fs.norb
        for k, nelec in enumerate(_sectors(norb)):
            g = _rs(4300 + 11 * k + norb)
            Ua = inputs.haar_unitary(norb, g)
            Ub = inputs.haar_unitary(norb, g)
            v = inputs.random_state(norb, nelec, g)
            ref = bf.orbital_rotation(fs, Ua, Ub, v, nelec)
            for i in range(ref.shape[0]):
                for j in range(ref.shape[1]):
                    got = oracle.rotated_amplitude(v, Ua, Ub, norb, nelec, i, j)
                    assert abs(got - ref[i, j]) < 1e-12, (nelec, i, j)


def test_rotated_amplitude_matches_jordan_wigner_n5():
    fs = bf.FockSpace(5)
    for nelec in [(2, 3), (4, 1)]:
        g = _rs(4400 + 7 * nelec[0] + nelec[1])
        U = inputs.haar_unitary(5, g)
        v = inputs.random_state(5, nelec, g)
        ref = bf.orbital_rotation(fs, U, None, v, nelec)
        for i in range(ref.shape[0]):
            for j in range(0, ref.shape[1], 2):
                got = oracle.rotated_amplitude(v, U, None, 5, nelec, i, j)
                assert abs(got - ref[i, j]) < 1e-12


@pytest.mark.parametrize("norb,nelec", [(6, (3, 2)), (8, (4, 4)), (8, (1, 7)), (7, (0, 3))])
def test_rotated_amplitude_matches_full_minor_rotation(norb, nelec):
    """At N up to 8 every amplitude of the single-entry route equals the
    whole-state minor route and the independent Givens route."""
    g = _rs(4500 + norb + 3 * nelec[0])
    Ua = inputs.haar_unitary(norb, g)
    Ub = inputs.haar_unitary(norb, g)
    v = inputs.random_state(norb, nelec, g)
    full = oracle.apply_orbital_rotation_minors(v, Ua, Ub, norb, nelec)
    giv = oracle.apply_orbital_rotation(v, Ua, Ub, norb, nelec, route="givens")
    assert np.max(np.abs(full - giv)) < 1e-12
    rows = range(full.shape[0])
    cols = range(full.shape[1])
    for i in rows:
        for j in cols:
            got = oracle.rotated_amplitude(v, Ua, Ub, norb, nelec, i, j)
            assert abs(got - full[i, j]) < 1e-12, (i, j)


@pytest.mark.parametrize("norb,nocc", [(4, 2), (6, 3), (7, 1), (8, 4), (5, 5)])
def test_rotated_string_is_a_column_of_the_minor_matrix(norb, nocc):
    g = _rs(4700 + norb * 3 + nocc)
    U = inputs.haar_unitary(norb, g)
    M = oracle.minor_matrix(U, norb, nocc)
    for b in range(M.shape[1]):
        assert np.max(np.abs(oracle.rotated_string(U, norb, nocc, b) - M[:, b])) < 1e-13


def test_rotated_string_of_hartree_fock_is_the_slater_closed_form():
    """b = 0 is the Hartree-Fock string: U|HF> per spin (§2.4)."""
    g = _rs(4750)
    U = inputs.haar_unitary(7, g)
    ref = oracle.slater_from_hf(U, U, 7, (3, 3))
    va = oracle.rotated_string(U, 7, 3, 0)
    assert np.max(np.abs(np.outer(va, va) - ref)) < 1e-13


def test_rotated_string_matches_jordan_wigner(fock4):
    """U(U_a) x U(U_b) on one basis determinant against dense evolution."""
    fs = fock4
    for k, nelec in enumerate([(2, 2), (1, 3), (3, 0)]):
        g = _rs(4800 + k)
        Ua, Ub = inputs.haar_unitary(4, g), inputs.haar_unitary(4, g)
        da, db = oracle.dims(4, nelec)
        for i in range(da):
            for j in range(db):
                e = np.zeros((da, db), complex)
                e[i, j] = 1
                ref = bf.orbital_rotation(fs, Ua, Ub, e, nelec)
                got = np.outer(oracle.rotated_string(Ua, 4, nelec[0], i),
                               oracle.rotated_string(Ub, 4, nelec[1], j))
                assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("norb,nelec", [(3, (2, 1)), (4, (2, 2)), (6, (3, 2)), (7, (0, 4))])
def test_diag_coulomb_angle_entry_matches_whole_matrix(norb, nelec):
    """The single-determinant angle against the whole angle matrix (pinned
    to dense Jordan-Wigner evolution above) with a non-symmetric J_ab."""
    g = _rs(4900 + norb)
    Jaa = inputs.random_symmetric(norb, 1.0, g)
    Jab = g.normal(0, 1, (norb, norb))
    Jbb = inputs.random_symmetric(norb, 1.0, g)
    for jbb in (Jbb, None):
        th = oracle.diag_coulomb_angle(Jaa, Jab, jbb, 0.37, norb, nelec)
        for i in range(th.shape[0]):
            for j in range(th.shape[1]):
                got = oracle.diag_coulomb_angle_entry(Jaa, Jab, jbb, 0.37, norb, nelec, i, j)
                assert abs(got - th[i, j]) < 1e-12


def test_diag_coulomb_angle_entry_matches_jordan_wigner(fock3):
    """exp(i theta) of every determinant against dense expm of the
    diagonal-Coulomb operator (§3.2.2)."""
    fs = fock3
    nelec = (2, 1)
    g = _rs(4950)
    Jaa = inputs.random_symmetric(3, 1.0, g)
    Jab = g.normal(0, 1, (3, 3))
    da, db = oracle.dims(3, nelec)
    ones = np.ones((da, db), complex)
    ref = bf.diag_coulomb(fs, Jaa, Jab, None, 0.8, ones, nelec)
    for i in range(da):
        for j in range(db):
            th = oracle.diag_coulomb_angle_entry(Jaa, Jab, None, 0.8, 3, nelec, i, j)
            assert abs(np.exp(1j * th) - ref[i, j]) < 1e-12
    # planted mistakes: a dropped 1/2, or the mixed term counted once
    th_bad = -0.8 * sum(Jaa[p, q] for p in (0, 1) for q in (0, 1))
    assert abs(np.exp(1j * th_bad) - ref[0, 0]) > 1e-3


def test_single_amplitude_pins_catch_planted_mistakes(fock3):
    """A row/column mix-up or a transposed U inside the single-row minor
    route fails the pins above."""
    fs = fock3
    nelec = (2, 1)
    g = _rs(4600)
    Ua = inputs.haar_unitary(3, g)
    Ub = inputs.haar_unitary(3, g)
    v = inputs.random_state(3, nelec, g)
    ref = bf.orbital_rotation(fs, Ua, Ub, v, nelec)
    M = oracle.minor_matrix(Ua, 3, 2)

    def column_instead_of_row(U, norb, nocc, a):
        s = oracle.strings(norb, nocc)
        occ = np.array([[p for p in range(norb) if (int(m) >> p) & 1] for m in s])
        sub = np.asarray(U, complex)[:, occ[a]]           # columns I_a: wrong
        return np.linalg.det(sub[occ, :])                  # det U[I, I_a] = M[I, a]

    bad_rows = [column_instead_of_row(Ua, 3, 2, a) for a in range(3)]
    assert max(np.max(np.abs(r - M[a])) for a, r in enumerate(bad_rows)) > 1e-3
    # a transposed U in both spins
    worst = max(abs(oracle.rotated_amplitude(v, Ua.T, Ub.T, 3, nelec, i, j) - ref[i, j])
                for i in range(3) for j in range(3))
    assert worst > 1e-3
    # the spins swapped
    worst = max(abs(oracle.rotated_amplitude(v, Ub, Ua, 3, nelec, i, j) - ref[i, j])
                for i in range(3) for j in range(3))
    assert worst > 1e-3


# ------------------------------------------------- planted mistakes (CPU)
def test_pins_catch_planted_mistakes(monkeypatch, fock3):
    """Plant plausible mistakes in the oracle and check that a pin fails."""
    fs = fock3
    nelec = (2, 2)
    g = _rs(99)
    U = inputs.haar_unitary(3, g)
    v = inputs.random_state(3, nelec, g)
    ref = bf.orbital_rotation(fs, U, None, v, nelec)
    J = inputs.random_symmetric(3, 1.0, g)
    refdc = bf.diag_coulomb(fs, J, J, None, 0.5, v, nelec)

    import oracle.gates as og
    # 1. drop the Jordan-Wigner sign from the Givens update
    orig_pairs = og.givens_pairs.__wrapped__

    def no_sign(norb, nocc, p, q):
        s, d, sg = orig_pairs(norb, nocc, p, q)
        return s, d, np.abs(sg)
    og.givens_pairs.cache_clear()
    monkeypatch.setattr(og, "givens_pairs", no_sign)
    bad = og.apply_orbital_rotation(v, U, None, 3, nelec, route="givens")
    assert np.max(np.abs(bad - ref)) > 1e-3
    monkeypatch.undo()
    og.givens_pairs.cache_clear()
    # 2. transpose U in the minor route
    bad = og.apply_orbital_rotation_minors(v, U.T, None, 3, nelec)
    assert np.max(np.abs(bad - ref)) > 1e-3
    # 3. drop the factor 1/2 of the diagonal-Coulomb phase
    bad = og.apply_diag_coulomb_evolution(v, J, J, None, 1.0, 3, nelec)
    assert np.max(np.abs(bad - refdc)) > 1e-3
