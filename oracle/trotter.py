"""Table-1 gates and Trotter-Suzuki time evolution (oracle; test
infrastructure only).

The remaining gates of Table 1 written from their definitions:
  number interaction           exp(i theta n_{p sigma})
  number-number interaction    exp(i theta n_{p sigma} n_{q tau})
  Givens rotation              exp(theta (a^dag_p a_q - a^dag_q a_p)) on one spin
  tunneling interaction        exp(i theta (a^dag_p a_q + a^dag_q a_p)) on one spin
  quadratic Hamiltonian        exp(-i t sum_pq M_pq a^dag_p a_q) per spin
The first two are diagonal phases computed per determinant; the other three
are orbital rotations exp(sum K_pq a^dag_p a_q) = U(expm(K)) (§2.3) with the
one-body generator K read off the definition.

Trotter-Suzuki product formulas (Hamiltonian time evolution section): for
H = H_1 + ... + H_L,
  S_0(t) = exp(-i H_L t) ... exp(-i H_1 t)
  S_1(t) = exp(-i H_1 t/2) ... exp(-i H_L t/2) exp(-i H_L t/2) ... exp(-i H_1 t/2)
  S_k(t) = S_{k-1}(u_k t)^2 S_{k-1}((1 - 4 u_k) t) S_{k-1}(u_k t)^2,
  u_k = 1 / (4 - 4^{1/(2k-1)}),
and exp(-i H T) ~ S(T/r)^r for r Trotter steps.  The term sequence is
expanded literally (no merging of neighbouring terms).

Hamiltonians:
  double factorized  H = sum_pq h_pq a^dag a + 1/2 sum_t sum_{pq sigma tau}
                     J^(t)_pq n^(t)_{p sigma} n^(t)_{q tau}, with
                     n^(t)_p = U(U^(t)) n_p U(U^(t))^dag, so the exponential of
                     term t is U(U^(t)) DC(J^(t), all spin pairs) U(U^(t))^dag;
  diagonal Coulomb   H = sum_pq h_pq a^dag a + 1/2 sum_{pq sigma tau}
                     J^{sigma tau}_pq n_{p sigma} n_{q tau}.
H_1 is the one-body term, whose exponential is the orbital rotation by
expm(-i h t); the two-body terms follow in their given order.
"""

import numpy as np
import scipy.linalg

from .gates import (apply_diag_coulomb_evolution, apply_orbital_rotation)
from .strings import strings


def _identity_other(norb):
    return np.eye(norb, dtype=complex)


def _rotate_spins(vec, U, spins, norb, nelec):
    """U(U) on the spins in `spins` (0 = alpha, 1 = beta), identity on the
    others."""
    I = _identity_other(norb)
    return apply_orbital_rotation(vec, U if 0 in spins else I, U if 1 in spins else I,
                                  norb, nelec)


def apply_num_interaction(vec, theta, p, spins, norb, nelec):
    """exp(i theta n_{p sigma}) for sigma in `spins` (Table 1)."""
    out = np.array(vec, dtype=complex, copy=True)
    sa, sb = strings(norb, nelec[0]), strings(norb, nelec[1])
    for i, ma in enumerate(sa):
        for j, mb in enumerate(sb):
            k = 0
            if 0 in spins and (int(ma) >> p) & 1:
                k += 1
            if 1 in spins and (int(mb) >> p) & 1:
                k += 1
            out[i, j] *= np.exp(1j * theta * k)
    return out


def apply_num_num_interaction(vec, theta, p, sigma, q, tau, norb, nelec):
    """exp(i theta n_{p sigma} n_{q tau}) (Table 1); spins 0 = alpha,
    1 = beta."""
    out = np.array(vec, dtype=complex, copy=True)
    sa, sb = strings(norb, nelec[0]), strings(norb, nelec[1])
    for i, ma in enumerate(sa):
        for j, mb in enumerate(sb):
            occ = (int(ma), int(mb))
            if (occ[sigma] >> p) & 1 and (occ[tau] >> q) & 1:
                out[i, j] *= np.exp(1j * theta)
    return out


def givens_generator(norb, theta, p, q):
    """K with sum K_pq a^dag_p a_q = theta (a^dag_p a_q - a^dag_q a_p)."""
    K = np.zeros((norb, norb), complex)
    K[p, q] += theta
    K[q, p] -= theta
    return K


def tunneling_generator(norb, theta, p, q):
    """K with sum K_pq a^dag_p a_q = i theta (a^dag_p a_q + a^dag_q a_p)."""
    K = np.zeros((norb, norb), complex)
    K[p, q] += 1j * theta
    K[q, p] += 1j * theta
    return K


def apply_givens_rotation(vec, theta, p, q, spins, norb, nelec):
    return _rotate_spins(vec, scipy.linalg.expm(givens_generator(norb, theta, p, q)), spins,
                         norb, nelec)


def apply_tunneling_interaction(vec, theta, p, q, spins, norb, nelec):
    return _rotate_spins(vec, scipy.linalg.expm(tunneling_generator(norb, theta, p, q)),
                         spins, norb, nelec)


def apply_quad_ham_evolution(vec, M_a, M_b, t, norb, nelec):
    """exp(-i t sum_{pq sigma} M^sigma_pq a^dag a): the orbital rotation by
    expm(-i M t) per spin (the equivalence stated after Table 1)."""
    if M_b is None:
        M_b = M_a
    return apply_orbital_rotation(vec, scipy.linalg.expm(-1j * t * np.asarray(M_a)),
                                  scipy.linalg.expm(-1j * t * np.asarray(M_b)), norb, nelec)


# ----------------------------------------------------------------- Trotter
def product_formula(n_terms, t, order):
    """The sequence of (term index j in 0..L-1, time) of S_order(t), first
    factor applied first."""
    if order == 0:
        return [(j, t) for j in range(n_terms)]
    if order == 1:
        half = [(j, t / 2) for j in range(n_terms)]
        return half + half[::-1]
    u = 1.0 / (4.0 - 4.0 ** (1.0 / (2 * order - 1)))
    outer = product_formula(n_terms, u * t, order - 1)
    inner = product_formula(n_terms, (1 - 4 * u) * t, order - 1)
    return outer + outer + inner + outer + outer


def _one_body_step(vec, h, tau, norb, nelec):
    U = scipy.linalg.expm(-1j * tau * np.asarray(h))
    return apply_orbital_rotation(vec, U, U, norb, nelec)


def simulate_trotter_double_factorized(vec, one_body, diag_coulomb_mats, orbital_rotations,
                                       time, norb, nelec, n_steps, order):
    """exp(-i H time) vec by n_steps steps of S_order(time / n_steps) for the
    double-factorized Hamiltonian; H_1 = one-body term, H_{1+t} = term t."""
    vec = np.array(vec, dtype=complex, copy=True)
    L = 1 + len(diag_coulomb_mats)
    seq = product_formula(L, time / n_steps, order)
    for _ in range(n_steps):
        for j, tau in seq:
            if j == 0:
                vec = _one_body_step(vec, one_body, tau, norb, nelec)
            else:
                J = np.asarray(diag_coulomb_mats[j - 1])
                U = np.asarray(orbital_rotations[j - 1])
                Ud = U.conj().T
                vec = apply_orbital_rotation(vec, Ud, Ud, norb, nelec)
                vec = apply_diag_coulomb_evolution(vec, J, J, J, tau, norb, nelec)
                vec = apply_orbital_rotation(vec, U, U, norb, nelec)
    return vec


def simulate_trotter_diag_coulomb(vec, one_body, J_aa, J_ab, J_bb, time, norb, nelec, n_steps,
                                  order):
    """exp(-i H time) vec for the diagonal-Coulomb Hamiltonian; H_1 =
    one-body term, H_2 = the two-body term (J_bb None means J_aa)."""
    vec = np.array(vec, dtype=complex, copy=True)
    seq = product_formula(2, time / n_steps, order)
    for _ in range(n_steps):
        for j, tau in seq:
            if j == 0:
                vec = _one_body_step(vec, one_body, tau, norb, nelec)
            else:
                vec = apply_diag_coulomb_evolution(vec, J_aa, J_ab, J_bb, tau, norb, nelec)
    return vec
