"""LUCJ forward pass and its reverse-mode gradient (oracle; test
infrastructure only).

Ansatz (§4.3, §4.5.1), as read for this library: one repetition is
U D U^dag with U = U(expm(K)) an orbital rotation (K anti-Hermitian) and D a
spin-balanced diagonal-Coulomb evolution at t = 1 (J_bb = J_aa).  The
repetitions act in order k = 0, 1, ..., n_reps-1 on the initial state (the
Hartree-Fock state by default); there is no final orbital rotation.  The
oracle applies every gate literally, without merging neighbouring rotations.

Gradient convention, for a real loss L = Re <g, psi_out> (g = dL/dpsi_out):
  * d psi_in = C^dag g for the (linear) circuit C;
  * dJ[p, q] = dL/dJ_pq with every entry of J treated as independent;
  * dK = dL/dRe K + i dL/dIm K for every entry of K.
"""

import numpy as np
import scipy.linalg

from .strings import strings, address_map, excite, occupations
from .gates import (apply_orbital_rotation, apply_diag_coulomb_evolution,
                    diag_coulomb_angle, hartree_fock, dims)


def _rotate(vec, U, norb, nelec):
    return apply_orbital_rotation(vec, U, U, norb, nelec)


def lucj_forward(K, J_aa, J_ab, norb, nelec, vec=None):
    """psi = prod_k [U(U_k) D(J_k) U(U_k)^dag] psi_0, literal composition."""
    psi = hartree_fock(norb, nelec) if vec is None else np.array(vec, complex)
    for k in range(len(K)):
        U = scipy.linalg.expm(np.asarray(K[k], complex))
        psi = _rotate(psi, U.conj().T, norb, nelec)
        psi = apply_diag_coulomb_evolution(psi, J_aa[k], J_ab[k], None, 1.0,
                                           norb, nelec)
        psi = _rotate(psi, U, norb, nelec)
    return psi


def transition_one_body(g, psi, norb, nelec, spins=(0, 1)):
    """T[p, q] = <g| E_pq |psi> with E_pq = sum_sigma a^dag_{p sigma} a_{q sigma},
    computed string by string with the anticommutation sign of `excite`.
    The alpha operators anticommute past cre_b(I_b) twice, so they carry no
    extra sign; the beta operators act directly on cre_b.  `spins` limits
    the sum to the listed spins (0 = alpha, 1 = beta)."""
    T = np.zeros((norb, norb), complex)
    for spin in spins:
        n = nelec[spin]
        s = strings(norb, n)
        amap = address_map(norb, n)
        for p in range(norb):
            for q in range(norb):
                src, dst, sg = [], [], []
                for i, m in enumerate(s):
                    r = excite(int(m), p, q)
                    if r is None:
                        continue
                    sign, m2 = r
                    src.append(i)
                    dst.append(amap[m2])
                    sg.append(sign)
                if not src:
                    continue
                src = np.array(src)
                dst = np.array(dst)
                sg = np.array(sg, float)
                if spin == 0:
                    # (E psi)[dst, :] += sg * psi[src, :]
                    T[p, q] += np.sum(sg[:, None] * np.conj(g[dst, :]) * psi[src, :])
                else:
                    T[p, q] += np.sum(sg[None, :] * np.conj(g[:, dst]) * psi[:, src])
    return T


def expm_frechet_adjoint(K, H):
    """Adjoint of the Frechet derivative of expm at K with respect to the real
    inner product <A, B> = Re tr(A^dag B):  L(K)^*[H] = L(K^dag)[H], read off
    the upper-right block of expm([[K^dag, H], [0, K^dag]])."""
    n = K.shape[0]
    Kd = np.asarray(K, complex).conj().T
    B = np.zeros((2 * n, 2 * n), complex)
    B[:n, :n] = Kd
    B[n:, n:] = Kd
    B[:n, n:] = H
    return scipy.linalg.expm(B)[:n, n:]


def lucj_vjp(K, J_aa, J_ab, g, norb, nelec, vec=None):
    """Reverse mode through the literal gate list, with every intermediate
    state stored.  Returns (dK, dJ_aa, dJ_ab, dpsi_in)."""
    n_reps = len(K)
    psi = hartree_fock(norb, nelec) if vec is None else np.array(vec, complex)
    Us = [scipy.linalg.expm(np.asarray(K[k], complex)) for k in range(n_reps)]
    # forward, storing the input of every gate
    tape = []
    for k in range(n_reps):
        for kind in ("Udag", "D", "U"):
            tape.append((k, kind, psi))
            if kind == "Udag":
                psi = _rotate(psi, Us[k].conj().T, norb, nelec)
            elif kind == "D":
                psi = apply_diag_coulomb_evolution(psi, J_aa[k], J_ab[k], None,
                                                   1.0, norb, nelec)
            else:
                psi = _rotate(psi, Us[k], norb, nelec)
    Oa = occupations(norb, nelec[0])
    Ob = occupations(norb, nelec[1])
    gU = [np.zeros((norb, norb), complex) for _ in range(n_reps)]
    dJaa = [np.zeros((norb, norb)) for _ in range(n_reps)]
    dJab = [np.zeros((norb, norb)) for _ in range(n_reps)]
    gcur = np.array(g, complex)
    for (k, kind, psi_in) in reversed(tape):
        if kind == "D":
            theta = diag_coulomb_angle(J_aa[k], J_ab[k], None, 1.0, norb, nelec)
            psi_out = np.exp(1j * theta) * psi_in
            # dL/dtheta = Re(conj(g) i psi_out) = -W
            W = np.imag(np.conj(gcur) * psi_out)
            # theta = -1/2 [oa Jaa oa + ob Jaa ob + 2 oa Jab ob]
            dJab[k] += Oa.T @ W @ Ob
            dJaa[k] += 0.5 * (Oa.T @ np.diag(W.sum(axis=1)) @ Oa
                              + Ob.T @ np.diag(W.sum(axis=0)) @ Ob)
            gcur = np.exp(-1j * theta) * gcur
        else:
            R = Us[k] if kind == "U" else Us[k].conj().T
            # g_in = U(R)^dag g = U(R^dag) g
            gcur = _rotate(gcur, R.conj().T, norb, nelec)
            T = transition_one_body(gcur, psi_in, norb, nelec)
            # dL = Re sum_pq (R^-1 dR)_pq T_pq  =>  Euclidean gradient R conj(T)
            gR = R @ np.conj(T)
            gU[k] += gR if kind == "U" else gR.conj().T
    dK = [expm_frechet_adjoint(np.asarray(K[k], complex), gU[k])
          for k in range(n_reps)]
    return np.array(dK), np.array(dJaa), np.array(dJab), gcur
