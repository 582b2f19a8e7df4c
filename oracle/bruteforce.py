"""Dense Jordan-Wigner check of the oracle on tiny systems (test
infrastructure only).

2N spin orbitals: alpha orbital p is mode p, beta orbital p is mode N + p.
With creation operators sorted ascending from right to left (§2.2),
cre(I_a U (N + I_b))|vac> = cre_b(I_b) cre_a(I_a)|vac> (§2.5) because every
beta mode index exceeds every alpha one, so the sector basis vector
|I_a, I_b> is the Fock basis vector with that occupation and no extra sign.

Operators are dense 4^N x 4^N matrices, so N <= 5.
"""

import numpy as np
import scipy.linalg

from .strings import strings


def creation_ops(n_modes):
    """a_j^dag on the 2^n_modes Fock space; basis index = occupation bitmask.
    a_j^dag |x> = (-1)^{#(occupied k > j)} |x + e_j> when j is empty."""
    dim = 1 << n_modes
    ops = []
    for j in range(n_modes):
        A = np.zeros((dim, dim))
        for x in range(dim):
            if (x >> j) & 1:
                continue
            sign = (-1) ** bin(x >> (j + 1)).count("1")
            A[x | (1 << j), x] = sign
        ops.append(A)
    return ops


class FockSpace:
    def __init__(self, norb):
        self.norb = norb
        self.cdag = creation_ops(2 * norb)
        self.c = [A.T for A in self.cdag]

    def one_body(self, M_a, M_b=None):
        """sum_pq M_a[p,q] a^dag_{p a} a_{q a} + M_b[p,q] a^dag_{p b} a_{q b}."""
        if M_b is None:
            M_b = M_a
        N = self.norb
        dim = 1 << (2 * N)
        H = np.zeros((dim, dim), complex)
        for p in range(N):
            for q in range(N):
                H += M_a[p, q] * (self.cdag[p] @ self.c[q])
                H += M_b[p, q] * (self.cdag[N + p] @ self.c[N + q])
        return H

    def number(self, mode):
        return self.cdag[mode] @ self.c[mode]

    def sector_indices(self, nelec):
        """Fock indices of the sector basis, as a (dim_a, dim_b) array."""
        N = self.norb
        sa = strings(N, nelec[0])
        sb = strings(N, nelec[1])
        return (sa[:, None] | (sb[None, :] << N)).astype(np.int64)

    def embed(self, vec, nelec):
        idx = self.sector_indices(nelec)
        full = np.zeros(1 << (2 * self.norb), complex)
        full[idx.ravel()] = np.asarray(vec).ravel()
        return full

    def extract(self, full, nelec):
        idx = self.sector_indices(nelec)
        return full[idx]


def orbital_rotation(fs, U_a, U_b, vec, nelec):
    """exp(sum_pq log(U)_pq a^dag_p a_q) per spin (§2.3), via scipy logm/expm."""
    if U_b is None:
        U_b = U_a
    K_a = scipy.linalg.logm(np.asarray(U_a, complex))
    K_b = scipy.linalg.logm(np.asarray(U_b, complex))
    G = scipy.linalg.expm(fs.one_body(K_a, K_b))
    return fs.extract(G @ fs.embed(vec, nelec), nelec)


def diag_coulomb(fs, J_aa, J_ab, J_bb, t, vec, nelec):
    """exp(-1/2 i t sum_{pq sigma tau} J^{sigma tau}_pq n_{p sigma} n_{q tau}),
    with J^{ba} = J^{ab}^T (Table 1)."""
    N = fs.norb
    if J_bb is None:
        J_bb = J_aa
    blocks = {(0, 0): J_aa, (0, 1): J_ab, (1, 0): np.asarray(J_ab).T, (1, 1): J_bb}
    dim = 1 << (2 * N)
    H = np.zeros((dim, dim))
    for (s, u), J in blocks.items():
        for p in range(N):
            for q in range(N):
                H += J[p, q] * (fs.number(s * N + p) @ fs.number(u * N + q))
    G = scipy.linalg.expm(-0.5j * t * H)
    return fs.extract(G @ fs.embed(vec, nelec), nelec)


def num_op_sum(fs, lam_a, lam_b, t, vec, nelec):
    """exp(-i t sum_{p sigma} lam^sigma_p n_{p sigma}) (Table 1)."""
    N = fs.norb
    if lam_b is None:
        lam_b = lam_a
    dim = 1 << (2 * N)
    H = np.zeros((dim, dim))
    for p in range(N):
        H += lam_a[p] * fs.number(p) + lam_b[p] * fs.number(N + p)
    G = scipy.linalg.expm(-1j * t * H)
    return fs.extract(G @ fs.embed(vec, nelec), nelec)
