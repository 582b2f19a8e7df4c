"""Fermionic gates on a fixed-(N_a, N_b) state (oracle; test infrastructure
only).  Plain, slow, complex128 definitions; nothing here is tuned.

A state is a complex128 array of shape (dim_a, dim_b): element (i, j) is the
coefficient gamma(I_a, I_b) of §3.1, with I_a the alpha string of address i
and I_b the beta string of address j (addresses as in `oracle.strings`).
"""

import functools

import numpy as np

from .strings import strings, address_map, occupations, excite


def dims(norb, nelec):
    from math import comb
    return comb(norb, nelec[0]), comb(norb, nelec[1])


def hartree_fock(norb, nelec):
    """|{0..n_a-1}, {0..n_b-1}> (§2.2): address 0 in both spins."""
    da, db = dims(norb, nelec)
    v = np.zeros((da, db), np.complex128)
    v[0, 0] = 1.0
    return v


# ---------------------------------------------------------------------------
# Number-operator-sum evolution, §3.2.1
# ---------------------------------------------------------------------------
def apply_num_op_sum_evolution(vec, lam_a, lam_b, t, norb, nelec):
    """gamma' = exp(-i t [sum_{p in I_a} lam_a[p] + sum_{p in I_b} lam_b[p]]) gamma.
    `lam_b=None` means the same vector for both spins."""
    if lam_b is None:
        lam_b = lam_a
    oa = occupations(norb, nelec[0])
    ob = occupations(norb, nelec[1])
    sa = oa @ np.asarray(lam_a, float)
    sb = ob @ np.asarray(lam_b, float)
    phase = np.exp(-1j * t * (sa[:, None] + sb[None, :]))
    return phase * vec


# ---------------------------------------------------------------------------
# Diagonal-Coulomb evolution, §3.2.2
# ---------------------------------------------------------------------------
def diag_coulomb_angle(J_aa, J_ab, J_bb, t, norb, nelec):
    """theta(I_a, I_b) = -(t/2) * sum over the multiset S of J_pq, where S holds
    (p, q) for p, q both in I_a (J_aa), p in I_a & q in I_b (J_ab), p in I_b &
    q in I_a (J_ba = J_ab^T), and p, q both in I_b (J_bb); p == q is included
    because n_p n_p = n_p.  Computed determinant by determinant from the
    occupied-orbital lists."""
    if J_bb is None:
        J_bb = J_aa
    J_aa = np.asarray(J_aa, float)
    J_ab = np.asarray(J_ab, float)
    J_bb = np.asarray(J_bb, float)
    sa = strings(norb, nelec[0])
    sb = strings(norb, nelec[1])
    occ_a = [[p for p in range(norb) if (m >> p) & 1] for m in sa]
    occ_b = [[p for p in range(norb) if (m >> p) & 1] for m in sb]
    # the same-spin parts depend on one string only
    aa = np.array([sum(J_aa[p, q] for p in o for q in o) for o in occ_a])
    bb = np.array([sum(J_bb[p, q] for p in o for q in o) for o in occ_b])
    # the mixed part: both orders (p in I_a, q in I_b) and (p in I_b, q in I_a)
    Ob = occupations(norb, nelec[1])
    ab = np.zeros((len(sa), len(sb)))
    for i, oa in enumerate(occ_a):
        # row[q] = sum_{p in I_a} (J_ab[p, q] + J_ba[q, p]); then sum over q in I_b
        row = J_ab[oa, :].sum(axis=0) + J_ab.T[:, oa].sum(axis=1)
        ab[i, :] = Ob @ row
    return -0.5 * t * (aa[:, None] + ab + bb[None, :])


def diag_coulomb_angle_entry(J_aa, J_ab, J_bb, t, norb, nelec, i, j):
    """theta of the single determinant with alpha address i and beta address
    j: the same multiset sum over occupied pairs as `diag_coulomb_angle`
    (p == q included, J_ba = J_ab^T), written out for one determinant, for
    checks at sizes where the whole angle matrix is too large."""
    if J_bb is None:
        J_bb = J_aa
    J_aa = np.asarray(J_aa, float)
    J_ab = np.asarray(J_ab, float)
    J_bb = np.asarray(J_bb, float)
    ma = int(strings(norb, nelec[0])[i])
    mb = int(strings(norb, nelec[1])[j])
    oa = [p for p in range(norb) if (ma >> p) & 1]
    ob = [p for p in range(norb) if (mb >> p) & 1]
    s = 0.0
    for p in oa:
        for q in oa:
            s += J_aa[p, q]
    for p in ob:
        for q in ob:
            s += J_bb[p, q]
    for p in oa:
        for q in ob:
            s += J_ab[p, q] + J_ab[p, q]      # (p in I_a, q in I_b) and its J_ba mirror
    return -0.5 * t * s


def apply_diag_coulomb_evolution(vec, J_aa, J_ab, J_bb, t, norb, nelec):
    theta = diag_coulomb_angle(J_aa, J_ab, J_bb, t, norb, nelec)
    return np.exp(1j * theta) * vec


# ---------------------------------------------------------------------------
# Orbital rotation, §2.3 and §3.2.3
# ---------------------------------------------------------------------------
def minor_matrix(U, norb, nocc):
    """M[J, I] = det(U[J, I]) with rows J and columns I both ascending.

    From the defining relation of §2.3, U a_p^dag U^dag = sum_q U_qp a_q^dag,
    applied to every creation operator of cre(I)|vac> (the vacuum is left
    unchanged): the coefficient of |J> collects one product per bijection
    I -> J with the sign of reordering, which is det(U[J, I])."""
    s = strings(norb, nocc)
    d = len(s)
    if nocc == 0:
        return np.ones((1, 1), np.complex128)
    occ = np.array([[p for p in range(norb) if (int(m) >> p) & 1] for m in s])
    M = np.empty((d, d), np.complex128)
    for a in range(d):
        sub = U[occ[a], :]                      # rows J, all columns
        blocks = np.transpose(sub[:, occ], (1, 0, 2))  # [I][row in J][col in I]
        M[a, :] = np.linalg.det(blocks)
    return M


def minor_matrix_row(U, norb, nocc, a):
    """Row `a` of the minor matrix: det(U[J_a, I]) for every string I."""
    s = strings(norb, nocc)
    if nocc == 0:
        return np.ones(1, np.complex128)
    occ = np.array([[p for p in range(norb) if (int(m) >> p) & 1] for m in s])
    sub = np.asarray(U, complex)[occ[a], :]
    return np.linalg.det(np.transpose(sub[:, occ], (1, 0, 2)))


def rotated_string(U, norb, nocc, b):
    """Amplitudes of U(U)|I_b> for one spin over every string J: column b of
    the minor matrix, det(U[J, I_b])."""
    s = strings(norb, nocc)
    if nocc == 0:
        return np.ones(1, np.complex128)
    occ = np.array([[p for p in range(norb) if (int(m) >> p) & 1] for m in s])
    sub = np.asarray(U, complex)[:, occ[b]]     # all rows, the columns of I_b
    return np.linalg.det(sub[occ, :])          # [J][rows J][columns I_b]


def rotated_amplitude(vec, U_a, U_b, norb, nelec, i, j):
    """One amplitude of M_a vec M_b^T, for checks at sizes where the full
    minor matrices are too large."""
    if U_b is None:
        U_b = U_a
    ra = minor_matrix_row(U_a, norb, nelec[0], i)
    rb = minor_matrix_row(U_b, norb, nelec[1], j)
    return ra @ vec @ rb


def apply_orbital_rotation_minors(vec, U_a, U_b, norb, nelec):
    """gamma' = M_a gamma M_b^T.  The alpha and beta one-body generators
    commute with each other and with the other spin's creation operators, so
    each spin is rotated independently."""
    if U_b is None:
        U_b = U_a
    Ma = minor_matrix(np.asarray(U_a, complex), norb, nelec[0])
    Mb = minor_matrix(np.asarray(U_b, complex), norb, nelec[1])
    return Ma @ vec @ Mb.T


@functools.lru_cache(maxsize=None)
def givens_pairs(norb, nocc, p, q):
    """For the Givens rotation on orbitals (p, q) of one spin: the addresses
    (i, i') with p in I, q not in I and I' = I^{p->q}, and the sign sigma
    defined by a_q^dag a_p |I> = sigma |I'>."""
    s = strings(norb, nocc)
    amap = address_map(norb, nocc)
    src, dst, sgn = [], [], []
    for i, m in enumerate(s):
        m = int(m)
        r = excite(m, q, p)  # a_q^dag a_p
        if r is None or p == q:
            continue
        sign, m2 = r
        src.append(i)
        dst.append(amap[m2])
        sgn.append(sign)
    return np.array(src, int), np.array(dst, int), np.array(sgn, float)


def apply_givens(vec, c, s, p, q, spin, norb, nelec):
    """The Givens update of §3.2.3 for G = [[c, s], [-s*, c]] on orbitals
    (p, q) of spin `spin` (0 = alpha rows, 1 = beta columns).

    The paper's three cases hold in the basis {|I>, a_q^dag a_p |I>}; in the
    configuration basis the second vector is sigma |I'>, which puts sigma on
    the off-diagonal terms:
        gamma'(I)  = c gamma(I) + s sigma gamma(I')
        gamma'(I') = -s* sigma gamma(I) + c gamma(I')
    and every other coefficient is unchanged."""
    nocc = nelec[spin]
    src, dst, sgn = givens_pairs(norb, nocc, p, q)
    out = vec.copy()
    if spin == 0:
        x = vec[src, :]
        y = vec[dst, :]
        sg = sgn[:, None]
        out[src, :] = c * x + s * sg * y
        out[dst, :] = -np.conj(s) * sg * x + c * y
    else:
        x = vec[:, src]
        y = vec[:, dst]
        sg = sgn[None, :]
        out[:, src] = c * x + s * sg * y
        out[:, dst] = -np.conj(s) * sg * x + c * y
    return out


def givens_matrix(norb, c, s, p, q):
    """The N x N unitary equal to the identity except for the 2 x 2 block
    [[c, s], [-s*, c]] on rows/columns (p, q)."""
    G = np.eye(norb, dtype=complex)
    G[p, p] = c
    G[p, q] = s
    G[q, p] = -np.conj(s)
    G[q, q] = c
    return G


def givens_decomposition(U):
    """Eliminate U to a diagonal by left multiplication with Givens matrices:
    for each column k and each row r > k, a rotation on rows (k, r) zeroes
    U[r, k] against the pivot U[k, k].  Returns (rotations, D) with
        G_M ... G_1 U = D   =>   U = G_1^dag ... G_M^dag D,
    rotations = [(c, s, k, r), ...] in the order G_1..G_M.  The pairs (k, r)
    are in general not adjacent."""
    A = np.array(U, dtype=complex)
    n = A.shape[0]
    rots = []
    for k in range(n):
        for r in range(k + 1, n):
            a, b = A[k, k], A[r, k]
            if abs(b) == 0.0:
                continue
            rho = np.hypot(abs(a), abs(b))
            if abs(a) == 0.0:
                c, s = 0.0, 1.0 + 0j
            else:
                c = abs(a) / rho
                s = (a / abs(a)) * np.conj(b) / rho
            G = givens_matrix(n, c, s, k, r)
            A = G @ A
            rots.append((c, s, k, r))
    return rots, np.diag(A).copy()


def apply_orbital_rotation_givens(vec, U_a, U_b, norb, nelec):
    """Orbital rotation by the oracle's own Givens decomposition (§3.2.3):
    U = G_1^dag ... G_M^dag D, and the map U -> operator is a homomorphism
    (§2.3), so the operator of D acts first and that of G_1^dag last.  The
    operator of D = diag(e^{i phi_p}) multiplies gamma by prod_{p in I} D_pp;
    G^dag is again of the Givens form with s -> -s."""
    if U_b is None:
        U_b = U_a
    out = np.array(vec, dtype=complex)
    for spin, U in ((0, U_a), (1, U_b)):
        rots, D = givens_decomposition(np.asarray(U, complex))
        occ = occupations(norb, nelec[spin])
        ph = np.array([np.prod(D[row.astype(bool)]) for row in occ])
        out = out * (ph[:, None] if spin == 0 else ph[None, :])
        for (c, s, k, r) in reversed(rots):
            out = apply_givens(out, c, -s, k, r, spin, norb, nelec)
    return out


def apply_orbital_rotation(vec, U_a, U_b, norb, nelec, route="auto"):
    """Minor route for small dimensions (the exact definition), Givens route
    otherwise; both are checked against each other by the oracle's pins."""
    if route == "auto":
        route = "minors" if max(dims(norb, nelec)) <= 924 else "givens"
    if route == "minors":
        return apply_orbital_rotation_minors(vec, U_a, U_b, norb, nelec)
    return apply_orbital_rotation_givens(vec, U_a, U_b, norb, nelec)


def slater_from_hf(U_a, U_b, norb, nelec):
    """U|HF> (§2.4): amplitudes det(U_a[I_a, 0..n_a-1]) * det(U_b[I_b, 0..n_b-1]),
    the first column of each minor matrix; an exact rank-1 matrix."""
    if U_b is None:
        U_b = U_a
    vs = []
    for U, n in ((U_a, nelec[0]), (U_b, nelec[1])):
        U = np.asarray(U, complex)
        s = strings(norb, n)
        cols = list(range(n))
        v = np.empty(len(s), complex)
        for k, m in enumerate(s):
            rows = [p for p in range(norb) if (int(m) >> p) & 1]
            v[k] = np.linalg.det(U[np.ix_(rows, cols)]) if n else 1.0
        vs.append(v)
    return np.outer(vs[0], vs[1])
