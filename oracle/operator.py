"""Action of a molecular Hamiltonian on a state (operator-action section;
oracle, test infrastructure only).

    H = constant + sum_{pq sigma} h_pq a^dag_{p sigma} a_{q sigma}
        + 1/2 sum_{pqrs sigma tau} h_pqrs a^dag_{p sigma} a^dag_{r tau}
          a_{s tau} a_{q sigma}       (the molecular Hamiltonian equation)

Every term is applied literally: each string of a spin is acted on by the
operators of that spin, right to left, with the signs of `strings`
(§2.2 ordering).  An operator product of one spin has an even number of
factors, so it passes the other spin's creation string of
|I_a, I_b> = cre_b(I_b) cre_a(I_a)|vac> (§2.5) without a sign, and the
mixed two-body term factorises as (a^dag_{p sigma} a_{q sigma})
(a^dag_{r tau} a_{s tau}) after two anticommutations of even blocks.
Complex coefficients are allowed.
"""

import numpy as np

from .strings import annihilate, create, strings


def _apply_ops(mask, ops):
    """ops = [(is_creation, orbital), ...] applied right to left to cre(I);
    returns (sign, mask) or None."""
    sign = 1
    for is_cre, p in reversed(ops):
        r = create(mask, p) if is_cre else annihilate(mask, p)
        if r is None:
            return None
        s, mask = r
        sign *= s
    return sign, mask


def _spin_map(norb, nocc, ops):
    """For every string of one spin: (source index, target index, sign) of
    the operator product `ops`."""
    ss = strings(norb, nocc)
    addr = {int(m): k for k, m in enumerate(ss)}
    src, dst, sgn = [], [], []
    for k, m in enumerate(ss):
        r = _apply_ops(int(m), ops)
        if r is not None:
            src.append(k)
            dst.append(addr[r[1]])
            sgn.append(r[0])
    return np.array(src, dtype=np.int64), np.array(dst, dtype=np.int64), np.array(sgn)


def apply_molecular_hamiltonian(vec, one_body, two_body, norb, nelec, constant=0.0):
    """H vec for the molecular Hamiltonian with tensors h_pq = one_body[p, q]
    and h_pqrs = two_body[p, q, r, s]."""
    vec = np.asarray(vec, dtype=complex)
    h1 = np.asarray(one_body)
    h2 = np.asarray(two_body)
    out = constant * vec.copy()
    na, nb = nelec
    N = norb
    one = {}
    for s, n in ((0, na), (1, nb)):
        for p in range(N):
            for q in range(N):
                one[s, p, q] = _spin_map(N, n, [(True, p), (False, q)])
    # one-body terms
    for p in range(N):
        for q in range(N):
            c = h1[p, q]
            if c == 0:
                continue
            src, dst, sg = one[0, p, q]
            np.add.at(out, (dst, slice(None)), c * sg[:, None] * vec[src, :])
            src, dst, sg = one[1, p, q]
            np.add.at(out, (slice(None), dst), c * sg[None, :] * vec[:, src])
    # two-body terms
    for p in range(N):
        for q in range(N):
            for r in range(N):
                for s in range(N):
                    c = 0.5 * h2[p, q, r, s]
                    if c == 0:
                        continue
                    ops = [(True, p), (True, r), (False, s), (False, q)]
                    # sigma = tau = alpha, and beta
                    src, dst, sg = _spin_map(N, na, ops)
                    np.add.at(out, (dst, slice(None)), c * sg[:, None] * vec[src, :])
                    src, dst, sg = _spin_map(N, nb, ops)
                    np.add.at(out, (slice(None), dst), c * sg[None, :] * vec[:, src])
                    # sigma = alpha, tau = beta: (a^dag_pa a_qa)(a^dag_rb a_sb)
                    sa, da, ga = one[0, p, q]
                    sb, db, gb = one[1, r, s]
                    if len(sa) and len(sb):
                        blk = vec[np.ix_(sa, sb)] * (ga[:, None] * gb[None, :])
                        np.add.at(out, (da[:, None], db[None, :]), c * blk)
                    # sigma = beta, tau = alpha: (a^dag_ra a_sa)(a^dag_pb a_qb)
                    sa, da, ga = one[0, r, s]
                    sb, db, gb = one[1, p, q]
                    if len(sa) and len(sb):
                        blk = vec[np.ix_(sa, sb)] * (ga[:, None] * gb[None, :])
                        np.add.at(out, (da[:, None], db[None, :]), c * blk)
    return out
