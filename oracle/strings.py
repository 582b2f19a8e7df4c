"""Occupation strings and their addresses (oracle; test infrastructure only).

An occupation string of one spin is a set I of occupied spatial orbitals,
stored as an N-bit mask with bit p set when orbital p is occupied.

Address convention (a reading of §3.1, which delegates addresses to an FCI
module without stating them): the strings with n electrons are enumerated by
walking every integer mask from 0 to 2^N - 1 and keeping those with n set
bits; a string's address is its position in that walk.  The address of the
Hartree-Fock string {0, ..., n-1} is therefore 0 (§2.2).

Fermionic signs follow the configuration convention of §2.2 and §2.5:
|I> = cre(I)|vac> with creation operators sorted ascending from right to
left, and |I_a, I_b> = cre_b(I_b) cre_a(I_a)|vac>.  The signs below are
obtained by literally anticommuting an operator to its place in that product.
"""

import numpy as np


def strings(norb, nocc):
    """Masks of all strings with `nocc` electrons in `norb` orbitals, in
    address order (ascending integer value)."""
    if not (0 <= nocc <= norb):
        raise ValueError("need 0 <= nocc <= norb")
    out = [m for m in range(1 << norb) if bin(m).count("1") == nocc]
    return np.array(out, dtype=np.int64)


def address_map(norb, nocc):
    """Dictionary mask -> address (the position in `strings`)."""
    return {int(m): k for k, m in enumerate(strings(norb, nocc))}


def occupations(norb, nocc):
    """0/1 matrix of shape (dim, norb); row k is the occupation vector of the
    string with address k."""
    s = strings(norb, nocc)
    return ((s[:, None] >> np.arange(norb)[None, :]) & 1).astype(np.float64)


def occupied_list(mask, norb):
    return [p for p in range(norb) if (mask >> p) & 1]


def annihilate(mask, q):
    """a_q cre(I)|vac>.  Returns (sign, new_mask) or None when q is empty.

    a_q anticommutes past every creation operator standing to its left in
    cre(I), i.e. past those with a larger orbital index (§2.2 ordering)."""
    if not (mask >> q) & 1:
        return None
    n_left = bin(mask >> (q + 1)).count("1")
    return (-1) ** n_left, mask & ~(1 << q)


def create(mask, p):
    """a_p^dagger cre(I)|vac>.  Returns (sign, new_mask) or None when p is
    already occupied.  The new operator is moved right, past the creation
    operators with a larger orbital index, to its sorted place."""
    if (mask >> p) & 1:
        return None
    n_left = bin(mask >> (p + 1)).count("1")
    return (-1) ** n_left, mask | (1 << p)


def excite(mask, p, q):
    """a_p^dagger a_q cre(I)|vac> = sign * cre(I')|vac>.

    Returns (sign, I') or None when the result vanishes.  For p == q this is
    the number operator n_p."""
    r = annihilate(mask, q)
    if r is None:
        return None
    s1, m1 = r
    r = create(m1, p)
    if r is None:
        return None
    s2, m2 = r
    return s1 * s2, m2
