"""Sampling configurations (oracle; test infrastructure only).

* From a state vector (sample-based algorithms section): configuration
  (I_a, I_b) with probability |psi(I_a, I_b)|^2 / ||psi||^2.  With a uniform
  u in [0, 1), the sample is the first address k (row-major over
  (alpha, beta)) whose inclusive cumulative probability exceeds u times the
  total: the inverse of the cumulative distribution in address order.

* From a Slater determinant U(U)|occ_a, occ_b> (Slater-sampling section):
  p(I_a, I_b) = |det U_a[I_a, occ_a]|^2 |det U_b[I_b, occ_b]|^2 (§2.4), so
  the spins are independent, each a determinantal point process whose kernel
  is the projection onto the columns Phi = U[:, occ].  Each spin is sampled
  by the chain rule for projection processes: with rows v_p of Phi, pick
  orbital p with probability |v_p|^2 / (number of orbitals still to pick),
  then project every row onto the complement of the chosen direction
  v_p / |v_p|; n picks in total.  The uniforms are inputs: one per pick,
  inverse-CDF over the orbitals in increasing order.
"""

import numpy as np


def _margin(c, x, k):
    """Distance from x to the nearer end of bin k of the cumulative sums c,
    relative to the total: how far the uniform is from a decision boundary."""
    lo = c[k - 1] if k > 0 else 0.0
    return min(x - lo, c[k] - x) / c[-1]


def sample_state(vec, uniforms, return_margin=False):
    """Addresses (row-major linear index into the (dim_a, dim_b) state) of the
    samples for the given uniforms; with return_margin, also each shot's
    distance to the nearest bin boundary, relative to the total."""
    p = np.abs(np.asarray(vec, dtype=complex).ravel()) ** 2
    c = np.cumsum(p)
    total = c[-1]
    x = np.asarray(uniforms) * total
    k = np.minimum(np.searchsorted(c, x, side="right"), len(c) - 1)
    if not return_margin:
        return k
    lo = np.where(k > 0, c[np.maximum(k - 1, 0)], 0.0)
    return k, np.minimum(x - lo, c[k] - x) / total


def _pick(weights, u):
    c = np.cumsum(weights)
    k = int(np.searchsorted(c, u * c[-1], side="right"))
    k = min(k, len(c) - 1)
    return k, _margin(c, u * c[-1], k)


def sample_slater_spin(U, occ, uniforms, return_margin=False):
    """Masks of one spin's samples; uniforms has shape (shots, len(occ)).
    With return_margin, also each shot's smallest distance (over its picks)
    from a decision boundary, relative to that pick's total."""
    U = np.asarray(U, dtype=complex)
    occ = list(occ)
    out, margins = [], []
    for us in np.atleast_2d(uniforms):
        V = U[:, occ].copy()
        mask = 0
        m = np.inf
        for i in range(len(occ)):
            w = np.sum(np.abs(V) ** 2, axis=1)
            p, mi = _pick(w, us[i])
            m = min(m, mi)
            mask |= 1 << p
            e = V[p] / np.linalg.norm(V[p])
            V = V - np.outer(V @ e.conj(), e)
        out.append(mask)
        margins.append(m)
    if return_margin:
        return np.array(out, dtype=object), np.array(margins)
    return np.array(out, dtype=object)


def chain_rule_probability(U, occ, order):
    """Probability that the chain rule picks the orbitals in `order`."""
    U = np.asarray(U, dtype=complex)
    V = U[:, list(occ)].copy()
    n = len(occ)
    prob = 1.0
    for i, p in enumerate(order):
        w = np.sum(np.abs(V) ** 2, axis=1)
        prob *= w[p] / (n - i)
        e = V[p] / np.linalg.norm(V[p])
        V = V - np.outer(V @ e.conj(), e)
    return prob
