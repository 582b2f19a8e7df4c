"""Seeded synthetic inputs (NumPy PCG64), shared by the tests, the benchmark
and the smoke check.  This module draws random numbers and shapes them; it
holds none of the state-vector arithmetic.

Recipes (stand-ins for the randomly generated benchmark objects of §5.2):
  * state: i.i.d. complex normal amplitudes, normalised to unit 2-norm;
  * Haar unitary: QR of a complex Gaussian matrix with the phases of R's
    diagonal moved into Q;
  * real symmetric J: upper triangle (diagonal included) ~ N(0, sigma),
    mirrored;
  * anti-Hermitian K: real and imaginary parts of the strict upper triangle
    ~ N(0, sigma), diagonal i*N(0, sigma), K_qp = -conj(K_pq);
  * LUCJ interaction pattern: J_aa only on nearest neighbours of a line
    (zero diagonal), J_ab only on the diagonal (same site).
Seeds are 1000 * workload + index.
"""

from math import comb

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def dims(norb, nelec):
    return comb(norb, nelec[0]), comb(norb, nelec[1])


def random_state(norb, nelec, g, dtype=np.complex128):
    da, db = dims(norb, nelec)
    v = g.standard_normal((da, db)) + 1j * g.standard_normal((da, db))
    v /= np.linalg.norm(v)
    return v.astype(dtype)


def haar_unitary(n, g):
    z = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def random_symmetric(n, sigma, g):
    a = np.triu(g.normal(0.0, sigma, (n, n)))
    return a + np.triu(a, 1).T


def random_antihermitian(n, sigma, g):
    up = np.triu(g.normal(0.0, sigma, (n, n)) + 1j * g.normal(0.0, sigma, (n, n)), 1)
    k = up - up.conj().T
    k += np.diag(1j * g.normal(0.0, sigma, n))
    return k


def lucj_pattern(n, sigma, g):
    """(J_aa, J_ab): J_aa on line neighbours (p, p+1), symmetric; J_ab diagonal."""
    jaa = np.zeros((n, n))
    v = g.normal(0.0, sigma, n - 1)
    for p in range(n - 1):
        jaa[p, p + 1] = jaa[p + 1, p] = v[p]
    jab = np.diag(g.normal(0.0, sigma, n))
    return jaa, jab


def antihermitian_log(u):
    """Principal logarithm of a unitary via its Schur form (u = Z diag(e^{i a}) Z^dag),
    returned exactly anti-Hermitian."""
    import scipy.linalg
    t, z = scipy.linalg.schur(np.asarray(u, complex), output="complex")
    ang = np.angle(np.diag(t))
    k = (z * (1j * ang)[None, :]) @ z.conj().T
    return 0.5 * (k - k.conj().T)


def random_cotangent(norb, nelec, g):
    return random_state(norb, nelec, g)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
def plain_small(index=0):
    """N=8 (4,4): random state, one Haar U, diagonal Coulomb with symmetric
    J_aa, J_ab ~ N(0,1) (J_bb = J_aa) at t = 0.7."""
    g = rng(1000 * 1 + index)
    norb, nelec = 8, (4, 4)
    return dict(norb=norb, nelec=nelec, vec=random_state(norb, nelec, g),
                U=haar_unitary(norb, g), J_aa=random_symmetric(norb, 1.0, g),
                J_ab=random_symmetric(norb, 1.0, g), t=0.7)


def lucj_layers(norb, nelec, n_layers, sigma_j, t, seed, from_hf=False, with_cot=True):
    """LUCJ parameters with Haar-random rotations: K_k = log(U_k) for Haar U_k,
    J_k = t * N(0, sigma_j) symmetric (the evolution time folded into J)."""
    g = rng(seed)
    Ks, Jaa, Jab = [], [], []
    for _ in range(n_layers):
        Ks.append(antihermitian_log(haar_unitary(norb, g)))
        Jaa.append(t * random_symmetric(norb, sigma_j, g))
        Jab.append(t * random_symmetric(norb, sigma_j, g))
    vec = None if from_hf else random_state(norb, nelec, g)
    cot = random_cotangent(norb, nelec, g) if with_cot else None
    return dict(norb=norb, nelec=nelec, K=np.array(Ks), J_aa=np.array(Jaa),
                J_ab=np.array(Jab), vec=vec, cot=cot, cot_seed=seed + 500000)


def plain_at_scale(index=0):
    """N=16 (8,8), 10 layers: Haar rotations interleaved with diagonal-Coulomb
    evolutions, J ~ N(0, 0.5) symmetric, t = 0.3, from a random state."""
    return lucj_layers(16, (8, 8), 10, 0.5, 0.3, 1000 * 2 + index)


def lucj_small(index=0):
    """N=12 (6,6), 4 repetitions from Hartree-Fock; K ~ N(0, 0.1)
    anti-Hermitian, J_aa on line neighbours, J_ab on the diagonal, ~N(0, 0.1)."""
    g = rng(1000 * 3 + index)
    norb, nelec, n_reps = 12, (6, 6), 4
    Ks, Jaa, Jab = [], [], []
    for _ in range(n_reps):
        Ks.append(random_antihermitian(norb, 0.1, g))
        a, b = lucj_pattern(norb, 0.1, g)
        Jaa.append(a)
        Jab.append(b)
    return dict(norb=norb, nelec=nelec, K=np.array(Ks), J_aa=np.array(Jaa),
                J_ab=np.array(Jab), vec=None, cot=random_cotangent(norb, nelec, g))


def batch_circuits(n_circuits=512, index=0, with_cot=False):
    """Circuits with norb uniform in {8, 10, 12, 14} at half filling, 2
    repetitions each from Hartree-Fock, parameters as in `plain_at_scale`.
    Cotangents (1.6e9 amplitudes over 512 circuits) are drawn on the device
    from each circuit's `cot_seed` unless `with_cot`."""
    g = rng(1000 * 4 + index)
    norbs = g.choice([8, 10, 12, 14], size=n_circuits)
    out = []
    for c, n in enumerate(norbs):
        n = int(n)
        out.append(lucj_layers(n, (n // 2, n // 2), 2, 0.5, 0.3,
                               1000 * 4 + 100000 + 1000 * index + c, from_hf=True,
                               with_cot=with_cot))
    return out


def largest_state(index=0):
    """N=18 (9,9), one repetition from Hartree-Fock, J ~ N(0, 0.2).  The
    2.36e9-amplitude cotangent is not drawn here: `device_state` draws it on
    the GPU from its own seed."""
    g = rng(1000 * 5 + index)
    K = antihermitian_log(haar_unitary(18, g))[None]
    return dict(norb=18, nelec=(9, 9), K=K, J_aa=random_symmetric(18, 0.2, g)[None],
                J_ab=random_symmetric(18, 0.2, g)[None], vec=None, cot=None,
                cot_seed=1000 * 5 + 500 + index)


def device_state(norb, nelec, seed, dtype, device="cuda"):
    """A normalised random state drawn on the device (torch Philox generator
    seeded with `seed`), for states too large to draw on the host."""
    import torch
    da, db = dims(norb, nelec)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    real = torch.float32 if dtype == torch.complex64 else torch.float64
    v = torch.randn((da, db, 2), generator=gen, device=device, dtype=real)
    v = torch.view_as_complex(v)
    v /= torch.linalg.vector_norm(v)
    return v
