"""Sampling on the GPU against the oracle, shot by shot on the same seeded
uniforms: configurations from a state (inverse CDF over |psi|^2) and
orbital occupations from Slater determinants (chain rule).  A shot whose
uniform lies within 1e-10 of a decision boundary (relative to the total,
as the oracle reports it) may go to either side; it is checked for validity
instead.  Edge cases: zero-amplitude runs spanning groups and tiles, clamped
uniforms, zero and non-finite states, empty and full occupations, masks
wider than one word, argument errors."""

import os

import numpy as np
import pytest

import oracle
from paper_2605_03123_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MARGIN = 1e-10


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


def check_state_shots(v_host, u, got):
    """got (addresses from the GPU) against the oracle on the state the GPU
    saw (v_host, complex128)."""
    ref, margin = oracle.sample_state(v_host, u, return_margin=True)
    p = np.abs(v_host.ravel()) ** 2
    c = np.cumsum(p)
    sure = margin > MARGIN
    assert np.array_equal(got[sure], ref[sure]), np.flatnonzero(got[sure] != ref[sure])[:10]
    for k in np.flatnonzero(~sure):  # near a boundary: valid and adjacent
        a = got[k]
        assert 0 <= a < p.size and p[a] > 0
        lo = c[a - 1] if a > 0 else 0.0
        assert lo - 1e-9 * c[-1] <= u[k] * c[-1] <= c[a] + 1e-9 * c[-1]
    return int(np.sum(~sure))


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec", [(4, (2, 1)), (8, (4, 4)), (10, (5, 4)), (12, (6, 5))])
def test_sample_state_parity(lib, dt, norb, nelec):
    """Element-by-element agreement with the oracle; N=12 (6,5) spans
    eleven tiles of 65536 amplitudes and a ragged tail."""
    g = inputs.rng(1500 + norb)
    v = inputs.random_state(norb, nelec, g)
    x = dev(v, dt)
    u = g.random(20000)
    got = lib.sample_state(x, norb, nelec, uniforms=u).cpu().numpy()
    check_state_shots(x.cpu().numpy().astype(np.complex128), u, got)


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_sample_state_sparse(lib, dt):
    """A state that is zero except on a few scattered amplitudes, with
    zero runs longer than a group (256) and a tile (65536): zero-amplitude
    configurations are never returned, and every shot matches the oracle."""
    norb, nelec = 12, (6, 5)
    g = inputs.rng(1520)
    v = np.zeros((924, 792), complex)
    flat = v.reshape(-1)
    idx = np.concatenate([[0, 1, 300, 70000, 70001], g.choice(flat.size, 40, replace=False),
                          [flat.size - 1]])
    flat[idx] = g.normal(size=idx.size) + 1j * g.normal(size=idx.size)
    x = dev(v, dt)
    u = np.concatenate([g.random(5000), [0.0, np.nextafter(1.0, 0.0)]])
    got = lib.sample_state(x, norb, nelec, uniforms=u).cpu().numpy()
    vh = x.cpu().numpy().astype(np.complex128)
    assert np.all(np.abs(vh.reshape(-1)[got]) > 0)
    check_state_shots(vh, u, got)


def test_sample_state_edges(lib):
    norb, nelec = 8, (4, 4)
    g = inputs.rng(1530)
    v = inputs.random_state(norb, nelec, g)
    v.reshape(-1)[:10] = 0
    v.reshape(-1)[-7:] = 0
    x = dev(v, "c128")
    nz = np.flatnonzero(np.abs(v.reshape(-1)) > 0)
    got = lib.sample_state(x, norb, nelec, uniforms=[0.0, -0.5, float("nan"), 1.0, 7.0]).cpu()
    assert got.tolist() == [nz[0], nz[0], nz[0], nz[-1], nz[-1]]
    # zero and non-finite states give -1
    z = torch.zeros_like(x)
    assert lib.sample_state(z, norb, nelec, uniforms=[0.3, 0.9]).cpu().tolist() == [-1, -1]
    y = x.clone()
    y[3, 5] = float("nan")
    assert lib.sample_state(y, norb, nelec, uniforms=[0.3]).cpu().tolist() == [-1]
    # no shots, one-configuration sector
    assert lib.sample_state(x, norb, nelec, uniforms=np.zeros(0)).numel() == 0
    one = dev(np.ones((1, 1)), "c64")
    assert lib.sample_state(one, 4, (0, 4), uniforms=[0.0, 0.5, 0.99]).cpu().tolist() == [0] * 3


def test_sample_state_matches_strings(lib):
    """Addresses map to the oracle's strings, and seeded draws repeat."""
    norb, nelec = 6, (3, 2)
    g = inputs.rng(1540)
    x = dev(inputs.random_state(norb, nelec, g), "c128")
    a1 = lib.sample_state(x, norb, nelec, shots=1000, seed=5)
    a2 = lib.sample_state(x, norb, nelec, shots=1000, seed=5)
    assert torch.equal(a1, a2)
    ma, mb = lib.addresses_to_strings(a1, norb, nelec)
    sa, sb = oracle.strings(norb, 3), oracle.strings(norb, 2)
    a = a1.cpu().numpy()
    assert np.array_equal(ma, sa[a // len(sb)]) and np.array_equal(mb, sb[a % len(sb)])


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_sample_state_full_size(lib, dt):
    """N=16 (8,8), 1.66e8 amplitudes (the LUCJ workload's state), in the
    configuration the benchmark times: shots compared with the oracle one by
    one on the full state."""
    norb, nelec = 16, (8, 8)
    x = inputs.device_state(norb, nelec, 31, torch.complex128 if dt == "c128" else torch.complex64)
    g = inputs.rng(1550)
    u = g.random(3000)
    got = lib.sample_state(x, norb, nelec, uniforms=u).cpu().numpy()
    vh = x.cpu().numpy().astype(np.complex128)
    del x
    check_state_shots(vh, u, got)


def masks_as_ints(m):
    m = np.asarray(m)
    if m.ndim == 1:
        return [int(w) for w in m]
    return [sum(int(w) << (64 * k) for k, w in enumerate(row)) for row in m]


def check_slater_shots(U, occ, u, got):
    ref, margin = oracle.sample_slater_spin(U, occ, u, return_margin=True)
    got = masks_as_ints(got)
    n_unsure = 0
    for k in range(len(got)):
        assert bin(got[k]).count("1") == len(occ)
        if margin[k] > MARGIN:
            assert got[k] == int(ref[k]), k
        else:
            n_unsure += 1
    return n_unsure


@pytest.mark.parametrize("N,n,shots", [(5, 2, 2000), (16, 4, 2000), (40, 10, 1000),
                                       (64, 16, 500), (65, 16, 500), (100, 25, 300),
                                       (300, 75, 40)])
def test_sample_slater_parity(lib, N, n, shots):
    """Every shot's mask equals the oracle's, at sizes covering one and
    several warps per CTA, one and two mask words, and the coefficients held
    in shared memory (N n <= 12000) or in global scratch (N=300)."""
    g = inputs.rng(1600 + N)
    U = inputs.haar_unitary(N, g)
    occ = sorted(g.choice(N, n, replace=False).tolist())
    u = g.random((shots, n))
    got = lib.sample_slater(N, occ, U, uniforms=u)
    check_slater_shots(U, occ, u, got)


def test_sample_slater_spinful_and_edges(lib):
    g = inputs.rng(1650)
    N = 8
    Ua, Ub = inputs.haar_unitary(N, g), inputs.haar_unitary(N, g)
    ua, ub = g.random((500, 3)), g.random((500, 2))
    ma, mb = lib.sample_slater(N, ([0, 1, 2], [0, 1]), (Ua, Ub), uniforms=(ua, ub))
    check_slater_shots(Ua, [0, 1, 2], ua, ma)
    check_slater_shots(Ub, [0, 1], ub, mb)
    # empty and full occupations
    assert masks_as_ints(lib.sample_slater(N, [], Ua, shots=5)) == [0] * 5
    full = lib.sample_slater(N, list(range(N)), Ua, shots=5)
    assert masks_as_ints(full) == [(1 << N) - 1] * 5
    # a permutation matrix puts the electrons where it sends the columns
    P = np.eye(N)[[3, 0, 6, 1, 2, 4, 5, 7]].astype(complex)
    m = masks_as_ints(lib.sample_slater(N, [0, 1], P, shots=50))
    want = sum(1 << int(np.flatnonzero(P[:, j])[0]) for j in (0, 1))
    assert set(m) == {want}
    # argument errors
    with pytest.raises(lib.FsError) as e:
        lib.sample_slater(N, [0, 0], Ua, shots=3)
    assert e.value.code == -1
    with pytest.raises(lib.FsError) as e:
        lib.sample_slater(N, [0, 1], Ua * 1.01, shots=3)
    assert e.value.code == -2
