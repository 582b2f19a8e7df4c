"""GPU parity: string tables (bit-exact) and the gates of §3.2 against the
oracle on the same seeded inputs, through the C ABI."""

import os

import numpy as np
import pytest

import oracle
from paper_2605_03123_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 2e-5}


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


def host(t):
    return t.cpu().numpy().astype(np.complex128)


SECTORS = [(1, (0, 1)), (1, (1, 1)), (2, (1, 1)), (3, (1, 2)), (4, (2, 2)), (5, (0, 3)),
           (5, (5, 2)), (6, (3, 3)), (7, (2, 5)), (8, (4, 4)), (9, (4, 5)), (10, (3, 7)),
           (12, (6, 6)), (13, (2, 6))]


# ------------------------------------------------------------------ tables
@pytest.mark.parametrize("norb", list(range(0, 13)) + [16])
def test_string_tables_bit_exact(lib, norb):
    for n in range(norb + 1):
        if norb == 0:
            continue
        got = lib.string_table(norb, n)
        ref = oracle.strings(norb, n).astype(np.uint32)
        assert np.array_equal(got, ref), (norb, n)


def test_string_table_n18_bit_exact(lib):
    assert np.array_equal(lib.string_table(18, 9), oracle.strings(18, 9).astype(np.uint32))


@pytest.mark.parametrize("norb", [1, 2, 3, 5, 8])
def test_excitation_table_bit_exact(lib, norb):
    for n in range(norb + 1):
        tab = lib.excitation_table(norb, n)
        s = oracle.strings(norb, n)
        amap = oracle.address_map(norb, n)
        for i, m in enumerate(s):
            for p in range(norb):
                for q in range(norb):
                    r = oracle.excite(int(m), p, q)
                    v = int(tab[i, p, q])
                    if r is None:
                        assert v == 0xFFFFFFFF
                    else:
                        sign, m2 = r
                        assert v & 0x7FFFFFFF == amap[m2]
                        assert (v >> 31) == (1 if sign < 0 else 0)


# ------------------------------------------------------------------- gates
@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec", SECTORS)
def test_orbital_rotation_parity(lib, dt, norb, nelec):
    g = inputs.rng(7000 + 37 * norb + nelec[0] * 5 + nelec[1])
    Ua, Ub = inputs.haar_unitary(norb, g), inputs.haar_unitary(norb, g)
    v = inputs.random_state(norb, nelec, g)
    ref = oracle.apply_orbital_rotation(v, Ua, Ub, norb, nelec)
    got = host(lib.apply_orbital_rotation(dev(v, dt), Ua, norb, nelec, U_b=Ub))
    assert np.max(np.abs(got - ref)) < TOL[dt]
    # spin-balanced call (U_b omitted)
    ref = oracle.apply_orbital_rotation(v, Ua, None, norb, nelec)
    got = host(lib.apply_orbital_rotation(dev(v, dt), Ua, norb, nelec))
    assert np.max(np.abs(got - ref)) < TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_rotation_of_hartree_fock_closed_form(lib, dt):
    w = inputs.plain_small()
    norb, nelec, U = w["norb"], w["nelec"], w["U"]
    got = host(lib.apply_orbital_rotation(dev(oracle.hartree_fock(norb, nelec), dt), U,
                                          norb, nelec))
    ref = oracle.slater_from_hf(U, None, norb, nelec)
    assert np.max(np.abs(got - ref)) < TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec", SECTORS)
def test_diag_coulomb_parity(lib, dt, norb, nelec):
    g = inputs.rng(8000 + 37 * norb + nelec[0] * 5 + nelec[1])
    Jaa = inputs.random_symmetric(norb, 1.0, g)
    Jab = g.normal(0, 1, (norb, norb))
    Jbb = inputs.random_symmetric(norb, 1.0, g)
    v = inputs.random_state(norb, nelec, g)
    ref = oracle.apply_diag_coulomb_evolution(v, Jaa, Jab, Jbb, 0.7, norb, nelec)
    got = host(lib.apply_diag_coulomb_evolution(dev(v, dt), Jaa, Jab, 0.7, norb, nelec,
                                                J_bb=Jbb))
    assert np.max(np.abs(got - ref)) < TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec", SECTORS)
def test_num_op_sum_parity(lib, dt, norb, nelec):
    g = inputs.rng(9000 + 37 * norb + nelec[0] * 5 + nelec[1])
    la, lb = g.normal(0, 1, norb), g.normal(0, 1, norb)
    v = inputs.random_state(norb, nelec, g)
    ref = oracle.apply_num_op_sum_evolution(v, la, lb, 0.9, norb, nelec)
    got = host(lib.apply_num_op_sum_evolution(dev(v, dt), la, 0.9, norb, nelec, lam_b=lb))
    assert np.max(np.abs(got - ref)) < TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_plain_small_workload(lib, dt):
    """N=8 (4,4): one Haar rotation then diagonal Coulomb at t = 0.7."""
    w = inputs.plain_small()
    norb, nelec = w["norb"], w["nelec"]
    ref = oracle.apply_orbital_rotation(w["vec"], w["U"], None, norb, nelec)
    ref = oracle.apply_diag_coulomb_evolution(ref, w["J_aa"], w["J_ab"], None, w["t"],
                                              norb, nelec)
    x = lib.apply_orbital_rotation(dev(w["vec"], dt), w["U"], norb, nelec)
    x = lib.apply_diag_coulomb_evolution(x, w["J_aa"], w["J_ab"], w["t"], norb, nelec)
    assert np.max(np.abs(host(x) - ref)) < TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec", [(17, (8, 1)), (18, (9, 1)), (18, (2, 9))])
def test_rotation_long_vectors_use_clusters(lib, dt, norb, nelec):
    """String dimensions beyond one SM's shared memory (24310, 48620): the
    sweep splits each vector over a thread-block cluster.  Whole rows of the
    result are checked against the minor-matrix definition."""
    g = inputs.rng(9500 + norb + nelec[0])
    Ua, Ub = inputs.haar_unitary(norb, g), inputs.haar_unitary(norb, g)
    v = inputs.random_state(norb, nelec, g)
    got = host(lib.apply_orbital_rotation(dev(v, dt), Ua, norb, nelec, U_b=Ub))
    Mb = oracle.minor_matrix(Ub, norb, nelec[1]) if nelec[1] <= 2 or norb < 10 else None
    da = v.shape[0]
    rows = [0, 1, da // 3, da // 2, da - 1]
    for i in rows:
        if Mb is not None:
            ra = oracle.minor_matrix_row(Ua, norb, nelec[0], i)
            ref_row = (ra @ v) @ Mb.T
            assert np.max(np.abs(got[i] - ref_row)) < TOL[dt]
        else:
            for j in (0, v.shape[1] // 2, v.shape[1] - 1):
                ref = oracle.rotated_amplitude(v, Ua, Ub, norb, nelec, i, j)
                assert abs(got[i, j] - ref) < TOL[dt]
    assert abs(np.linalg.norm(got) - 1) < (1e-12 if dt == "c128" else 1e-5)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_full_size_rotation_sampled(lib, dt):
    """N=16 (8,8), 1.66e8 amplitudes: sampled amplitudes against the minor
    definition; norm preservation; U then U^dag returns the input."""
    g = inputs.rng(2000 + 77)
    norb, nelec = 16, (8, 8)
    U = inputs.haar_unitary(norb, g)
    v = inputs.random_state(norb, nelec, g)
    x = dev(v, dt)
    lib.apply_orbital_rotation_(x, U, norb, nelec)
    got = host(x)
    for (i, j) in [(0, 0), (1, 12869), (6000, 7), (12869, 12869), (4321, 8765)]:
        ref = oracle.rotated_amplitude(v, U, None, norb, nelec, i, j)
        assert abs(got[i, j] - ref) < TOL[dt], (i, j)
    assert abs(np.linalg.norm(got) - 1) < (1e-12 if dt == "c128" else 1e-4)
    lib.apply_orbital_rotation_(x, U.conj().T, norb, nelec)
    assert np.max(np.abs(host(x) - v)) < TOL[dt]


def test_argument_errors(lib):
    norb, nelec = 4, (2, 2)
    x = dev(inputs.random_state(norb, nelec, inputs.rng(1)), "c128")
    with pytest.raises(lib.FsError) as e:
        lib.apply_orbital_rotation(x, 2 * np.eye(norb), norb, nelec)
    assert e.value.code == -2
    with pytest.raises(ValueError):
        lib.apply_orbital_rotation(x, np.eye(norb), norb, (1, 2))
    with pytest.raises(TypeError):
        lib.apply_orbital_rotation(x.to(torch.complex32) if hasattr(torch, "complex32")
                                   else x.real, np.eye(norb), norb, nelec)


# ------------------------------------------------- dense minor-matrix path
@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec", [(1, (1, 0)), (4, (2, 2)), (6, (3, 2)), (8, (4, 4)),
                                        (10, (5, 5)), (12, (6, 6)), (7, (0, 3)), (9, (9, 4)),
                                        (14, (2, 3))])
def test_minor_path_parity(lib, dt, norb, nelec):
    """psi' = M_a psi M_b^T with M[J, I] = det(U[J, I]) (§2.3), forced."""
    ctx = lib.Context(torch.cuda.current_device())
    try:
        ctx.set_rotation_path(lib.FS_ROT_MINORS)
        g = inputs.rng(13000 + 17 * norb + nelec[0])
        Ua, Ub = inputs.haar_unitary(norb, g), inputs.haar_unitary(norb, g)
        v = inputs.random_state(norb, nelec, g)
        ref = oracle.apply_orbital_rotation(v, Ua, Ub, norb, nelec)
        got = host(lib.apply_orbital_rotation(dev(v, dt), Ua, norb, nelec, U_b=Ub, ctx=ctx))
        assert np.max(np.abs(got - ref)) < TOL[dt]
    finally:
        ctx.close()


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_autotuned_rotation_path(lib, dt):
    """FS_ROT_AUTO times both methods once and keeps the faster; either way
    the result matches the oracle, on the first and on later calls."""
    ctx = lib.Context(torch.cuda.current_device())
    try:
        for norb, nelec in [(8, (4, 4)), (10, (5, 4)), (8, (4, 4))]:
            g = inputs.rng(13500 + norb)
            U = inputs.haar_unitary(norb, g)
            v = inputs.random_state(norb, nelec, g)
            ref = oracle.apply_orbital_rotation(v, U, None, norb, nelec)
            got = host(lib.apply_orbital_rotation(dev(v, dt), U, norb, nelec, ctx=ctx))
            assert np.max(np.abs(got - ref)) < TOL[dt]
    finally:
        ctx.close()


def test_minor_path_rejects_large_sectors(lib):
    ctx = lib.Context(torch.cuda.current_device())
    try:
        ctx.set_rotation_path(lib.FS_ROT_MINORS)
        x = dev(inputs.random_state(16, (8, 1), inputs.rng(3)), "c64")
        with pytest.raises(lib.FsError) as e:
            lib.apply_orbital_rotation(x, np.eye(16), 16, (8, 1), ctx=ctx)
        assert e.value.code == -7
    finally:
        ctx.close()


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("norb,nelec", [(17, (2, 3)), (20, (2, 2)), (16, (8, 1)), (24, (1, 2))])
def test_diag_coulomb_parity_wide(lib, dt, norb, nelec):
    """More than 16 orbitals: the complex64 cross term takes two k-steps of
    the tensor-core contraction."""
    g = inputs.rng(15000 + norb * 3 + nelec[0])
    Jaa = inputs.random_symmetric(norb, 1.0, g)
    Jab = g.normal(0, 1, (norb, norb))
    v = inputs.random_state(norb, nelec, g)
    ref = oracle.apply_diag_coulomb_evolution(v, Jaa, Jab, None, 0.45, norb, nelec)
    got = host(lib.apply_diag_coulomb_evolution(dev(v, dt), Jaa, Jab, 0.45, norb, nelec))
    assert np.max(np.abs(got - ref)) < TOL[dt]
