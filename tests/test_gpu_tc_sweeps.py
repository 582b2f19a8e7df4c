"""The tensor-core window steps of the complex64 Givens sweeps (tcgen05,
compound matrices of each step of six adjacent orbitals, three-pass TF32
split) against the oracle and against the CUDA-core sweeps, through the C
ABI.  The sweep engine is a context setting; every test restores it."""

import os

import numpy as np
import pytest

import oracle
from paper_2605_03123_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 2e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2605_03123_gb300 import build, fsgpu
    if not os.path.exists(build.lib_path()):
        build.build()
    fsgpu.load_library()
    return fsgpu


@pytest.fixture
def engine(lib):
    ctx = lib.context(0)

    def use(e):
        ctx.set_sweep_engine(e)
        return ctx
    yield use
    ctx.set_sweep_engine(lib.FS_SWEEP_AUTO)


def dev(v):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda", torch.complex64)


def host(t):
    return t.cpu().numpy().astype(np.complex128)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# every class of a six-orbital window (m = 1 .. 5), ragged tiles, many
# vectors per CTA, electron counts near 0 and N, a 16-orbital vector
SECTORS = [(6, (3, 3)), (6, (1, 5)), (7, (2, 5)), (8, (4, 4)), (9, (4, 5)), (10, (3, 7)),
           (11, (5, 2)), (12, (6, 6)), (13, (2, 6)), (14, (7, 7)), (16, (8, 1))]


@pytest.mark.parametrize("norb,nelec", SECTORS)
def test_tc_rotation_against_oracle(lib, engine, norb, nelec):
    ctx = engine(lib.FS_SWEEP_TENSOR)
    g = inputs.rng(21000 + 17 * norb + nelec[0])
    Ua, Ub = inputs.haar_unitary(norb, g), inputs.haar_unitary(norb, g)
    v = inputs.random_state(norb, nelec, g)
    ref = oracle.apply_orbital_rotation(v, Ua, Ub, norb, nelec)
    x = dev(v)
    lib.apply_orbital_rotation_(x, Ua, norb, nelec, U_b=Ub, ctx=ctx)
    assert ctx.sync_status() == 0
    err = np.max(np.abs(host(x) - ref))
    assert err < TOL64, err
    assert err < 1e-4 * np.max(np.abs(ref)), err


def test_tc_rotation_of_hartree_fock_closed_form(lib, engine):
    """U|HF> from a state (not the closed-form shortcut): every amplitude is
    a product of two minors (§2.4), here with amplitudes of order one."""
    ctx = engine(lib.FS_SWEEP_TENSOR)
    norb, nelec = 10, (5, 4)
    U = inputs.haar_unitary(norb, inputs.rng(21500))
    x = dev(oracle.hartree_fock(norb, nelec))
    lib.apply_orbital_rotation_(x, U, norb, nelec, ctx=ctx)
    ref = oracle.slater_from_hf(U, None, norb, nelec)
    assert np.max(np.abs(host(x) - ref)) < TOL64
    assert ctx.sync_status() == 0


def test_tc_matches_cuda_core_at_full_size(lib, engine):
    """N=16 (8,8), 1.66e8 amplitudes: the two engines on the same rotation."""
    norb, nelec = 16, (8, 8)
    v = inputs.device_state(norb, nelec, 21600, torch.complex64)
    U = inputs.haar_unitary(norb, inputs.rng(21601))
    out = {}
    for e in (lib.FS_SWEEP_CUDA_CORE, lib.FS_SWEEP_TENSOR):
        ctx = engine(e)
        x = v.clone()
        lib.apply_orbital_rotation_(x, U, norb, nelec, ctx=ctx)
        assert ctx.sync_status() == 0
        out[e] = x
    d = float((out[lib.FS_SWEEP_CUDA_CORE] - out[lib.FS_SWEEP_TENSOR]).abs().max().item())
    scale = float(out[lib.FS_SWEEP_CUDA_CORE].abs().max().item())
    assert d < 1e-3 * scale, (d, scale)


@pytest.mark.parametrize("norb,nelec,n_reps,from_hf", [(8, (4, 4), 2, True), (9, (3, 5), 1, False),
                                                       (12, (6, 6), 4, True)])
def test_tc_lucj_forward_and_vjp_against_oracle(lib, engine, norb, nelec, n_reps, from_hf):
    ctx = engine(lib.FS_SWEEP_TENSOR)
    if (norb, n_reps) == (12, 4):
        w = inputs.lucj_small()
        K, Jaa, Jab, v, c = w["K"], w["J_aa"], w["J_ab"], None, w["cot"]
    else:
        g = inputs.rng(22000 + norb)
        K = np.array([inputs.random_antihermitian(norb, 0.5, g) for _ in range(n_reps)])
        Jaa = np.array([inputs.random_symmetric(norb, 0.5, g) for _ in range(n_reps)])
        Jab = np.array([g.normal(0, 0.5, (norb, norb)) for _ in range(n_reps)])
        v = None if from_hf else inputs.random_state(norb, nelec, g)
        c = inputs.random_state(norb, nelec, g)
    ref = oracle.lucj_forward(K, Jaa, Jab, norb, nelec, vec=v)
    rK, rJa, rJb, rv = oracle.lucj_vjp(K, Jaa, Jab, c, norb, nelec, vec=v)
    start = oracle.hartree_fock(norb, nelec) if from_hf else v
    x = dev(start)
    lib.lucj_forward_(x, K, Jaa, Jab, norb, nelec, from_hf=from_hf, ctx=ctx)
    assert np.max(np.abs(host(x) - ref)) < TOL64
    y = dev(c)
    dK, dJa, dJb = lib.lucj_vjp_(x, y, K, Jaa, Jab, norb, nelec, from_hf=from_hf, ctx=ctx)
    assert ctx.sync_status() == 0
    for a, b in ((dK, rK), (dJa, rJa), (dJb, rJb)):
        assert _rel(a, b) < 2e-4
        assert np.max(np.abs(a - b)) < 1e-3 * np.max(np.abs(b))
    assert np.max(np.abs(host(x) - start)) < TOL64
    if not from_hf:
        assert np.max(np.abs(host(y) - rv)) < TOL64


def test_tc_reverse_on_cluster_pairs_at_full_size(lib, engine):
    """N=16 (8,8), two layers: the reverse sweeps carry two states, 206 KB
    per vector, so the tensor-core path splits each vector over a pair of
    CTAs (the strings with and without the top orbital); the forward state,
    the recovered input, dL/dpsi_in and the gradients against the CUDA-core
    engine."""
    w = inputs.lucj_layers(16, (8, 8), 2, 0.5, 0.3, 2000 + 13, with_cot=False)
    norb, nelec = 16, (8, 8)
    v0 = inputs.device_state(norb, nelec, 22500, torch.complex64)
    c0 = inputs.device_state(norb, nelec, 22501, torch.complex64)
    res = {}
    for e in (lib.FS_SWEEP_CUDA_CORE, lib.FS_SWEEP_TENSOR):
        ctx = engine(e)
        x, y = v0.clone(), c0.clone()
        lib.lucj_forward_(x, w["K"], w["J_aa"], w["J_ab"], norb, nelec, ctx=ctx)
        out = x.clone()
        g = lib.lucj_vjp_(x, y, w["K"], w["J_aa"], w["J_ab"], norb, nelec, ctx=ctx)
        assert ctx.sync_status() == 0
        assert float((x - v0).abs().max().item()) < TOL64
        res[e] = (out, y, g)
    (o1, y1, g1), (o2, y2, g2) = res[lib.FS_SWEEP_CUDA_CORE], res[lib.FS_SWEEP_TENSOR]
    assert float((o1 - o2).abs().max().item()) < 1e-3 * float(o1.abs().max().item())
    assert float((y1 - y2).abs().max().item()) < 1e-3 * float(y1.abs().max().item())
    for a, b in zip(g2, g1):
        assert _rel(a, b) < 1e-4
