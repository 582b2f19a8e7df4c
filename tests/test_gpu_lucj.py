"""GPU parity of the LUCJ forward pass (§4.3, §4.5.1) and its VJP against
the oracle, through the C ABI."""

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


@pytest.fixture(scope="module")
def lucj_small_ref():
    w = inputs.lucj_small()
    ref = oracle.lucj_forward(w["K"], w["J_aa"], w["J_ab"], w["norb"], w["nelec"])
    return w, ref


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_lucj_forward_from_hf(lib, dt, lucj_small_ref):
    """N=12 (6,6), 4 repetitions from Hartree-Fock."""
    w, ref = lucj_small_ref
    norb, nelec = w["norb"], w["nelec"]
    x = dev(np.zeros((924, 924)), dt)
    lib.lucj_forward_(x, w["K"], w["J_aa"], w["J_ab"], norb, nelec, from_hf=True)
    assert np.max(np.abs(host(x) - ref)) < TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec,n_reps", [(6, (3, 2), 3), (7, (1, 4), 2), (5, (5, 0), 1),
                                               (8, (4, 4), 1)])
def test_lucj_forward_from_state(lib, dt, norb, nelec, n_reps):
    g = inputs.rng(11000 + norb * 10 + n_reps)
    K = np.array([inputs.random_antihermitian(norb, 0.5, g) for _ in range(n_reps)])
    Jaa = np.array([inputs.random_symmetric(norb, 0.5, g) for _ in range(n_reps)])
    Jab = np.array([g.normal(0, 0.5, (norb, norb)) for _ in range(n_reps)])
    v = inputs.random_state(norb, nelec, g)
    ref = oracle.lucj_forward(K, Jaa, Jab, norb, nelec, vec=v)
    x = dev(v, dt)
    lib.lucj_forward_(x, K, Jaa, Jab, norb, nelec)
    assert np.max(np.abs(host(x) - ref)) < TOL[dt]


def test_lucj_zero_reps_from_hf(lib):
    x = dev(inputs.random_state(6, (3, 3), inputs.rng(5)), "c128")
    z = np.zeros((0, 6, 6))
    lib.lucj_forward_(x, z, z, z, 6, (3, 3), from_hf=True)
    assert np.array_equal(host(x), oracle.hartree_fock(6, (3, 3)))


# ---------------------------------------------------------------------- VJP
def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _elementwise(a, b):
    """max |a - b| over the entries, relative to max |b|: a wrong small entry
    (an off-pattern coupling, say) cannot hide under the norm of the rest."""
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _small_case(norb, nelec, n_reps, seed, from_hf):
    g = inputs.rng(seed)
    K = np.array([inputs.random_antihermitian(norb, 0.5, g) for _ in range(n_reps)])
    Jaa = np.array([inputs.random_symmetric(norb, 0.5, g) for _ in range(n_reps)])
    Jab = np.array([g.normal(0, 0.5, (norb, norb)) for _ in range(n_reps)])
    v = None if from_hf else inputs.random_state(norb, nelec, g)
    c = inputs.random_state(norb, nelec, g)
    return K, Jaa, Jab, v, c


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec,n_reps,from_hf", [
    (6, (3, 2), 2, False), (5, (2, 3), 3, False), (6, (3, 3), 2, True), (4, (4, 1), 2, False),
    (2, (1, 1), 1, False), (7, (0, 3), 2, False), (8, (4, 4), 1, True)])
def test_lucj_vjp_small_against_oracle(lib, dt, norb, nelec, n_reps, from_hf):
    K, Jaa, Jab, v, c = _small_case(norb, nelec, n_reps, 12000 + norb * 7 + n_reps, from_hf)
    rK, rJa, rJb, rv = oracle.lucj_vjp(K, Jaa, Jab, c, norb, nelec, vec=v)
    x = dev(oracle.hartree_fock(norb, nelec) if from_hf else v, dt)
    lib.lucj_forward_(x, K, Jaa, Jab, norb, nelec, from_hf=from_hf)
    cg = dev(c, dt)
    dK, dJa, dJb = lib.lucj_vjp_(x, cg, K, Jaa, Jab, norb, nelec, from_hf=from_hf)
    tol = 1e-11 if dt == "c128" else 2e-4
    assert _rel(dK, rK) < tol and _rel(dJa, rJa) < tol and _rel(dJb, rJb) < tol
    tel = 1e-6 if dt == "c128" else 1e-3
    for a, b in ((dK, rK), (dJa, rJa), (dJb, rJb)):
        assert _elementwise(a, b) < tel
    v_in = oracle.hartree_fock(norb, nelec) if from_hf else v
    assert np.max(np.abs(host(x) - v_in)) < TOL[dt]            # uncomputed input
    if not from_hf:
        assert np.max(np.abs(host(cg) - rv)) < TOL[dt]         # dL/dpsi_in


@pytest.fixture(scope="module")
def lucj_small_vjp_ref(lucj_small_ref):
    w, ref = lucj_small_ref
    r = oracle.lucj_vjp(w["K"], w["J_aa"], w["J_ab"], w["cot"], w["norb"], w["nelec"])
    return w, ref, r


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_lucj_vjp_n12_against_oracle(lib, dt, lucj_small_vjp_ref):
    """N=12 (6,6), 4 repetitions from Hartree-Fock: gradients within 1e-6
    relative of the oracle's stored-state reverse mode in complex128."""
    w, ref, (rK, rJa, rJb, rv) = lucj_small_vjp_ref
    norb, nelec = w["norb"], w["nelec"]
    x = dev(np.zeros((924, 924)), dt)
    lib.lucj_forward_(x, w["K"], w["J_aa"], w["J_ab"], norb, nelec, from_hf=True)
    cg = dev(w["cot"], dt)
    dK, dJa, dJb = lib.lucj_vjp_(x, cg, w["K"], w["J_aa"], w["J_ab"], norb, nelec, from_hf=True)
    tol = 1e-6 if dt == "c128" else 1e-3
    for a, b in ((dK, rK), (dJa, rJa), (dJb, rJb)):
        assert _rel(a, b) < tol
        assert _elementwise(a, b) < tol
    assert np.max(np.abs(host(x) - oracle.hartree_fock(norb, nelec))) < TOL[dt]


def test_lucj_vjp_n12_central_differences(lib, lucj_small_ref):
    """Central differences (step 1e-6) of the GPU forward pass in complex128
    along random anti-Hermitian / symmetric directions, against the VJP."""
    w, _ = lucj_small_ref
    norb, nelec = w["norb"], w["nelec"]
    K, Jaa, Jab, cot = w["K"], w["J_aa"], w["J_ab"], w["cot"]

    def loss(K_, Ja_, Jb_):
        x = dev(np.zeros((924, 924)), "c128")
        lib.lucj_forward_(x, K_, Ja_, Jb_, norb, nelec, from_hf=True)
        return float(np.real(np.vdot(cot, host(x))))

    x = dev(np.zeros((924, 924)), "c128")
    lib.lucj_forward_(x, K, Jaa, Jab, norb, nelec, from_hf=True)
    dK, dJa, dJb = lib.lucj_vjp_(x, dev(cot, "c128"), K, Jaa, Jab, norb, nelec, from_hf=True)
    g = inputs.rng(31337)
    h = 1e-6
    for trial in range(3):
        eK = np.array([inputs.random_antihermitian(norb, 1.0, g) for _ in range(len(K))])
        eA = np.array([inputs.random_symmetric(norb, 1.0, g) for _ in range(len(K))])
        eB = np.array([g.normal(0, 1, (norb, norb)) for _ in range(len(K))])
        fd = (loss(K + h * eK, Jaa + h * eA, Jab + h * eB)
              - loss(K - h * eK, Jaa - h * eA, Jab - h * eB)) / (2 * h)
        an = (np.sum(dK.real * eK.real + dK.imag * eK.imag) + np.sum(dJa * eA)
              + np.sum(dJb * eB))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (trial, fd, an)


def test_lucj_vjp_n16_central_differences(lib):
    """N=16 (8,8), complex128, 2 layers of the metric workload from a random
    state: the state (2.65 GB) exceeds L2, so the reverse alpha sweeps run on
    transposed copies; central differences (step 1e-5) along random
    directions against the VJP, in all parameters, with the loss reduced on
    the device in row blocks."""
    w = inputs.lucj_layers(16, (8, 8), 2, 0.5, 0.3, 2000 + 7, with_cot=False)
    norb, nelec = 16, (8, 8)
    K, Jaa, Jab = w["K"], w["J_aa"], w["J_ab"]
    v0 = inputs.device_state(norb, nelec, 41, torch.complex128)
    cot = inputs.device_state(norb, nelec, 42, torch.complex128)

    def loss(K_, Ja_, Jb_):
        x = v0.clone()
        lib.lucj_forward_(x, K_, Ja_, Jb_, norb, nelec)
        return _vdot_rows(cot, x).real

    x = v0.clone()
    lib.lucj_forward_(x, K, Jaa, Jab, norb, nelec)
    cg = cot.clone()
    dK, dJa, dJb = lib.lucj_vjp_(x, cg, K, Jaa, Jab, norb, nelec)
    assert float((x - v0).abs().max().item()) < 1e-10
    g = inputs.rng(31338)
    h = 1e-5
    for trial in range(2):
        eK = np.array([inputs.random_antihermitian(norb, 1.0, g) for _ in range(len(K))])
        eA = np.array([inputs.random_symmetric(norb, 1.0, g) for _ in range(len(K))])
        eB = np.array([g.normal(0, 1, (norb, norb)) for _ in range(len(K))])
        fd = (loss(K + h * eK, Jaa + h * eA, Jab + h * eB)
              - loss(K - h * eK, Jaa - h * eA, Jab - h * eB)) / (2 * h)
        an = (np.sum(dK.real * eK.real + dK.imag * eK.imag) + np.sum(dJa * eA)
              + np.sum(dJb * eB))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (trial, fd, an)
    # the mixed-coupling gradient alone (the part that comes out transposed)
    eB = np.array([g.normal(0, 1, (norb, norb)) for _ in range(len(K))])
    fd = (loss(K, Jaa, Jab + h * eB) - loss(K, Jaa, Jab - h * eB)) / (2 * h)
    an = np.sum(dJb * eB)
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (fd, an)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_lucj_vjp_full_size_properties(lib, dt):
    """N=16 (8,8), 2 layers of the metric workload: the reverse sweeps recover
    the input state, and dL/dpsi_in = C^dag g satisfies <C^dag g, psi_in> =
    <g, psi_out> with unit norm (C unitary)."""
    w = inputs.lucj_layers(16, (8, 8), 2, 0.5, 0.3, 2000 + 5)
    norb, nelec = 16, (8, 8)
    x = dev(w["vec"], dt)
    lib.lucj_forward_(x, w["K"], w["J_aa"], w["J_ab"], norb, nelec)
    out = host(x)
    cg = dev(w["cot"], dt)
    dK, dJa, dJb = lib.lucj_vjp_(x, cg, w["K"], w["J_aa"], w["J_ab"], norb, nelec)
    rec, dv = host(x), host(cg)
    tol = TOL[dt] if dt == "c128" else 2e-5
    assert np.max(np.abs(rec - w["vec"])) < tol
    lhs, rhs = np.vdot(dv, w["vec"]), np.vdot(w["cot"], out)
    assert abs(lhs - rhs) < (1e-11 if dt == "c128" else 1e-4)
    assert abs(np.linalg.norm(dv) - 1) < (1e-11 if dt == "c128" else 1e-4)
    assert np.all(np.isfinite(dK)) and np.all(np.isfinite(dJa)) and np.all(np.isfinite(dJb))


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_lucj_forward_full_size_matches_gate_composition(lib, dt):
    """N=16 (8,8), 2 layers: the LUCJ forward pass (merged rotations, the
    diagonal-Coulomb gates fused into sweeps, the layouts alternating between
    the state and its transpose) equals, element by element, the literal
    composition U(U_k) D(J_k) U(U_k)^dag of the separate gate calls."""
    from scipy.linalg import expm
    w = inputs.lucj_layers(16, (8, 8), 2, 0.5, 0.3, 2000 + 9, with_cot=False)
    norb, nelec = 16, (8, 8)
    x = dev(w["vec"], dt)
    lib.lucj_forward_(x, w["K"], w["J_aa"], w["J_ab"], norb, nelec)
    y = dev(w["vec"], dt)
    for K, Ja, Jb in zip(w["K"], w["J_aa"], w["J_ab"]):
        U = expm(K)
        lib.apply_orbital_rotation_(y, U.conj().T, norb, nelec)
        lib.apply_diag_coulomb_evolution_(y, Ja, Jb, 1.0, norb, nelec)
        lib.apply_orbital_rotation_(y, U, norb, nelec)
    err = float((x.to(torch.complex128) - y.to(torch.complex128)).abs().max())
    assert err < TOL[dt], err


def test_autograd_function_matches_oracle(lib):
    from paper_2605_03123_gb300.autograd import lucj
    norb, nelec, n_reps = 6, (3, 2), 2
    K, Jaa, Jab, v, c = _small_case(norb, nelec, n_reps, 777, False)
    rK, rJa, rJb, rv = oracle.lucj_vjp(K, Jaa, Jab, c, norb, nelec, vec=v)
    vt = dev(v, "c128").requires_grad_(True)
    Kt = torch.from_numpy(K).requires_grad_(True)
    At = torch.from_numpy(Jaa).requires_grad_(True)
    Bt = torch.from_numpy(Jab).requires_grad_(True)
    out = lucj(vt, Kt, At, Bt, norb, nelec)
    loss = torch.real(torch.vdot(dev(c, "c128").flatten(), out.flatten()))
    loss.backward()
    assert np.max(np.abs(Kt.grad.numpy() - rK)) < 1e-11
    assert np.max(np.abs(At.grad.numpy() - rJa)) < 1e-11
    assert np.max(np.abs(Bt.grad.numpy() - rJb)) < 1e-11
    assert np.max(np.abs(host(vt.grad) - rv)) < 1e-12


def test_lucj_vjp_cluster_path_against_oracle(lib):
    """complex128, N=16 (8,1): an alpha vector of 12870 strings with both
    states is 412 KB, so the reverse sweeps split it over a 2-CTA cluster
    (distributed shared memory); gradients against the oracle."""
    norb, nelec, n_reps = 16, (8, 1), 1
    K, Jaa, Jab, v, c = _small_case(norb, nelec, n_reps, 14000, False)
    rK, rJa, rJb, rv = oracle.lucj_vjp(K, Jaa, Jab, c, norb, nelec, vec=v)
    x = dev(v, "c128")
    lib.lucj_forward_(x, K, Jaa, Jab, norb, nelec)
    cg = dev(c, "c128")
    dK, dJa, dJb = lib.lucj_vjp_(x, cg, K, Jaa, Jab, norb, nelec)
    assert _rel(dK, rK) < 1e-10 and _rel(dJa, rJa) < 1e-10 and _rel(dJb, rJb) < 1e-10
    for a, b in ((dK, rK), (dJa, rJa), (dJb, rJb)):
        assert _elementwise(a, b) < 1e-6
    assert np.max(np.abs(host(cg) - rv)) < 1e-12
    assert np.max(np.abs(host(x) - v)) < 1e-12


@pytest.fixture(scope="module")
def n18_cluster_case():
    """N=18 (9,1): 48620 alpha strings, so the alpha sweeps run on clusters
    of 2 (complex64 forward), 4 (complex64 reverse, complex128 forward) and
    8 CTAs (complex128 reverse), each rank holding the strings of one
    occupation pattern of the top orbitals."""
    norb, nelec = 18, (9, 1)
    K, Jaa, Jab, v, c = _small_case(norb, nelec, 1, 14500, False)
    return (norb, nelec, K, Jaa, Jab, v, c,
            oracle.lucj_forward(K, Jaa, Jab, norb, nelec, vec=v),
            oracle.lucj_vjp(K, Jaa, Jab, c, norb, nelec, vec=v))


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_lucj_blocked_clusters_against_oracle(lib, dt, n18_cluster_case):
    norb, nelec, K, Jaa, Jab, v, c, out, (rK, rJa, rJb, rv) = n18_cluster_case
    x = dev(v, dt)
    lib.lucj_forward_(x, K, Jaa, Jab, norb, nelec)
    assert np.max(np.abs(host(x) - out)) < TOL[dt]
    cg = dev(c, dt)
    dK, dJa, dJb = lib.lucj_vjp_(x, cg, K, Jaa, Jab, norb, nelec)
    tg = 1e-10 if dt == "c128" else 2e-4
    assert _rel(dK, rK) < tg and _rel(dJa, rJa) < tg and _rel(dJb, rJb) < tg
    te = 1e-6 if dt == "c128" else 1e-3
    for a, b in ((dK, rK), (dJa, rJa), (dJb, rJb)):
        assert _elementwise(a, b) < te
    assert np.max(np.abs(host(cg) - rv)) < TOL[dt]
    assert np.max(np.abs(host(x) - v)) < TOL[dt]


def _vdot_rows(a, b, rows=4096):
    """<a, b> over row blocks (one cuBLAS dot is limited to 2^31 elements)."""
    return sum(complex(torch.vdot(a[i:i + rows].flatten(), b[i:i + rows].flatten()).item())
               for i in range(0, a.shape[0], rows))


def test_lucj_norb18_properties(lib):
    """N=18 (9,9), one repetition from Hartree-Fock (2.36e9 amplitudes; the
    sweeps run on 4- and 8-CTA clusters): unit norm, the recovered input is
    Hartree-Fock, <g, psi_out> equals the conjugate HF amplitude of
    dL/dpsi_in, and complex64 agrees with complex128 (forward state and
    gradients)."""
    w = inputs.largest_state()
    N, ne = w["norb"], w["nelec"]
    K, Ja, Jb = w["K"], w["J_aa"], w["J_ab"]
    res = {}
    for dt in (torch.complex64, torch.complex128):
        cot0 = inputs.device_state(N, ne, w["cot_seed"], torch.complex64).to(dt)
        x = torch.zeros_like(cot0)
        lib.lucj_forward_(x, K, Ja, Jb, N, ne, from_hf=True)
        assert abs(float(torch.linalg.vector_norm(x).item()) - 1) < 1e-4
        lhs = _vdot_rows(cot0, x)
        fwd = x[:64, :].clone(), x[-64:, :].clone()
        cg = cot0.clone()
        del cot0
        g = lib.lucj_vjp_(x, cg, K, Ja, Jb, N, ne, from_hf=True)
        assert abs(float(x[0, 0].real.item()) - 1) < 1e-5
        x[0, 0] = 0
        assert float(x.abs().max().item()) < 1e-5
        rhs = complex(cg[0, 0].item()).conjugate()
        assert abs(lhs - rhs) < 1e-4
        res[dt] = fwd, g
        del x, cg
        torch.cuda.empty_cache()
    (f64a, f64b), g64 = res[torch.complex64]
    (f128a, f128b), g128 = res[torch.complex128]
    assert float((f64a.to(torch.complex128) - f128a).abs().max().item()) < 2e-5
    assert float((f64b.to(torch.complex128) - f128b).abs().max().item()) < 2e-5
    for a, b in zip(g64, g128):
        assert _rel(a, b) < 1e-3
