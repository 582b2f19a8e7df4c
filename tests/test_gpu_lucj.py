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
