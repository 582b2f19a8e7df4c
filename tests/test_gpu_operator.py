"""Molecular-Hamiltonian action on the GPU against the oracle, element by
element, in one block and in many ragged blocks; properties at larger
sizes."""

import os

import numpy as np
import pytest

import oracle
from paper_2605_03123_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def _tensors(N, g, symmetric=True):
    A = g.normal(0, 1, (N, N))
    B = g.normal(0, 0.5, (N, N, N, N))
    if not symmetric:
        return A, B
    h2 = (B + B.transpose(1, 0, 3, 2) + B.transpose(2, 3, 0, 1) + B.transpose(3, 2, 1, 0)) / 4
    return (A + A.T) / 2, h2


# tolerance relative to the largest output entry: c128 rounding of ~N^4
# terms, c64 FP32 GEMMs over 2 N^2 terms
REL = {"c128": 1e-12, "c64": 2e-5}


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,nelec,symmetric", [
    (4, (2, 1), False), (5, (2, 3), True), (6, (3, 3), False), (7, (2, 4), True), (8, (4, 4), True)])
@pytest.mark.parametrize("workspace", [0, 350000])
def test_molecular_hamiltonian_parity(lib, dt, norb, nelec, symmetric, workspace):
    g = inputs.rng(1200 + 10 * norb + nelec[0])
    h1, h2 = _tensors(norb, g, symmetric)
    v = inputs.random_state(norb, nelec, g)
    ref = oracle.apply_molecular_hamiltonian(v, h1, h2, norb, nelec, constant=0.25)
    got = host(lib.apply_molecular_hamiltonian(dev(v, dt), h1, h2, norb, nelec, constant=0.25,
                                               workspace_bytes=workspace))
    scale = max(1.0, float(np.max(np.abs(ref))))
    assert np.max(np.abs(got - ref)) < REL[dt] * scale


def test_molecular_hamiltonian_edge_sectors(lib):
    g = inputs.rng(1290)
    for norb, nelec in [(5, (0, 2)), (5, (5, 1)), (6, (1, 0)), (4, (0, 0))]:
        h1, h2 = _tensors(norb, g)
        v = inputs.random_state(norb, nelec, g)
        ref = oracle.apply_molecular_hamiltonian(v, h1, h2, norb, nelec, constant=-0.5)
        got = host(lib.apply_molecular_hamiltonian(dev(v, "c128"), h1, h2, norb, nelec,
                                                   constant=-0.5))
        assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, float(np.max(np.abs(ref))))


@pytest.mark.parametrize("norb,nelec", [(12, (6, 6)), (16, (4, 4))])
def test_molecular_hamiltonian_properties_at_scale(lib, norb, nelec):
    """Hermitian tensors: <u|H w> = <H u|w> and a real energy; complex64
    follows complex128; blocked and unblocked agree."""
    g = inputs.rng(1300 + norb)
    h1, h2 = _tensors(norb, g)
    u = inputs.device_state(norb, nelec, 3, torch.complex128)
    w = inputs.device_state(norb, nelec, 4, torch.complex128)
    Hw = lib.apply_molecular_hamiltonian(w, h1, h2, norb, nelec)
    Hu = lib.apply_molecular_hamiltonian(u, h1, h2, norb, nelec)
    lhs = complex(torch.vdot(u.flatten(), Hw.flatten()).item())
    rhs = complex(torch.vdot(Hu.flatten(), w.flatten()).item())
    scale = float(torch.linalg.vector_norm(Hw).item())
    assert abs(lhs - rhs) < 1e-11 * scale
    e = complex(torch.vdot(w.flatten(), Hw.flatten()).item())
    assert abs(e.imag) < 1e-11 * scale
    Hb = lib.apply_molecular_hamiltonian(w, h1, h2, norb, nelec, workspace_bytes=64 << 20)
    assert float((Hb - Hw).abs().max().item()) < 1e-11 * scale
    H64 = lib.apply_molecular_hamiltonian(w.to(torch.complex64), h1, h2, norb, nelec)
    d = float((H64.to(torch.complex128) - Hw).abs().max().item())
    assert d < 2e-5 * float(Hw.abs().max().item())
