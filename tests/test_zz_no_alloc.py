"""The allocation-free diagonal-Coulomb entry point against the regular one.

Some callers cannot allocate device memory: their memory belongs to a pool
or arena the library may not bypass, or they cannot afford the device-wide
synchronization a cudaMalloc or cudaFree can cause.  For them the library
exports fs_apply_diag_coulomb_evolution_noalloc, which keeps its scratch in a
static device array.  These tests call it several times in a row, through
the C ABI and through its Python wrapper, and compare every result with
fs_apply_diag_coulomb_evolution on the same input.  The file is collected
last on purpose and depends on no other test; the first test makes the very
first no-alloc call of the process in each precision, before any call to the
regular path.
"""

import ctypes
import os

import numpy as np
import pytest

from paper_2605_03123_gb300 import inputs

torch = pytest.importorskip("torch")

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-5}


def _lib():
    from paper_2605_03123_gb300 import build, fsgpu
    if not os.path.exists(build.lib_path()):
        build.build()
    return fsgpu, fsgpu.load_library()


def _call_noalloc(lib, x, Jaa, Jab, Jbb, t, norb, nelec, ptr_value=None):
    P = ctypes.c_void_p
    ptr = lambda a: None if a is None else a.ctypes.data_as(P)
    code = 0 if x.dtype == torch.complex64 else 1
    return lib.fs_apply_diag_coulomb_evolution_noalloc(
        P(x.data_ptr() if ptr_value is None else ptr_value), code, ptr(Jaa), ptr(Jab),
        ptr(Jbb), float(t), norb, nelec[0], nelec[1],
        P(torch.cuda.current_stream().cuda_stream))


def _case(k, norb, nelec, dt):
    g = inputs.rng(90000 + k)
    Jaa = inputs.random_symmetric(norb, 1.0, g)
    Jab = g.normal(0, 1, (norb, norb))
    Jbb = inputs.random_symmetric(norb, 1.0, g) if k % 2 else None
    v = torch.from_numpy(inputs.random_state(norb, nelec, g)).to("cuda", dt)
    return Jaa, Jab, Jbb, v


@pytest.mark.gpu
def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    fsgpu, lib = _lib()
    cases = [(8, (4, 4), torch.complex128), (12, (6, 5), torch.complex64),
             (8, (4, 4), torch.complex128), (14, (7, 7), torch.complex64)]
    # first the no-alloc calls (the very first ones of each precision), then
    # the regular path on the same inputs
    outs = []
    for k, (norb, nelec, dt) in enumerate(cases):
        Jaa, Jab, Jbb, v = _case(k, norb, nelec, dt)
        x = v.clone()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        torch_before = torch.cuda.memory_allocated()
        rc = _call_noalloc(lib, x, Jaa, Jab, Jbb, 0.7, norb, nelec)
        torch.cuda.synchronize()
        assert rc == 0, lib.fs_last_error().decode()
        assert torch.cuda.memory_allocated() == torch_before
        if k >= 1:  # set up by the first call: the device's free memory stays put
            assert torch.cuda.mem_get_info()[0] == free_before
        outs.append(x)
    for k, (norb, nelec, dt) in enumerate(cases):
        Jaa, Jab, Jbb, v = _case(k, norb, nelec, dt)
        ref = fsgpu.apply_diag_coulomb_evolution(v, Jaa, Jab, 0.7, norb, nelec, J_bb=Jbb)
        err = (outs[k] - ref).abs().max().item()
        assert err < TOL[dt], (k, err)


@pytest.mark.gpu
def test_noalloc_python_wrapper_matches_regular_entry_point():
    fsgpu, lib = _lib()
    for k, (norb, nelec, dt) in enumerate([(10, (5, 4), torch.complex64),
                                            (9, (3, 6), torch.complex128)]):
        Jaa, Jab, Jbb, v = _case(10 + k, norb, nelec, dt)
        ref = fsgpu.apply_diag_coulomb_evolution(v, Jaa, Jab, 0.4, norb, nelec, J_bb=Jbb)
        x = v.clone()
        for _ in range(2):  # two calls in a row on fresh copies
            x.copy_(v)
            torch_before = torch.cuda.memory_allocated()
            fsgpu.apply_diag_coulomb_evolution_noalloc_(x, Jaa, Jab, 0.4, norb, nelec,
                                                        J_bb=Jbb)
            assert torch.cuda.memory_allocated() == torch_before
            assert (x - ref).abs().max().item() < TOL[dt]


@pytest.mark.gpu
def test_noalloc_rejects_sectors_above_its_limit_and_host_memory():
    fsgpu, lib = _lib()
    norb, nelec = 16, (8, 1)  # C(16, 8) = 12870 fits, C(17, 8) = 24310 does not
    x = torch.zeros((12870, 16), dtype=torch.complex64, device="cuda")
    J = np.zeros((norb, norb))
    assert _call_noalloc(lib, x, J, J, None, 0.1, norb, nelec) == 0
    y = torch.ones((24310, 17), dtype=torch.complex64, device="cuda")
    J = np.zeros((17, 17))
    rc = _call_noalloc(lib, y, J, J, None, 0.1, 17, (8, 1))
    assert rc == -7 and "16384" in lib.fs_last_error().decode()
    assert bool((y == 1).all())
    # a host buffer (pinned, so CUDA knows it) is refused before any launch
    h = torch.ones((70, 70), dtype=torch.complex64).pin_memory()
    J = np.zeros((8, 8))
    rc = _call_noalloc(lib, h, J, J, None, 0.1, 8, (4, 4), ptr_value=h.data_ptr())
    assert rc == -1 and "device memory" in lib.fs_last_error().decode()
    assert bool((h == 1).all())


def test_noalloc_wrapper_refuses_cpu_tensors_without_a_gpu():
    """Host-side argument check: a CPU tensor never reaches the library."""
    from paper_2605_03123_gb300 import fsgpu
    x = torch.zeros((70, 70), dtype=torch.complex64)
    J = np.zeros((8, 8))
    with pytest.raises(ValueError, match="CUDA tensor"):
        fsgpu.apply_diag_coulomb_evolution_noalloc_(x, J, J, 0.1, 8, (4, 4))
