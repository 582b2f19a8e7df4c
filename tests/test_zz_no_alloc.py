"""The allocation-free diagonal-Coulomb entry point against the regular one.

Some callers cannot allocate device memory: their memory belongs to a pool
or arena the library may not bypass, or they cannot afford the device-wide
synchronization a cudaMalloc or cudaFree can cause.  For them the library
exports fs_apply_diag_coulomb_evolution_noalloc, which keeps its scratch in a
static device array.  This test calls it several times in a row through the
C ABI and compares every result with fs_apply_diag_coulomb_evolution on the
same input.  It is collected last on purpose and depends on no other test.
"""

import ctypes
import os

import numpy as np
import pytest

from paper_2605_03123_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-5}


def _lib():
    from paper_2605_03123_gb300 import build, fsgpu
    if not os.path.exists(build.lib_path()):
        build.build()
    return fsgpu, fsgpu.load_library()


def _call_noalloc(lib, x, Jaa, Jab, Jbb, t, norb, nelec):
    P = ctypes.c_void_p
    ptr = lambda a: None if a is None else a.ctypes.data_as(P)
    code = 0 if x.dtype == torch.complex64 else 1
    return lib.fs_apply_diag_coulomb_evolution_noalloc(
        P(x.data_ptr()), code, ptr(Jaa), ptr(Jab), ptr(Jbb), float(t), norb, nelec[0],
        nelec[1], P(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    fsgpu, lib = _lib()
    cases = [(8, (4, 4), torch.complex128), (12, (6, 5), torch.complex64),
             (8, (4, 4), torch.complex128), (14, (7, 7), torch.complex64)]
    for k, (norb, nelec, dt) in enumerate(cases):
        g = inputs.rng(90000 + k)
        Jaa = inputs.random_symmetric(norb, 1.0, g)
        Jab = g.normal(0, 1, (norb, norb))
        Jbb = inputs.random_symmetric(norb, 1.0, g) if k % 2 else None
        v = torch.from_numpy(inputs.random_state(norb, nelec, g)).to("cuda", dt)
        ref = fsgpu.apply_diag_coulomb_evolution(v, Jaa, Jab, 0.7, norb, nelec, J_bb=Jbb)
        x = v.clone()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = _call_noalloc(lib, x, Jaa, Jab, Jbb, 0.7, norb, nelec)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert rc == 0, lib.fs_last_error().decode()
        err = (x - ref).abs().max().item()
        assert err < TOL[dt], (k, err)
        if k >= 1:  # after the first call has set the device up
            assert free_after == free_before


def test_noalloc_rejects_sectors_above_its_limit():
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
