"""Thin Python binding of libfsgpu.so (include/fsgpu.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch supplies device memory and the current stream.  There is
no CPU fallback: if the library is missing or no GPU is present, calls raise.

State tensors are complex64 or complex128 CUDA tensors of shape
(dim_a, dim_b), contiguous, in the address convention of the C header.
Functional calls return a new tensor (the paper's style, §4.1); the `*_`
variants update in place.
"""

import ctypes
import os
import threading

import numpy as np

from .build import lib_path

FS_C64, FS_C128 = 0, 1
FS_ROT_AUTO, FS_ROT_GIVENS, FS_ROT_MINORS = 0, 1, 2
FS_SWEEP_AUTO, FS_SWEEP_CUDA_CORE, FS_SWEEP_TENSOR = 0, 1, 2

STATUS = {0: "FS_OK", -1: "FS_ERR_ARG", -2: "FS_ERR_NOT_UNITARY", -3: "FS_ERR_NOMEM",
          -4: "FS_ERR_CUDA", -5: "FS_ERR_TIMEOUT", -6: "FS_ERR_BOUNDS",
          -7: "FS_ERR_UNSUPPORTED"}


class FsError(RuntimeError):
    def __init__(self, func, code, msg):
        super().__init__("%s failed: %s (%d): %s" % (func, STATUS.get(code, "?"), code, msg))
        self.code = code


class LUCJ(ctypes.Structure):
    _fields_ = [("norb", ctypes.c_int), ("n_alpha", ctypes.c_int), ("n_beta", ctypes.c_int),
                ("n_reps", ctypes.c_int), ("K", ctypes.c_void_p), ("J_aa", ctypes.c_void_p),
                ("J_ab", ctypes.c_void_p), ("from_hf", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_I64 = ctypes.c_int64
SIGNATURES = {
    "fs_create": [ctypes.POINTER(_P), _I],
    "fs_destroy": [_P],
    "fs_last_error": [],
    "fs_sync_status": [_P, _P],
    "fs_set_rotation_path": [_P, _I],
    "fs_profile_start": [_P],
    "fs_profile_stop": [_P, ctypes.c_char_p, _I64],
    "fs_string_table": [_P, _I, _I, _P, _I64],
    "fs_excitation_table": [_P, _I, _I, _P, _I64],
    "fs_apply_orbital_rotation": [_P, _P, _I, _P, _P, _I, _I, _I, _P],
    "fs_apply_num_op_sum_evolution": [_P, _P, _I, _P, _P, _D, _I, _I, _I, _P],
    "fs_apply_diag_coulomb_evolution": [_P, _P, _I, _P, _P, _P, _D, _I, _I, _I, _P],
    "fs_apply_diag_coulomb_evolution_noalloc": [_P, _I, _P, _P, _P, _D, _I, _I, _I, _P],
    "fs_lucj_forward": [_P, ctypes.POINTER(LUCJ), _P, _I, _P],
    "fs_lucj_vjp": [_P, ctypes.POINTER(LUCJ), _P, _P, _I, _P, _P, _P, _P],
    "fs_apply_num_interaction": [_P, _P, _I, _D, _I, _I, _I, _I, _I, _P],
    "fs_apply_num_num_interaction": [_P, _P, _I, _D, _I, _I, _I, _I, _I, _I, _I, _P],
    "fs_apply_givens_rotation": [_P, _P, _I, _D, _I, _I, _I, _I, _I, _I, _P],
    "fs_apply_tunneling_interaction": [_P, _P, _I, _D, _I, _I, _I, _I, _I, _I, _P],
    "fs_apply_quad_ham_evolution": [_P, _P, _I, _P, _P, _D, _I, _I, _I, _P],
    "fs_simulate_trotter_double_factorized": [_P, _P, _I, _P, _I, _P, _P, _D, _I, _I, _I, _I,
                                              _I, _P],
    "fs_simulate_trotter_diag_coulomb": [_P, _P, _I, _P, _P, _P, _P, _D, _I, _I, _I, _I, _I,
                                         _P],
    "fs_apply_molecular_hamiltonian": [_P, _P, _P, _I, _P, _P, _D, _I64, _I, _I, _I, _P],
    "fs_sample_state": [_P, _P, _I, _I, _I, _I, _P, _I64, _P, _P],
    "fs_sample_slater": [_P, _P, _I, _P, _I, _P, _I64, _P, _P],
    "fs_set_sweep_engine": [_P, _I],
    "fs_set_batch_tuning": [_P, _I],
    "fs_tuning_report": [_P, _P, _I64],
    "fs_measure_fp32_fma": [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "fs_lucj_batch": [_P, _I, ctypes.POINTER(LUCJ), ctypes.POINTER(_P), ctypes.POINTER(_P), _I,
                      _I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _P],
}

_lib = None
_lib_lock = threading.Lock()


def load_library(path=None):
    """Load libfsgpu.so (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        p = path or lib_path()
        if not os.path.exists(p):
            raise FsError("load_library", -7, "%s is missing; build it with "
                          "paper_2605_03123_gb300.build.build()" % p)
        lib = ctypes.CDLL(p)
        for name, args in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name == "fs_last_error" else ctypes.c_int
        _lib = lib
        return lib


def _check(name, rc):
    if rc != 0:
        raise FsError(name, rc, load_library().fs_last_error().decode())


class Context:
    """A library context on one CUDA device (tables and scratch live here)."""

    def __init__(self, device=0):
        lib = load_library()
        h = _P()
        _check("fs_create", lib.fs_create(ctypes.byref(h), int(device)))
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            _check("fs_destroy", load_library().fs_destroy(self.handle))
            self.handle = None

    def set_rotation_path(self, path):
        _check("fs_set_rotation_path", load_library().fs_set_rotation_path(self.handle, int(path)))

    def set_sweep_engine(self, engine):
        _check("fs_set_sweep_engine", load_library().fs_set_sweep_engine(self.handle, int(engine)))

    def set_batch_tuning(self, on):
        _check("fs_set_batch_tuning", load_library().fs_set_batch_tuning(self.handle, int(bool(on))))

    def tuning_report(self):
        """The batched-sweep autotuner's choices, one dict per sector and sweep kind."""
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        _check("fs_tuning_report", load_library().fs_tuning_report(self.handle, buf, len(buf)))
        return json.loads(buf.value.decode())

    def sync_status(self, stream=None):
        """The device status word (FS_OK, or FS_ERR_TIMEOUT / FS_ERR_BOUNDS
        from a kernel's bounded checks), reset to FS_OK."""
        return load_library().fs_sync_status(self.handle, _stream_ptr(stream))

    def profile_start(self):
        _check("fs_profile_start", load_library().fs_profile_start(self.handle))

    def profile_stop(self):
        """{step: (records, total_ms, kernel_launches)} since profile_start."""
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        _check("fs_profile_stop", load_library().fs_profile_stop(self.handle, buf, len(buf)))
        return {k: tuple(v) for k, v in json.loads(buf.value.decode()).items()}


_contexts = {}


def context(device=None):
    import torch
    if device is None:
        device = torch.cuda.current_device()
    if device not in _contexts:
        _contexts[device] = Context(device)
    return _contexts[device]


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(t):
    import torch
    if t.dtype == torch.complex64:
        return FS_C64
    if t.dtype == torch.complex128:
        return FS_C128
    raise TypeError("state must be complex64 or complex128, got %s" % t.dtype)


def _check_state(vec, norb, nelec):
    from math import comb
    if not vec.is_cuda:
        raise ValueError("state must be a CUDA tensor (there is no CPU path)")
    shape = (comb(norb, nelec[0]), comb(norb, nelec[1]))
    if tuple(vec.shape) != shape:
        raise ValueError("state shape %s, expected %s" % (tuple(vec.shape), shape))
    if not vec.is_contiguous():
        raise ValueError("state must be contiguous")


def _f64(a, shape=None, complex_=False):
    a = np.ascontiguousarray(a, dtype=np.complex128 if complex_ else np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _ptr(a):
    return a.ctypes.data_as(_P) if a is not None else None


# ----------------------------------------------------------------- tables
def string_table(norb, nocc, ctx=None):
    from math import comb
    ctx = ctx or context()
    out = np.zeros(comb(norb, nocc), np.uint32)
    _check("fs_string_table", load_library().fs_string_table(ctx.handle, norb, nocc,
                                                             _ptr(out), out.size))
    return out


def excitation_table(norb, nocc, ctx=None):
    from math import comb
    ctx = ctx or context()
    d = comb(norb, nocc)
    out = np.zeros(d * norb * norb, np.uint32)
    _check("fs_excitation_table", load_library().fs_excitation_table(
        ctx.handle, norb, nocc, _ptr(out), out.size))
    return out.reshape(d, norb, norb)


# ------------------------------------------------------------------ gates
def apply_orbital_rotation_(vec, U, norb, nelec, U_b=None, ctx=None):
    _check_state(vec, norb, nelec)
    ctx = ctx or context(vec.device.index)
    Ua = _f64(U, (norb, norb), True)
    Ub = None if U_b is None else _f64(U_b, (norb, norb), True)
    _check("fs_apply_orbital_rotation", load_library().fs_apply_orbital_rotation(
        ctx.handle, _P(vec.data_ptr()), _dtype_code(vec), _ptr(Ua), _ptr(Ub), norb,
        nelec[0], nelec[1], _stream_ptr()))
    return vec


def apply_orbital_rotation(vec, U, norb, nelec, U_b=None, ctx=None):
    return apply_orbital_rotation_(vec.clone(), U, norb, nelec, U_b, ctx)


def apply_num_op_sum_evolution_(vec, lam, t, norb, nelec, lam_b=None, ctx=None):
    _check_state(vec, norb, nelec)
    ctx = ctx or context(vec.device.index)
    la = _f64(lam, (norb,))
    lb = None if lam_b is None else _f64(lam_b, (norb,))
    _check("fs_apply_num_op_sum_evolution", load_library().fs_apply_num_op_sum_evolution(
        ctx.handle, _P(vec.data_ptr()), _dtype_code(vec), _ptr(la), _ptr(lb), float(t),
        norb, nelec[0], nelec[1], _stream_ptr()))
    return vec


def apply_num_op_sum_evolution(vec, lam, t, norb, nelec, lam_b=None, ctx=None):
    return apply_num_op_sum_evolution_(vec.clone(), lam, t, norb, nelec, lam_b, ctx)


def apply_diag_coulomb_evolution_(vec, J_aa, J_ab, t, norb, nelec, J_bb=None, ctx=None):
    _check_state(vec, norb, nelec)
    ctx = ctx or context(vec.device.index)
    a = _f64(J_aa, (norb, norb))
    b = _f64(J_ab, (norb, norb))
    c = None if J_bb is None else _f64(J_bb, (norb, norb))
    _check("fs_apply_diag_coulomb_evolution", load_library().fs_apply_diag_coulomb_evolution(
        ctx.handle, _P(vec.data_ptr()), _dtype_code(vec), _ptr(a), _ptr(b), _ptr(c), float(t),
        norb, nelec[0], nelec[1], _stream_ptr()))
    return vec


def apply_diag_coulomb_evolution(vec, J_aa, J_ab, t, norb, nelec, J_bb=None, ctx=None):
    return apply_diag_coulomb_evolution_(vec.clone(), J_aa, J_ab, t, norb, nelec, J_bb, ctx)


def apply_diag_coulomb_evolution_noalloc_(vec, J_aa, J_ab, t, norb, nelec, J_bb=None):
    """In-place diagonal-Coulomb evolution that allocates no device memory
    (for callers that must not allocate; at most 16384 strings per spin).
    Runs on the state's own device and that device's current stream; needs
    no context."""
    _check_state(vec, norb, nelec)
    a = _f64(J_aa, (norb, norb))
    b = _f64(J_ab, (norb, norb))
    c = None if J_bb is None else _f64(J_bb, (norb, norb))
    import torch
    with torch.cuda.device(vec.device):
        stream = torch.cuda.current_stream(vec.device).cuda_stream
        _check("fs_apply_diag_coulomb_evolution_noalloc",
               load_library().fs_apply_diag_coulomb_evolution_noalloc(
                   _P(vec.data_ptr()), _dtype_code(vec), _ptr(a), _ptr(b), _ptr(c),
                   float(t), norb, nelec[0], nelec[1], _P(stream)))
    return vec


# ------------------------------------------------------------------- LUCJ
def _lucj_struct(K, J_aa, J_ab, norb, nelec, from_hf):
    K = _f64(K, None, True)
    J_aa = _f64(J_aa)
    J_ab = _f64(J_ab)
    n_reps = K.shape[0]
    if K.shape != (n_reps, norb, norb) or J_aa.shape != K.shape or J_ab.shape != K.shape:
        raise ValueError("K, J_aa, J_ab must have shape (n_reps, norb, norb)")
    op = LUCJ(norb, nelec[0], nelec[1], n_reps, K.ctypes.data, J_aa.ctypes.data,
              J_ab.ctypes.data, int(bool(from_hf)))
    return op, (K, J_aa, J_ab)


def lucj_forward_(vec, K, J_aa, J_ab, norb, nelec, from_hf=False, ctx=None):
    _check_state(vec, norb, nelec)
    ctx = ctx or context(vec.device.index)
    op, keep = _lucj_struct(K, J_aa, J_ab, norb, nelec, from_hf)
    _check("fs_lucj_forward", load_library().fs_lucj_forward(
        ctx.handle, ctypes.byref(op), _P(vec.data_ptr()), _dtype_code(vec), _stream_ptr()))
    return vec


def lucj_vjp_(vec, cot, K, J_aa, J_ab, norb, nelec, from_hf=False, ctx=None):
    """In place: vec (forward output) -> recomputed input, cot -> dL/dpsi_in.
    Returns (dK, dJ_aa, dJ_ab) as NumPy arrays."""
    _check_state(vec, norb, nelec)
    _check_state(cot, norb, nelec)
    if cot.dtype != vec.dtype:
        raise TypeError("state and cotangent must have the same dtype")
    ctx = ctx or context(vec.device.index)
    op, keep = _lucj_struct(K, J_aa, J_ab, norb, nelec, from_hf)
    n_reps = op.n_reps
    dK = np.zeros((n_reps, norb, norb), np.complex128)
    dJa = np.zeros((n_reps, norb, norb))
    dJb = np.zeros((n_reps, norb, norb))
    _check("fs_lucj_vjp", load_library().fs_lucj_vjp(
        ctx.handle, ctypes.byref(op), _P(vec.data_ptr()), _P(cot.data_ptr()),
        _dtype_code(vec), _ptr(dK), _ptr(dJa), _ptr(dJb), _stream_ptr()))
    return dK, dJa, dJb


def lucj_batch_(vecs, cots, circuits, do_vjp=True, ctx=None):
    """Forward pass (and, with do_vjp, the VJP) of many independent LUCJ
    circuits in one CUDA graph.  circuits[c] = dict(K, J_aa, J_ab, norb,
    nelec, from_hf); vecs[c] / cots[c] are that circuit's state and
    cotangent tensors (one dtype for all), updated in place exactly as by
    lucj_forward_ followed by lucj_vjp_.  All circuits share n_reps.
    Returns [(dK, dJ_aa, dJ_ab)] (None without do_vjp)."""
    n = len(circuits)
    if len(vecs) != n or (do_vjp and len(cots) != n):
        raise ValueError("one state (and cotangent) per circuit")
    dt = _dtype_code(vecs[0])
    ctx = ctx or context(vecs[0].device.index)
    ops = (LUCJ * n)()
    keep, grads = [], []
    pK, pA, pB = (_P * n)(), (_P * n)(), (_P * n)()
    for c, cir in enumerate(circuits):
        norb, nelec = cir["norb"], tuple(cir["nelec"])
        _check_state(vecs[c], norb, nelec)
        if _dtype_code(vecs[c]) != dt:
            raise TypeError("all states of a batch need one dtype")
        if do_vjp:
            _check_state(cots[c], norb, nelec)
        op, k = _lucj_struct(cir["K"], cir["J_aa"], cir["J_ab"], norb, nelec,
                             cir.get("from_hf", False))
        ops[c] = op
        keep.append(k)
        r = op.n_reps
        g = (np.zeros((r, norb, norb), np.complex128), np.zeros((r, norb, norb)),
             np.zeros((r, norb, norb)))
        grads.append(g)
        pK[c], pA[c], pB[c] = g[0].ctypes.data, g[1].ctypes.data, g[2].ctypes.data
    pv = (_P * n)(*[v.data_ptr() for v in vecs])
    pc = (_P * n)(*[x.data_ptr() for x in cots]) if do_vjp else (_P * n)()
    _check("fs_lucj_batch", load_library().fs_lucj_batch(
        ctx.handle, n, ops, pv, pc, dt, int(bool(do_vjp)), pK, pA, pB, _stream_ptr()))
    return grads if do_vjp else [None] * n


# ------------------------------------------------- remaining Table 1 gates
_SPINS = {"alpha": 1, "beta": 2, "both": 3, 1: 1, 2: 2, 3: 3}


def _spins(spin):
    if spin not in _SPINS:
        raise ValueError("spin must be 'alpha', 'beta' or 'both'")
    return _SPINS[spin]


def _spin_index(s):
    return {"alpha": 0, "beta": 1, 0: 0, 1: 1}[s]


def _state_call(name, vec, norb, nelec, ctx, *args):
    _check_state(vec, norb, nelec)
    ctx = ctx or context(vec.device.index)
    _check(name, getattr(load_library(), name)(
        ctx.handle, _P(vec.data_ptr()), _dtype_code(vec), *args, norb, nelec[0], nelec[1],
        _stream_ptr()))
    return vec


def apply_num_interaction_(vec, theta, p, norb, nelec, spin="both", ctx=None):
    """exp(i theta n_{p sigma}) in place (Table 1)."""
    return _state_call("fs_apply_num_interaction", vec, norb, nelec, ctx, float(theta), int(p),
                       _spins(spin))


def apply_num_num_interaction_(vec, theta, p, q, norb, nelec, spins=("alpha", "alpha"),
                               ctx=None):
    """exp(i theta n_{p sigma} n_{q tau}) in place (Table 1); spins = (sigma, tau)."""
    return _state_call("fs_apply_num_num_interaction", vec, norb, nelec, ctx, float(theta),
                       int(p), _spin_index(spins[0]), int(q), _spin_index(spins[1]))


def apply_givens_rotation_(vec, theta, p, q, norb, nelec, spin="both", ctx=None):
    """exp(theta (a^dag_p a_q - a^dag_q a_p)) in place (Table 1)."""
    return _state_call("fs_apply_givens_rotation", vec, norb, nelec, ctx, float(theta), int(p),
                       int(q), _spins(spin))


def apply_tunneling_interaction_(vec, theta, p, q, norb, nelec, spin="both", ctx=None):
    """exp(i theta (a^dag_p a_q + a^dag_q a_p)) in place (Table 1)."""
    return _state_call("fs_apply_tunneling_interaction", vec, norb, nelec, ctx, float(theta),
                       int(p), int(q), _spins(spin))


def apply_quad_ham_evolution_(vec, M, t, norb, nelec, M_b=None, ctx=None):
    """exp(-i t sum M_pq a^dag_p a_q) in place, per spin (Table 1)."""
    Ma = _f64(M, (norb, norb), True)
    Mb = None if M_b is None else _f64(M_b, (norb, norb), True)
    return _state_call("fs_apply_quad_ham_evolution", vec, norb, nelec, ctx, _ptr(Ma), _ptr(Mb),
                       float(t))


# ------------------------------------------------------------ Trotter
def simulate_trotter_double_factorized_(vec, one_body, diag_coulomb_mats, orbital_rotations,
                                        time, norb, nelec, n_steps=1, order=0, ctx=None):
    """Trotter-Suzuki evolution by a double-factorized Hamiltonian, in place."""
    h = _f64(one_body, (norb, norb), True)
    J = _f64(diag_coulomb_mats)
    U = _f64(orbital_rotations, None, True)
    n_terms = J.shape[0] if J.ndim == 3 else 0
    if n_terms and (J.shape != (n_terms, norb, norb) or U.shape != (n_terms, norb, norb)):
        raise ValueError("diag_coulomb_mats and orbital_rotations must be (n_terms, norb, norb)")
    return _state_call("fs_simulate_trotter_double_factorized", vec, norb, nelec, ctx, _ptr(h),
                       n_terms, _ptr(J) if n_terms else None, _ptr(U) if n_terms else None,
                       float(time), int(n_steps), int(order))


def simulate_trotter_diag_coulomb_(vec, one_body, J_aa, J_ab, time, norb, nelec, n_steps=1,
                                   order=0, J_bb=None, ctx=None):
    """Trotter-Suzuki evolution by a diagonal-Coulomb Hamiltonian, in place."""
    h = _f64(one_body, (norb, norb), True)
    Ja, Jb = _f64(J_aa, (norb, norb)), _f64(J_ab, (norb, norb))
    Jbb = None if J_bb is None else _f64(J_bb, (norb, norb))
    return _state_call("fs_simulate_trotter_diag_coulomb", vec, norb, nelec, ctx, _ptr(h),
                       _ptr(Ja), _ptr(Jb), _ptr(Jbb), float(time), int(n_steps), int(order))


# ------------------------------------------------------ operator action
def apply_molecular_hamiltonian(vec, one_body, two_body, norb, nelec, constant=0.0, out=None,
                                workspace_bytes=0, ctx=None):
    """H vec for the molecular Hamiltonian with real tensors h_pq, h_pqrs;
    returns a new tensor (or fills `out`)."""
    import torch
    _check_state(vec, norb, nelec)
    h1 = _f64(one_body, (norb, norb))
    h2 = _f64(two_body, (norb, norb, norb, norb))
    if out is None:
        out = torch.empty_like(vec)
    _check_state(out, norb, nelec)
    if out.dtype != vec.dtype or out.data_ptr() == vec.data_ptr():
        raise ValueError("out must be a distinct tensor of the same dtype")
    ctx = ctx or context(vec.device.index)
    _check("fs_apply_molecular_hamiltonian", load_library().fs_apply_molecular_hamiltonian(
        ctx.handle, _P(vec.data_ptr()), _P(out.data_ptr()), _dtype_code(vec), _ptr(h1), _ptr(h2),
        float(constant), int(workspace_bytes), norb, nelec[0], nelec[1], _stream_ptr()))
    return out


# ------------------------------------------------------------- sampling
def _uniforms(uniforms, count, seed, device):
    """FP64 uniforms on the device: the given ones, or `count` drawn from a
    torch generator seeded with `seed`."""
    import torch
    if uniforms is not None:
        if isinstance(uniforms, torch.Tensor):
            u = uniforms.to(device=device, dtype=torch.float64)
        else:
            u = torch.from_numpy(np.ascontiguousarray(uniforms, dtype=np.float64)).to(device)
        return u.contiguous()
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.rand(count, dtype=torch.float64, device=device, generator=g)


def sample_state(vec, norb, nelec, shots=None, uniforms=None, seed=0, ctx=None):
    """Addresses a = i * dim_b + j (int64 CUDA tensor) of configurations drawn
    from |vec|^2 by inverse CDF in address order, one per uniform (FP64 in
    [0, 1), given or drawn from a seeded generator)."""
    import torch
    _check_state(vec, norb, nelec)
    if uniforms is None and shots is None:
        raise ValueError("give shots or uniforms")
    u = _uniforms(uniforms, shots, seed, vec.device).reshape(-1)
    out = torch.empty(u.numel(), dtype=torch.int64, device=vec.device)
    ctx = ctx or context(vec.device.index)
    _check("fs_sample_state", load_library().fs_sample_state(
        ctx.handle, _P(vec.data_ptr()), _dtype_code(vec), norb, nelec[0], nelec[1],
        _P(u.data_ptr()), u.numel(), _P(out.data_ptr()), _stream_ptr()))
    return out


def addresses_to_strings(addr, norb, nelec, ctx=None):
    """(alpha masks, beta masks) of sampled addresses, from the library's
    string tables."""
    ma, mb = string_table(norb, nelec[0], ctx), string_table(norb, nelec[1], ctx)
    a = addr.cpu().numpy() if hasattr(addr, "cpu") else np.asarray(addr)
    return ma[a // len(mb)], mb[a % len(mb)]


def _slater_spin(U, occ, norb, shots, uniforms, seed, device, ctx):
    import torch
    occ = np.ascontiguousarray(occ, dtype=np.int32).reshape(-1)
    Um = _f64(U, (norb, norb), True)
    n = occ.size
    if uniforms is None and shots is None:
        raise ValueError("give shots or uniforms")
    u = _uniforms(uniforms, (shots or 0) * n, seed, device).reshape(-1)
    if n and u.numel() % n:
        raise ValueError("uniforms must have shape (shots, len(occ))")
    shots = u.numel() // n if n else int(shots)
    words = (norb + 63) // 64
    out = torch.empty(max(shots * words, 1), dtype=torch.int64, device=device)
    _check("fs_sample_slater", load_library().fs_sample_slater(
        ctx.handle, _ptr(Um), norb, _ptr(occ) if n else None, n,
        _P(u.data_ptr()) if u.numel() else None, shots, _P(out.data_ptr()), _stream_ptr()))
    m = out[:shots * words].cpu().numpy().view(np.uint64).reshape(shots, words)
    return m[:, 0] if words == 1 else m


def sample_slater(norb, occ, U, shots=None, uniforms=None, seed=0, device=None, ctx=None):
    """Occupation masks (uint64 per shot; rows of ceil(norb/64) words when
    norb > 64) sampled from the Slater determinant U(U)|occ>.  Spinless:
    occ is a list of orbitals.  Spinful: occ = (occ_a, occ_b), U one matrix
    or a pair (U_a, U_b), uniforms None or a pair; returns (masks_a,
    masks_b), the spins drawn independently."""
    import torch
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    device = torch.device(device)
    ctx = ctx or context(device.index or 0)
    spinful = len(occ) == 2 and not np.isscalar(occ[0])
    if not spinful:
        return _slater_spin(U, occ, norb, shots, uniforms, seed, device, ctx)
    Us = U if (isinstance(U, (tuple, list)) and len(U) == 2) else (U, U)
    us = uniforms if uniforms is not None else (None, None)
    return tuple(_slater_spin(Us[s], occ[s], norb, shots, us[s], seed + s, device, ctx)
                 for s in range(2))


# ------------------------------------------------------------ measurement
def measure_fp32_fma(device=None):
    """FP32 FMA throughput of the current (or given) device in TFLOP/s, and
    the time of one probe launch in ms (library kernel, CUDA events)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    with torch.cuda.device(dev):
        tf, ms = _D(0), _D(0)
        _check("fs_measure_fp32_fma", load_library().fs_measure_fp32_fma(
            _P(torch.cuda.current_stream(dev).cuda_stream), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value
