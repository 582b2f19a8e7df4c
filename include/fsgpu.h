/*
 * fsgpu: fixed-sector fermionic state vectors on one GB300 GPU (sm_103a).
 *
 * C ABI of libfsgpu.so.  No C++ or PyTorch types cross this boundary:
 * pointers are plain device or host addresses, sizes are plain integers and
 * a stream is passed as `void *` holding a cudaStream_t (NULL = the legacy
 * default stream).
 *
 * State layout (the paper's state-vector representation, §3.1): a state in
 * the sector (norb, n_alpha, n_beta) is a row-major dim_a x dim_b complex
 * matrix, dim_s = C(norb, n_s).  Element (i, j) is the coefficient of the
 * configuration |I_a, I_b> = cre_b(I_b) cre_a(I_a)|vac> (§2.2, §2.5) whose
 * alpha string has address i and beta string address j.  The address of a
 * string (occupied-orbital bitmask, bit p = orbital p) is its position among
 * all strings with the same electron count listed in ascending integer
 * order; equivalently sum_k C(o_k, k+1) over the occupied orbitals
 * o_0 < o_1 < ... (combinatorial number system).  The Hartree-Fock string
 * {0, ..., n-1} has address 0.  Complex numbers are interleaved (re, im):
 * FS_C64 = two floats, FS_C128 = two doubles.  A state pointer must be
 * 16-byte aligned.
 *
 * Ownership: every state/cotangent pointer belongs to the caller, who
 * allocates and frees it; the library updates it in place and never keeps
 * it after the call returns.  The library owns its context, its cached
 * string tables and its scratch buffers (allocated on first use for a
 * sector, freed by fs_destroy).
 *
 * Host matrices are row-major `const double *`; an N x N complex matrix is
 * 2*N*N doubles (interleaved re, im); a real N x N matrix is N*N doubles.
 *
 * Asynchrony: calls enqueue work on `stream` and return; host inputs are
 * copied before the call returns, so they may be reused at once.  Calls on
 * one context share its scratch buffers (host calls on a context are
 * serialised by a lock, GPU work is not): issue them on one stream, or
 * order their streams, since calls of one context that overlap on the GPU
 * race on that scratch.  Separate contexts have separate scratch.  Calls
 * that return host outputs (fs_lucj_vjp gradients, fs_string_table,
 * fs_excitation_table) synchronize the stream before returning.
 *
 * Errors: every call returns an fs_status.  Argument errors are detected on
 * the host before any work is enqueued and leave the state untouched.
 * fs_last_error() returns a per-thread message for the last failure.
 * Kernels that can fail on the device (bounded waits, index checks) record
 * a code in the context's device status word; fs_sync_status() reads and
 * clears it.
 */
#ifndef FSGPU_H
#define FSGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FS_OK = 0,
  FS_ERR_ARG = -1,         /* invalid argument (sizes, pointers, alignment) */
  FS_ERR_NOT_UNITARY = -2, /* a matrix that must be unitary is not (1e-10) */
  FS_ERR_NOMEM = -3,       /* device or host allocation failed */
  FS_ERR_CUDA = -4,        /* a CUDA runtime call failed */
  FS_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
  FS_ERR_BOUNDS = -6,      /* a device-side index check failed */
  FS_ERR_UNSUPPORTED = -7  /* valid request outside what the library supports */
} fs_status;

typedef enum { FS_C64 = 0, FS_C128 = 1 } fs_dtype;

/* Orbital-rotation method: Givens sweeps (§3.2.3), dense minor-matrix
 * products (§2.3), or the faster of the two as measured by the library's
 * autotuner for the sector and dtype. */
typedef enum { FS_ROT_AUTO = 0, FS_ROT_GIVENS = 1, FS_ROT_MINORS = 2 } fs_rot_path;

typedef struct fs_ctx fs_ctx;

/* Create a context bound to CUDA device `device`.  The device must be an
 * sm_103 GPU.  Returns FS_ERR_ARG for a bad device index. */
int fs_create(fs_ctx **ctx, int device);
/* Free the context, its tables and scratch.  Synchronizes the device. */
int fs_destroy(fs_ctx *ctx);
/* Message of the last failing call on this host thread ("" if none). */
const char *fs_last_error(void);
/* Wait for `stream`, then read and clear the device status word.  Returns
 * FS_OK, FS_ERR_TIMEOUT or FS_ERR_BOUNDS, or FS_ERR_CUDA if the stream
 * itself failed. */
int fs_sync_status(fs_ctx *ctx, void *stream);

/* Kernel tracing.  fs_profile_start clears the record and brackets every
 * following kernel launch of this context with CUDA events on its launch
 * stream.  fs_profile_stop synchronizes those events, stops recording and
 * writes a JSON object {"<step>": [records, total_ms, kernel_launches], ...}
 * (NUL terminated) into out[0..cap); a record brackets one launch helper,
 * which may launch several kernels.  FS_ERR_ARG if it does not fit. */
int fs_profile_start(fs_ctx *ctx);
int fs_profile_stop(fs_ctx *ctx, char *out, int64_t cap);

/* Force or release the orbital-rotation method (default FS_ROT_AUTO).
 * Under FS_ROT_AUTO the first fs_apply_orbital_rotation call for a sector
 * and dtype whose string dimensions allow the minor-matrix method (both at
 * most 4096) times both methods on a scratch copy of the state, which
 * synchronizes the stream once, and the faster method is used from then on
 * for that sector and dtype.  FS_ROT_MINORS on a larger sector returns
 * FS_ERR_UNSUPPORTED. */
int fs_set_rotation_path(fs_ctx *ctx, int path);

/* Arithmetic engine of the complex64 Givens sweeps (§3.2.3).
 *   FS_SWEEP_AUTO:      the CUDA cores (measured faster on GB300 at the
 *                       benchmarked sectors, see FS_SWEEP_TENSOR);
 *   FS_SWEEP_CUDA_CORE: every Givens rotation as FP32 FMAs on CUDA cores;
 *   FS_SWEEP_TENSOR:    each window step of 6 adjacent orbitals as one
 *                       dense product with the compound matrices of the
 *                       step (det V[S', S], §2.3) on the tcgen05 tensor
 *                       cores, both operands split exactly into three
 *                       BF16 pieces and six products kept (FP32
 *                       accuracy); falls back to the CUDA cores where the
 *                       tensor path does not apply (complex128, fewer than
 *                       6 orbitals, vectors spanning more than 2 CTAs).
 * Results agree to FP32 rounding.  FS_ERR_ARG for another value. */
enum { FS_SWEEP_AUTO = 0, FS_SWEEP_CUDA_CORE = 1, FS_SWEEP_TENSOR = 2 };
int fs_set_sweep_engine(fs_ctx *ctx, int engine);

/* Autotuner of the batched LUCJ sweeps (fs_lucj_batch): on the first call
 * that meets a sector (norb, electrons of both spins), precision and sweep
 * kind, every slab width (vectors per CTA, 1 .. 64 within the stage's
 * shared-memory budget; at least 2 for complex64 forward sweeps, which run
 * on packed vector pairs) is timed as a one-circuit launch of the batched
 * kernel on scratch states, before the batch is captured, and the fastest
 * is kept for the context.  on = 0 switches it off (and forgets the choices;
 * untuned batches use about eight slabs per circuit); on = 1 (the default)
 * switches it on.  Not part of the paper's method: a scheduling aid. */
int fs_set_batch_tuning(fs_ctx *ctx, int on);
/* The autotuner's choices as JSON, NUL terminated, into out[0..cap):
 * [{"norb", "n_this", "n_other", "dtype", "states", "reverse", "cross",
 *   "budget_kb", "vectors_per_cta", "widths": [the timed slab widths],
 *   "ms": [the time of each]}].
 * FS_ERR_ARG if it does not fit. */
int fs_tuning_report(fs_ctx *ctx, char *out, int64_t cap);

/* Measures the device's FP32 fused multiply-add throughput (the denominator
 * of the arithmetic roofline of the Givens sweeps): 8 blocks of 256 threads
 * per SM, each thread running 8 independent FMA chains, timed with CUDA
 * events on `stream` after two warm-up launches.  Writes TFLOP/s (2 flops
 * per FMA) to *tflops and, if ms is not NULL, the time of one launch.
 * Synchronizes `stream`; allocates a small result buffer with
 * cudaMallocAsync.  Not part of the paper's method: a measurement aid. */
int fs_measure_fp32_fma(void *stream, double *tflops, double *ms);

/* Sector string tables, built on the device with the combinatorial number
 * system (§3.1 addressing).  Copies dim = C(norb, nocc) masks to
 * `masks_host` (caller-owned, dim entries) in address order.
 * Synchronous.  norb <= 32, dim < 2^31. */
int fs_string_table(fs_ctx *ctx, int norb, int nocc, uint32_t *masks_host,
                    int64_t dim);

/* Single-excitation table for E_pq = a^dag_p a_q on strings of one spin
 * (§2.2 sign convention).  For string address i and the pair (p, q):
 * out[(i * norb + p) * norb + q] = (sign << 31) | target, where target is
 * the address of I^{q->p} and sign = 1 when a^dag_p a_q |I> = -|I'>, or
 * 0xFFFFFFFF when a^dag_p a_q |I> = 0.  For p == q the target is i and the
 * sign is 0 when q is occupied.  `out_host` holds dim*norb*norb entries.
 * Synchronous. */
int fs_excitation_table(fs_ctx *ctx, int norb, int nocc, uint32_t *out_host,
                        int64_t n_entries);

/* Orbital rotation exp(sum_{pq sigma} log(U_sigma)_pq a^dag_{p sigma} a_{q sigma})
 * (§2.3, §3.2.3, Table 1).  U_a and U_b are N x N unitary (host,
 * complex); U_b == NULL means U_b = U_a.  `vec` is updated in place.
 * Errors: FS_ERR_NOT_UNITARY when ||U^dag U - I||_max > 1e-10;
 * FS_ERR_UNSUPPORTED when a string dimension exceeds 65535. */
int fs_apply_orbital_rotation(fs_ctx *ctx, void *vec, int dtype,
                              const double *U_a, const double *U_b, int norb,
                              int n_alpha, int n_beta, void *stream);

/* Number-operator-sum evolution exp(-i t sum_{p sigma} lambda^sigma_p n_{p sigma})
 * (§3.2.1, Table 1).  lam_a, lam_b: N reals (host); lam_b == NULL means
 * lam_b = lam_a. */
int fs_apply_num_op_sum_evolution(fs_ctx *ctx, void *vec, int dtype,
                                  const double *lam_a, const double *lam_b,
                                  double t, int norb, int n_alpha, int n_beta,
                                  void *stream);

/* Diagonal-Coulomb evolution
 *   exp(-1/2 i t sum_{pq sigma tau} J^{sigma tau}_pq n_{p sigma} n_{q tau})
 * (§3.2.2, Table 1), J^{beta alpha} = (J^{alpha beta})^T.  J_aa, J_ab,
 * J_bb: N x N reals (host); J_bb == NULL means J_bb = J_aa. */
int fs_apply_diag_coulomb_evolution(fs_ctx *ctx, void *vec, int dtype,
                                    const double *J_aa, const double *J_ab,
                                    const double *J_bb, double t, int norb,
                                    int n_alpha, int n_beta, void *stream);

/* The same diagonal-Coulomb evolution for callers that must not allocate
 * device memory: callers whose device memory belongs to a pool or arena the
 * library may not bypass, and callers that cannot afford the device-wide
 * synchronization a cudaMalloc or cudaFree can cause.  The paper has no
 * counterpart; this is a deployment variant of the call above.
 *
 * Needs no context and allocates nothing (no cudaMalloc, no cudaFree, no
 * allocating library routine): its scratch (string masks and per-string
 * phase factors, 640 KiB) is one static device array that every GPU which
 * loads the library holds until the process exits.  The caller still owns
 * `vec`, which must be device memory of the current device (else
 * FS_ERR_ARG).  Arguments and results are those of
 * fs_apply_diag_coulomb_evolution; each spin may have at most 16384 strings
 * (C(norb, n) <= 16384), larger sectors return FS_ERR_UNSUPPORTED before any
 * work is enqueued.
 *
 * The first call on a device looks up the array's device address with that
 * device current and loads every kernel the call launches, in both
 * precisions; make that first call before any stream capture.  All calls share the one array and
 * overwrite all of it that they read, so nothing carries over between calls;
 * calls that overlap on the GPU (on different streams, or from different
 * host threads without ordering) race on it. */
int fs_apply_diag_coulomb_evolution_noalloc(void *vec, int dtype,
                                            const double *J_aa,
                                            const double *J_ab,
                                            const double *J_bb, double t,
                                            int norb, int n_alpha, int n_beta,
                                            void *stream);

/* LUCJ ansatz (§4.3, §4.5.1): n_reps repetitions U_k D_k U_k^dag, k = 0 ..
 * n_reps-1 applied in order, with U_k = U(expm(K_k)) (K_k anti-Hermitian,
 * N x N complex) and D_k the spin-balanced diagonal-Coulomb evolution with
 * J_bb = J_aa = J_aa[k], J_ab = J_ab[k] at t = 1.  No final rotation.
 * K: n_reps*2*N*N doubles; J_aa, J_ab: n_reps*N*N doubles (host). */
typedef struct {
  int norb, n_alpha, n_beta, n_reps;
  const double *K;
  const double *J_aa;
  const double *J_ab;
  int from_hf; /* 1: start from the Hartree-Fock state, ignoring vec's input */
} fs_lucj;

/* vec: in = initial state (ignored when from_hf), out = final state. */
int fs_lucj_forward(fs_ctx *ctx, const fs_lucj *op, void *vec, int dtype,
                    void *stream);

/* Vector-Jacobian product of the forward pass for L = Re <cot, psi_out>,
 * by reverse sweeps that uncompute the state (no stored intermediates).
 *   vec: in = psi_out (the forward result), out = the recomputed input state;
 *   cot: in = dL/dpsi_out, out = dL/dpsi_in (conjugate-Wirtinger convention,
 *        i.e. C^dag cot for the circuit C);
 *   dK:   n_reps*2*N*N doubles, dL/dRe K + i dL/dIm K for every entry;
 *   dJ_aa, dJ_ab: n_reps*N*N doubles, dL/dJ_pq with entries independent.
 * Host outputs; synchronizes the stream.  Any of dK, dJ_aa, dJ_ab may be
 * NULL to skip it.  The device-side sums behind the gradients reach the host
 * through a small mapped pinned buffer of the context (at least 128 KB,
 * written by a kernel rather than copied by a copy engine, so that the
 * call does not wait behind the caller's own large host copies); the first
 * call on a context allocates it (an allocation of pinned memory, which
 * synchronizes the device), and fs_destroy frees it. */
int fs_lucj_vjp(fs_ctx *ctx, const fs_lucj *op, void *vec, void *cot,
                int dtype, double *dK, double *dJ_aa, double *dJ_ab,
                void *stream);

/* ---- Remaining gates of Table 1 (each a special case of the gates above,
 * as listed after Table 1).  `spins` is a mask: 1 = alpha, 2 = beta,
 * 3 = both (the two spin parts commute).  All act in place on `vec` on the
 * stream, like fs_apply_orbital_rotation; orbital indices are 0-based.
 *
 * Number interaction exp(i theta n_{p sigma}). */
int fs_apply_num_interaction(fs_ctx *ctx, void *vec, int dtype, double theta, int p, int spins,
                             int norb, int n_alpha, int n_beta, void *stream);
/* Number-number interaction exp(i theta n_{p sigma} n_{q tau}); sigma, tau
 * are 0 (alpha) or 1 (beta); p == q with sigma == tau is n_p. */
int fs_apply_num_num_interaction(fs_ctx *ctx, void *vec, int dtype, double theta, int p,
                                 int sigma, int q, int tau, int norb, int n_alpha, int n_beta,
                                 void *stream);
/* Givens rotation exp(theta (a^dag_p a_q - a^dag_q a_p)) on the spins of
 * the mask (p != q): the orbital rotation by expm(theta (E_pq - E_qp)). */
int fs_apply_givens_rotation(fs_ctx *ctx, void *vec, int dtype, double theta, int p, int q,
                             int spins, int norb, int n_alpha, int n_beta, void *stream);
/* Tunneling interaction exp(i theta (a^dag_p a_q + a^dag_q a_p)) on the
 * spins of the mask (p != q): the orbital rotation by
 * expm(i theta (E_pq + E_qp)). */
int fs_apply_tunneling_interaction(fs_ctx *ctx, void *vec, int dtype, double theta, int p,
                                   int q, int spins, int norb, int n_alpha, int n_beta,
                                   void *stream);
/* Quadratic Hamiltonian evolution exp(-i t sum_{pq sigma} M^sigma_pq
 * a^dag_{p sigma} a_{q sigma}): the orbital rotation by expm(-i M t) per
 * spin.  M_a, M_b: host N x N complex Hermitian (interleaved), M_b NULL
 * means M_a; FS_ERR_ARG if not Hermitian to 1e-10. */
int fs_apply_quad_ham_evolution(fs_ctx *ctx, void *vec, int dtype, const double *M_a,
                                const double *M_b, double t, int norb, int n_alpha, int n_beta,
                                void *stream);

/* ---- Operator action (operator-action section): out = H vec for the
 * molecular Hamiltonian (the molecular Hamiltonian equation)
 *   H = constant + sum_{pq sigma} h_pq a^dag_{p sigma} a_{q sigma}
 *       + 1/2 sum_{pqrs sigma tau} h_pqrs a^dag_{p sigma} a^dag_{r tau} a_{s tau} a_{q sigma}
 * with REAL tensors: one_body = h (N x N doubles), two_body = h_pqrs (N^4
 * doubles, index ((p*N + q)*N + r)*N + s).  `vec` and `out` are distinct
 * device states of the same sector and dtype; `vec` is read only, `out` is
 * overwritten.  The work runs in blocks whose N^2-fold intermediates use at
 * most `workspace_bytes` of scratch (0: min(8 GiB, a quarter of free
 * memory)).  The contractions over the two-body tensor are cuBLAS GEMMs in
 * the state's precision; everything else runs in the library's kernels.
 * N <= 32.  Asynchronous on `stream`. */
int fs_apply_molecular_hamiltonian(fs_ctx *ctx, const void *vec, void *out, int dtype,
                                   const double *one_body, const double *two_body,
                                   double constant, int64_t workspace_bytes, int norb,
                                   int n_alpha, int n_beta, void *stream);

/* ---- Trotter-Suzuki time evolution (Hamiltonian time evolution section).
 * exp(-i H time) vec ~ S_order(time / n_steps)^n_steps with
 *   S_0(t) = exp(-i H_L t) .. exp(-i H_1 t),
 *   S_1(t) = exp(-i H_1 t/2) .. exp(-i H_L t/2) exp(-i H_L t/2) .. exp(-i H_1 t/2),
 *   S_k(t) = S_{k-1}(u_k t)^2 S_{k-1}((1 - 4 u_k) t) S_{k-1}(u_k t)^2,
 *   u_k = 1 / (4 - 4^{1/(2k-1)}),  order in 0 .. 6, n_steps >= 1.
 * H_1 is the one-body term sum_{pq sigma} h_pq a^dag a (exponential: the
 * orbital rotation by expm(-i h t)); the two-body terms follow in order.
 * Neighbouring factors of the same term are joined, neighbouring rotations
 * multiplied on the host, and every diagonal-Coulomb evolution runs fused
 * into a rotation's beta sweep.  In place on `vec`, on the stream.
 *
 * Double-factorized Hamiltonian (eq. for the double factorized form):
 * H = sum h_pq a^dag a + 1/2 sum_t sum_{pq sigma tau} J^(t)_pq n^(t)_{p sigma}
 * n^(t)_{q tau}, n^(t)_p the number operator rotated by U^(t); term t's
 * exponential is U(U^(t)) DC(J^(t), t) U(U^(t))^dag.  one_body: N x N
 * complex Hermitian; diag_coulomb_mats: n_terms x N x N real symmetric;
 * orbital_rotations: n_terms x N x N complex unitary (interleaved). */
int fs_simulate_trotter_double_factorized(fs_ctx *ctx, void *vec, int dtype,
                                          const double *one_body, int n_terms,
                                          const double *diag_coulomb_mats,
                                          const double *orbital_rotations, double time,
                                          int n_steps, int order, int norb, int n_alpha,
                                          int n_beta, void *stream);
/* Diagonal-Coulomb Hamiltonian H = sum h_pq a^dag a + 1/2 sum_{pq sigma tau}
 * J^{sigma tau}_pq n_{p sigma} n_{q tau} (J^{beta alpha} = J_ab^T, J_bb NULL
 * means J_aa): H_1 the one-body term, H_2 the diagonal-Coulomb term. */
int fs_simulate_trotter_diag_coulomb(fs_ctx *ctx, void *vec, int dtype, const double *one_body,
                                     const double *J_aa, const double *J_ab,
                                     const double *J_bb, double time, int n_steps, int order,
                                     int norb, int n_alpha, int n_beta, void *stream);

/* ---- Sampling configurations.
 *
 * From a state (sample-based algorithms section: the probabilities are the
 * squared magnitudes of the entries).  For shot k, with the uniform
 * u_k = uniforms[k], out[k] is the first row-major address a = i * dim_b + j
 * whose inclusive prefix sum_{a' <= a} |vec[a']|^2 exceeds u_k * ||vec||^2:
 * the inverse of the cumulative distribution in address order, so each
 * configuration is drawn with probability |vec[a]|^2 / ||vec||^2.  A
 * configuration of zero amplitude is never returned.  uniforms: `shots`
 * doubles in [0, 1) (device); values below 0 (and NaN) act as 0, values
 * of 1 or more give the last configuration of nonzero amplitude.  out:
 * `shots` int64 (device); every entry is -1 when ||vec||^2 is zero or not
 * finite.  vec is read only.  Prefix sums run in FP64 for FS_C128 and in
 * double-float pairs (about 48 significant bits) for FS_C64, so a uniform
 * within about 1e-13 * ||vec||^2 of a boundary may land on either side of
 * it.  Asynchronous on `stream`; the context's scratch holds the prefix
 * tables (8 bytes per 256 amplitudes). */
int fs_sample_state(fs_ctx *ctx, const void *vec, int dtype, int norb, int n_alpha, int n_beta,
                    const double *uniforms, int64_t shots, int64_t *out, void *stream);

/* From a Slater determinant (Slater-sampling section), one spin: the state
 * U(U)|occ> has |amplitude|^2 = |det U[I, occ]|^2 (§2.4), a determinantal
 * point process with kernel U[:, occ] U[:, occ]^dag.  Each shot picks nocc
 * orbitals by the chain rule: at step i it takes orbital p with probability
 * w_p / sum_q w_q, w_q being the squared norm of row q of U[:, occ] after
 * projecting out the rows already picked, chosen by inverse CDF over the
 * orbitals in increasing order with the uniform uniforms[k * nocc + i].
 * U: host N x N complex (interleaved), of which only the columns listed in
 * occ (host, nocc distinct orbitals) are read; they must be orthonormal to
 * 1e-10 (FS_ERR_NOT_UNITARY otherwise).  uniforms: shots * nocc doubles in
 * [0, 1) (device).  out: shots * ceil(norb / 64) words (device); bit p of
 * word p / 64 of shot k is set when orbital p is occupied.  FP64
 * throughout.  1 <= norb <= 1024.  Asynchronous on `stream`.  For both spins
 * call once per spin with that spin's columns and uniforms: the spins are
 * independent. */
int fs_sample_slater(fs_ctx *ctx, const double *U, int norb, const int *occ, int nocc,
                     const double *uniforms, int64_t shots, uint64_t *out, void *stream);

/* Batched LUCJ (the ansatz of fs_lucj_forward, many independent circuits,
 * uneven sectors): ops[c], vecs[c], cots[c] describe circuit c exactly as
 * for fs_lucj_forward (and, when do_vjp, fs_lucj_vjp, which then follows
 * the forward pass: vec ends as the recomputed input, cot as dL/dpsi_in,
 * and dK[c], dJ_aa[c], dJ_ab[c] receive the gradients; any of these arrays
 * or entries may be NULL to skip).  Every stage of the circuits runs once
 * for all of them: each sweep is one persistent kernel launch over a work
 * queue of (circuit, slab) items, largest circuits first, and the whole
 * stage sequence is one captured CUDA graph.  Requirements: one dtype, the
 * same n_reps for all circuits, 6 <= norb <= 32, 2 <= C(norb, n_s) <= 65535.
 * Host outputs; synchronizes the stream when do_vjp.  The paper applies
 * its gates to one state at a time; batching is a deployment form of the
 * same operations. */
int fs_lucj_batch(fs_ctx *ctx, int n_circuits, const fs_lucj *ops,
                  void *const *vecs, void *const *cots, int dtype, int do_vjp,
                  double *const *dK, double *const *dJ_aa,
                  double *const *dJ_ab, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FSGPU_H */
