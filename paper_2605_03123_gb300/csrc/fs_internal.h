// Internal declarations shared by the fsgpu translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <complex>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "fsgpu.h"

namespace fs {

using zd = std::complex<double>;

// Largest orbital count handled by the string tables (masks are uint32).
constexpr int kMaxNorb = 32;
constexpr int kMaxOrb = kMaxNorb;
// Largest number of Givens rotations in one program: N(N-1)/2 for N = 32.
constexpr int kMaxGivens = kMaxNorb * (kMaxNorb - 1) / 2;
// Vector length limit of the sweep kernels (16-bit addresses in pair lists).
constexpr int64_t kMaxSweepDim = 65535;
// String-dimension limit of the dense minor-matrix rotation.
constexpr int64_t kMaxMinorDim = 4096;

// ------------------------------------------------------------- host math
// One adjacent-pair Givens rotation G = [[c, s], [-s*, c]] on orbitals
// (p, p+1).
struct Givens {
  int p;
  double c;
  zd s;
};
// U = D * G_M ... G_1 with D = diag(phase): G_1 acts first on the state.
struct RotProgram {
  std::vector<Givens> g;
  std::vector<zd> phase;
};

void mat_mul(int n, const zd* A, const zd* B, zd* C);            // C = A B
void mat_adjoint(int n, const zd* A, zd* out);                   // out = A^dag
void expm(int n, const zd* A, zd* out);                          // FP64
void expm_frechet_adjoint(int n, const zd* K, const zd* H, zd* out);
double unitarity_error(int n, const zd* U);
RotProgram decompose_adjacent(int n, const zd* U);

// Window steps of a Givens program: step s applies the listed rotations
// (indices into RotProgram::g, in program order), all acting on orbitals
// inside [a, a + W).
struct WinStep {
  int a;
  std::vector<int> givens;
};
std::vector<WinStep> schedule_windows(const RotProgram& rp, int N, int W);
// Orbit tables of the strings of n electrons in N orbitals for windows of W
// adjacent orbitals: for each window position a, orbits[off[a] .. off[a+1])
// hold R_O | c_lo << 16 | m << 24 grouped by m (classes in descending order
// of work, each padded with empty descriptors, m = 0, to a multiple of 32),
// okey[i] is the occupation of
// the top three orbitals in orbit i's outside configuration (a 3-bit
// number), and offs[((a * (n+1) + c_lo) << W) + S] is the in-window rank
// offset.
void window_tables_host(int N, int n, int W, std::vector<uint32_t>& orbits,
                        std::vector<int>& off, std::vector<uint16_t>& offs,
                        std::vector<uint8_t>& okey);
// The orbits regrouped for clusters of 2^b CTAs: per window position a,
// group r (occupation of the top b orbitals, the strings of cluster rank r)
// at gorb[goff[a * 9 + r] .. goff[a * 9 + r + 1]), class order kept inside,
// without the padding.
void window_groups_host(const std::vector<uint32_t>& orbits, const std::vector<int>& off,
                        const std::vector<uint8_t>& okey, int b, std::vector<uint32_t>& gorb,
                        std::vector<int>& goff);

// One segment of the gather indices of the tensor-core window steps: for a
// window position (and, for a cluster, one rank's orbits), the orbits of the
// classes m = 3, 2, 4, 1, 5 in that order, each orbit a row of its C(6, m)
// string addresses (ascending local masks) padded to a multiple of 8;
// idx[start .. start + len) in uint16 units (both multiples of 8), cnt[i]
// orbits of the i-th class.
struct TcSeg {
  int start, len;
  int cnt[5];
  int pad_;
};

// Device copy of a pass: the subset, the owned slots, the record range.
// mode: 2 = the pass owns all 16 local slots, 1 = all twelve off-diagonal
// slots and no diagonal, 0 = any other ownership (tested per slot).
struct TPassDev {
  int q[4];
  uint32_t keep;
  int rec0, rec1;
  int mode;
};
// Transition-reduction passes (see tpass_tables_host): a subset of four
// orbitals q[0] < .. < q[3], the local slots (i*4 + j <-> E_{q_i q_j}) this
// pass owns, and its orbit records recs[rec0 .. rec1) grouped by m (classes
// in descending order of work, each padded with empty records to a multiple
// of 32).
struct TPass {
  int q[4];
  uint32_t keep;
  int rec0, rec1;
};
struct alignas(16) TRecord {
  uint16_t addr[6];  // addresses of O u S, S in ascending local-mask order
  uint8_t m;         // electrons inside the subset
  uint8_t gbits;     // bit j: parity of |O| between q_0 and q_j (j = 1..3)
  uint16_t flips;    // bit k: omega(S_k), the parity of the gbits of S_k's orbitals
};
// rkey[i]: occupation of the top three orbitals in record i's configuration
// outside the subset (a 3-bit number).
void tpass_tables_host(int N, int n, std::vector<TPass>& passes,
                       std::vector<TRecord>& recs, std::vector<uint8_t>& rkey);
// The records regrouped for clusters of 2^b CTAs: per pass i, group r at
// grec[goff[i * 9 + r] .. goff[i * 9 + r + 1]), class order kept inside,
// without the padding.
void tpass_groups_host(const std::vector<TPass>& passes, const std::vector<TRecord>& recs,
                       const std::vector<uint8_t>& rkey, int b, std::vector<TRecord>& grec,
                       std::vector<int>& goff);

// ------------------------------------------------------ device tables
// Per-sector-spin tables: strings of `nocc` electrons in `norb` orbitals.
struct Space {
  int norb = 0, nocc = 0;
  int64_t dim = 0;
  uint32_t* masks = nullptr;  // [dim] string masks in address order
  uint32_t* pairs = nullptr;  // [(norb-1) * npp]: adjacent Givens pair lists
  int npp = 0;                // C(norb-2, nocc-1) pairs per adjacent (p, p+1)
  // pair lists for all ordered (p, q), p != q, and the diagonal lists, used by
  // the transition one-body reductions
  uint32_t* xpairs = nullptr;  // [norb*norb][nx] packed (src | dst << 16)
  uint32_t* xsign = nullptr;   // [norb*norb][ceil(nx/32)] sign bits
  int nx = 0;                  // entries per (p, q) list (max over p, q)
  int* xcount = nullptr;       // [norb*norb] actual entries per list
  // window tables for the register-blocked sweeps, per window width W:
  // orbit descriptors R_O | c_lo << 16 | m << 24 grouped by window position
  // and grouped by m (padded per class), and in-window rank offsets
  // F[a][c_lo][S]
  struct Win {
    uint32_t* orbits = nullptr;
    int* off = nullptr;
    uint16_t* offs = nullptr;
    bool built = false;
    // regrouped for clusters of 2^b CTAs (index b), built on first use from
    // the host copies
    uint32_t* gorb[4] = {};
    int* goff[4] = {};
    // gather indices of the tensor-core steps (W = 6 only), for the whole
    // orbit list (b = 0) and for the rank groups of 2-CTA clusters (b = 1)
    TcSeg* tc_seg[2] = {};
    uint16_t* tc_idx[2] = {};
    int tc_seg_max[2] = {};  // largest segment, bytes
    std::vector<uint32_t> orb_h;
    std::vector<int> off_h;
    std::vector<uint8_t> okey_h;
  } win[8];
  // transition-reduction passes (reverse mode), built on first use, and the
  // records regrouped for clusters of 2^b CTAs
  struct TPassDev* tpass = nullptr;
  struct TRecord* trec = nullptr;
  int npass = 0;
  bool tbuilt = false;
  struct TRecord* tgrec[4] = {};
  int* tgoff[4] = {};
  std::vector<TPass> tpass_h;
  std::vector<TRecord> trec_h;
  std::vector<uint8_t> rkey_h;
  // single-excitation gather table (operator action), built on first use:
  // per string t, ne = n(N-n)+n entries (pq = p*N+q, src = E_qp t | sign<<31)
  uint16_t* gpq = nullptr;
  uint32_t* gsrc = nullptr;
  int ne = 0;
};

struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct ProfRec {
  std::string name;
  cudaEvent_t a, b;
  int kernels;
};

struct Ctx {
  int device = 0;
  // autotuned orbital-rotation method per (norb, n_alpha, n_beta, dtype)
  std::map<std::tuple<int, int, int, int>, int> rot_choice;
  // autotuned slab width (log2 of vectors per CTA) of the batched sweeps per
  // (norb, electrons of the rotated and the other spin, dtype, states,
  // reverse, cross term, shared-memory budget in KB), and the timings behind
  // each choice (ms per launch for lgKV = 0, 1, ...); tuned on first use on
  // a private stream
  std::map<std::array<int, 8>, int> sweep_tune;
  std::map<std::array<int, 8>, std::vector<float>> sweep_tune_ms;
  cudaStream_t tune_stream = nullptr;
  int batch_tuning = 1;
  bool prof_on = false;
  std::vector<ProfRec> prof;
  cudaDeviceProp prop{};
  int rot_path = FS_ROT_AUTO;
  int sweep_engine = FS_SWEEP_AUTO;
  std::map<std::pair<int, int>, Space*> spaces;
  std::map<std::string, Scratch> scratch;
  int* d_status = nullptr;  // device status word
  // small results the host needs right away (transition sums, coupling
  // gradients) land in a mapped pinned buffer, written by a kernel: a copy
  // through a copy engine would wait behind the caller's own large copies
  double* h_stage = nullptr;      // host address
  double* h_stage_dev = nullptr;  // its device address
  size_t h_stage_bytes = 0;
  // private non-blocking stream on which batched launches are captured into
  // a graph (a capture cannot run on the legacy default stream); the graph
  // itself is launched on the caller's stream
  cudaStream_t capture_stream = nullptr;
  std::mutex mu;
};

// Kernel tracing: when the current context has profiling on, every launch
// helper brackets its kernel with CUDA events on the launch stream.
Ctx*& current_ctx();
void prof_begin(cudaStream_t st, cudaEvent_t* a);
void prof_end(const char* name, cudaStream_t st, cudaEvent_t a, int kernels);
struct ProfScope {  // brackets `kernels` kernel launches
  const char* name;
  cudaStream_t st;
  int kernels;
  cudaEvent_t a = nullptr;
  ProfScope(const char* n, cudaStream_t s, int k = 1) : name(n), st(s), kernels(k) {
    prof_begin(st, &a);
  }
  ~ProfScope() { prof_end(name, st, a, kernels); }
};

Space* get_space(Ctx* ctx, int norb, int nocc, cudaStream_t st);
void free_space(Space* s);
void* scratch(Ctx* ctx, const std::string& name, size_t bytes);

// ------------------------------------------------------------- errors
void set_error(const std::string& msg);
struct Fail {
  int code;
};
#define FS_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      ::fs::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));     \
      throw ::fs::Fail{FS_ERR_CUDA};                                           \
    }                                                                          \
  } while (0)
#define FS_REQUIRE(cond, code, msg)    \
  do {                                 \
    if (!(cond)) {                     \
      ::fs::set_error(msg);            \
      throw ::fs::Fail{code};          \
    }                                  \
  } while (0)

// Runs the body of a C entry point and maps what it throws to a status
// code: Fail carries its own code, a failed host allocation is
// FS_ERR_NOMEM, any other standard exception FS_ERR_ARG.
template <class F>
static int guarded(F&& f) {
  try {
    f();
    return FS_OK;
  } catch (Fail& e) {
    return e.code;
  } catch (std::bad_alloc&) {
    set_error("host allocation failed");
    return FS_ERR_NOMEM;
  } catch (std::exception& e) {
    set_error(e.what());
    return FS_ERR_ARG;
  }
}

// ------------------------------------------------------ kernel launchers
// Small matrices travel to the kernels by value, as kernel parameters.
struct Mat {
  double v[kMaxOrb * kMaxOrb];
};
struct CMat {
  double v[2 * kMaxOrb * kMaxOrb];
};
struct StrPhase {  // per-string factor recipe, see launch_string_phase
  int use_d = 0, use_j = 0, use_lam = 0;
  double t = 0;
  double d[2 * kMaxOrb];
  double lam[kMaxOrb];
  Mat J;
};

// Phase of one configuration, factored as
//   f(i, j) = ea_a[i] * ea_b[j] * exp(i sum_{p in I_a, q in I_b} X[p][q])
// with per-string factor tables ea_* (device, may be null = 1) and a real
// cross matrix X (unused when has_x == 0).
struct PhaseDev {
  const void* ea_a = nullptr;
  const void* ea_b = nullptr;
  int has_x = 0;
  Mat X;
};

// Per-string factors: out[e] = prod_{p in I} d_p * exp(i(-(t/2) sum_{p,q in I} J[p][q]
//                                                    - t sum_{p in I} lam[p])).
void launch_string_phase(const Space* sp, void* out, int dtype, const StrPhase& f,
                         cudaStream_t st);

// Window program: step s applies Givens g0[s] .. g0[s+1]-1, all acting on
// orbitals inside the window [a[s], a[s] + W); u = p - a[s] is the local
// index of the rotated pair (p, p+1); pat[s] >= 0 names the step's
// u-sequence among the compile-time window patterns (-1: none).
// Coefficients of each rotation G = [[c, s], [-s*, c]] (c >= 0, as the
// adjacent decomposition makes it).  complex128 keeps c, Re s, Im s as
// doubles and updates a pair directly: x' = c x + s y, y' = -s* x + c y.
// complex64 keeps the shear form G = [[1, tau], [0, 1]] [[1, 0], [sig, 1]]
// [[1, tau], [0, 1]] with tau = s / (1 + c) and sig = -s* (so 1 + tau sig
// = c and tau (1 + c) = s): x += tau y; y += sig x; x += tau y, three
// complex multiply-adds that each update one amplitude in place, so a
// rotation leaves its amplitudes in the registers it found them in.  Since
// c >= 0, |tau| <= |s| <= 1.  Each complex64 coefficient is stored as a pair
// (x, x) for the packed two-lane FP32 updates (and Im tau once more negated),
// read as floats by the one-lane updates.
template <typename R>
struct GCoef {  // one rotation, direct form
  R c, sr, si;
};
template <>
struct GCoef<float> {  // one rotation, shear form
  float tr, ti, gr, gi;
};
template <typename R>
struct WCoef {
  R c[kMaxGivens];
  R sr[kMaxGivens];
  R si[kMaxGivens];
  __host__ __device__ GCoef<R> coef(int q) const { return GCoef<R>{c[q], sr[q], si[q]}; }
  __host__ void set(int q, double cv, double srv, double siv) {
    c[q] = (R)cv;
    sr[q] = (R)srv;
    si[q] = (R)siv;
  }
};
template <>
struct WCoef<float> {
  float2 tr2[kMaxGivens];   // Re tau
  float2 ti2[kMaxGivens];   // Im tau
  float2 nti2[kMaxGivens];  // -Im tau
  float2 gr2[kMaxGivens];   // Re sig = -Re s
  float2 gi2[kMaxGivens];   // Im sig = Im s
  __host__ __device__ GCoef<float> coef(int q) const {
    return GCoef<float>{tr2[q].x, ti2[q].x, gr2[q].x, gi2[q].x};
  }
  __host__ void set(int q, double cv, double srv, double siv) {
    const float tr = (float)(srv / (1.0 + cv)), ti = (float)(siv / (1.0 + cv));
    tr2[q] = make_float2(tr, tr);
    ti2[q] = make_float2(ti, ti);
    nti2[q] = make_float2(-ti, -ti);
    gr2[q] = make_float2((float)-srv, (float)-srv);
    gi2[q] = make_float2((float)siv, (float)siv);
  }
};
template <typename R>
struct WProg : WCoef<R> {
  int nsteps;
  int8_t a[kMaxGivens];
  int8_t pat[kMaxGivens];
  int16_t g0[kMaxGivens + 1];
  int8_t u[kMaxGivens];
};

// Geometry and phase/reduction pointers of one sweep launch (one job of a
// batched launch).
struct SweepGeom {
  void* st[2];
  int64_t d_b;  // row stride of the state
  int dir;      // 0: alpha, vectors are columns; 1: beta, vectors are rows
  int d;        // vector length (strings of the rotated spin)
  int nvec;     // number of vectors (strings of the other spin)
  int lgKV;     // log2 of vectors per slab
  int chunk;    // vector elements held by one CTA of the cluster (maximum)
  // cluster rank r holds elements [cb[r], cb[r + 1]) of each vector; with
  // `blocked`, rank r holds exactly the strings whose occupation of the top
  // lgcs orbitals reads r (so orbits of windows and subsets clear of those
  // orbitals stay within one CTA)
  int cb[9];
  int lgcs;
  int blocked;
  const uint32_t* pairs;
  int npp;
  const uint32_t* masks_this;
  const uint32_t* masks_other;
  int norb;
  int nchunk;  // 8-bit chunks of a string mask
  const void* ea_this;
  const void* ea_other;
  int has_x;  // cross angles X[p_alpha][q_beta] are passed separately
  // reverse mode (dual state: st[0] = psi, st[1] = cotangent g)
  const void* ea2_this;   // second phase (applied after the reductions)
  const void* ea2_other;
  const uint32_t* xpairs;  // E_pq pair lists of the rotated spin
  const uint32_t* xsign;
  const int* xcount;
  int nx;
  double* T;  // [norb][norb] complex accumulator: += <g| E_pq |psi>
  void* W;    // [d_a][d_b] real: Im(conj(g) psi), or null
  // transition-reduction passes of the rotated spin (reverse mode, N >= 4)
  const TPassDev* tpass;
  const TRecord* trec;
  int npass;
  // window tables of the rotated spin (window kernels only)
  const uint32_t* orbits;  // per window position, orbit descriptors grouped by m
  const int* orb_off;      // [npos + 1] start of each position's list
  // blocked clusters: orbits regrouped by cluster rank, rank r's orbits of
  // position a at orb_grp[orb_goff[a * 9 + r] .. orb_goff[a * 9 + r + 1]);
  // records likewise, rank r's of pass i at trec_grp[tgoff[i * 9 + r] ..)
  const uint32_t* orb_grp;
  const int* orb_goff;
  const TRecord* trec_grp;
  const int* tgoff;
  const uint16_t* offs;    // [npos][nocc + 1][1 << W] in-window rank offsets
  int offs_stride;         // (nocc + 1) << W
  // tensor-core window steps (W = 6): per step the B images of classes
  // m = 1..5 (tc::kStepBytes each step); gather-index segments per window
  // position (seg_full[a]) and, for blocked clusters, per position and rank
  // (seg_grp[a * 2 + rank]); idx_cap = bytes of one staged segment buffer
  const unsigned char* tc_b;
  const TcSeg* tc_seg_full;
  const uint16_t* tc_idx_full;
  const TcSeg* tc_seg_grp;
  const uint16_t* tc_idx_grp;
  int tc_idx_cap;
  int* status;  // device status word (bounded waits that gave up)
};

struct SweepJob {
  SweepGeom g;
  const void* prog;  // WProg<R> in device memory
  const Mat* X;      // device memory
  int item0;         // first work item of this job in the batched launch
};
struct BatchSweepPlan {
  SweepGeom g;
  int nslabs = 0;
  size_t smem = 0;
  bool pk = false;                  // packed vector pairs (complex64 forward)
  std::vector<unsigned char> prog;  // WProg<R> bytes
};
size_t wprog_bytes(int dtype);
void plan_batch_sweep(Ctx* ctx, Space* sa, Space* sb, int dir, void* st0, void* st1, int nst,
                      int dtype, const RotProgram& rp, const PhaseDev& ph, const struct RevArgs* rev,
                      size_t budget, BatchSweepPlan& out);
// jobs == nullptr: only set the kernel's shared-memory attribute.
// pk: every job's slab holds an even number of vectors (complex64 forward
// sweeps then run on packed vector pairs)
void launch_sweep_batch(Ctx* ctx, int dtype, int nst, const SweepJob* jobs, int njobs, int total,
                        int* counter, size_t smem, cudaStream_t st, bool pk = false);
void lucj_batch(Ctx* ctx, int n, const fs_lucj* ops, void* const* vecs, void* const* cots,
                int dtype, int do_vjp, double* const* dK, double* const* dJaa,
                double* const* dJab, cudaStream_t st);

// Reverse-mode extras of a dual-state sweep (st0 = psi, st1 = cotangent).
struct RevArgs {
  const void* ea2_a = nullptr;  // second phase, applied after the reductions
  const void* ea2_b = nullptr;
  double* T = nullptr;  // [norb][norb] complex, += <g| E_pq |psi> (this spin)
  void* W = nullptr;    // [d_a][d_b] real Im(conj(g) psi), or null
};

// Givens sweep over one spin: dir 0 rotates alpha (columns of the state),
// dir 1 rotates beta (rows).  With nst == 1 the epilogue multiplies by the
// phase `ph` (strings of both spins, cross matrix ph.X).  With nst == 2
// (reverse mode, `rev` required) both states get the program, then the
// per-string factors of `ph` (no cross term), then the reductions of `rev`,
// then the phase rev->ea2_* times the cross term ph.X.
void launch_sweep(Ctx* ctx, const Space* sa, const Space* sb, int dir,
                  void* st0, void* st1, int nst, int dtype,
                  const RotProgram& prog, const PhaseDev& ph, cudaStream_t st,
                  const RevArgs* rev = nullptr);

// dJ from W = Im(conj(g) psi) of one diagonal-Coulomb gate (t = 1):
//   dJ_ab[p][q] += sum_{ij} W_ij occ_a(i)_p occ_b(j)_q
//   dJ_aa[p][q] += 1/2 sum_{ij} W_ij (occ_a(i)_p occ_a(i)_q + occ_b(j)_p occ_b(j)_q)
// dJ_aa, dJ_ab: device [norb][norb] FP64 accumulators.
void build_gather_table(Space* sp, cudaStream_t st);
// H vec for a molecular Hamiltonian with real tensors (operator action);
// workspace_bytes bounds the intermediate blocks (0: automatic).
void molecular_hamiltonian(Ctx* ctx, Space* sa, Space* sb, const void* vec, void* out, int dtype,
                           const double* h1, const double* h2, double constant,
                           int64_t workspace_bytes, cudaStream_t st);
// Configurations drawn from |vec|^2 by inverse CDF in address order, for
// `shots` device uniforms; n = dim_a * dim_b amplitudes.
void sample_state(Ctx* ctx, const void* vec, int dtype, int64_t n, const double* u,
                  int64_t shots, int64_t* out, cudaStream_t st);
// Occupation masks (words of 64 bits per shot) of one spin of a Slater
// determinant with occupied columns Phi (N x n, row-major, orthonormal).
void sample_slater(Ctx* ctx, const std::vector<zd>& Phi, int N, int n, const double* u,
                   int64_t shots, uint64_t* out, cudaStream_t st);
// out = in^T for a [rows][cols] complex state (tiled, HBM-bound).
// out[0 .. na) = a, out[na .. na + nb) = b, out[na + nb .. na + nb + nc) = c
// (b, c may be null with nb, nc = 0); out may be a mapped host address.
void launch_gather_f64(const double* a, int64_t na, const double* b, int64_t nb,
                       const double* c, int64_t nc, double* out, cudaStream_t st);
void launch_transpose(const void* in, void* out, int64_t rows, int64_t cols, int dtype,
                      cudaStream_t st);
void launch_dc_grad(Ctx* ctx, const Space* sa, const Space* sb, const void* W, int dtype,
                    double* dJ_aa, double* dJ_ab, cudaStream_t st);

// Multiply the state by the phase `ph` (one streaming pass).
void launch_phase(const Space* sa, const Space* sb, void* vec, int dtype,
                  const PhaseDev& ph, cudaStream_t st);
// The same pass with the cross term contracted on the tensor cores
// (complex64, norb <= 32; needs scratch for the per-column angle table).
bool phase_tc_supported(int dtype, const Space* sa, const Space* sb, const void* vec);
void launch_phase_tc(Ctx* ctx, const Space* sa, const Space* sb, void* vec, const PhaseDev& ph,
                     cudaStream_t st);

// Hartree-Fock closed form (§2.4): psi[i][j] = det(R[I_a(i), 0..n_a-1]) *
// det(R[I_b(j), 0..n_b-1]) for the N x N matrix R, computed in FP64.
void launch_slater(Ctx* ctx, const Space* sa, const Space* sb, void* vec, int dtype,
                   const CMat& R, cudaStream_t st);

void launch_exc_table(const Space* sp, uint32_t* out, cudaStream_t st);

// Dense minor-matrix rotation psi <- M_a psi M_b^T (§2.3), U_a and U_b by
// value.  Supported for string dimensions up to kMaxMinorDim.
bool minor_path_supported(const Space* sa, const Space* sb);
void launch_minor_rotation(Ctx* ctx, const Space* sa, const Space* sb, void* vec, int dtype,
                           const CMat& Ua, const CMat& Ub, cudaStream_t st);
// masks[dim] of the strings of nocc electrons in norb orbitals, into `out`.
void launch_masks(uint32_t* out, int norb, int nocc, cudaStream_t st);
// ------------------------------------------------ tensor-core GEMM
// C[m][n] = sum_k A[m][k] B[n][k] on the tcgen05 tensor cores with both
// operands as three exact BF16 pieces (K contiguous, rows a multiple of 16
// bytes apart), FP32 accuracy (fs_gemm_tc.cu).  Output forms:
//   GEMM_REAL:          float out[m * ldo + n];
//   GEMM_REAL_T:        float out[n * ldo + m];
//   GEMM_CPLX_T:        N even, (C[m][2j], C[m][2j+1]) is the complex
//                       float2 out[j * ldo + m];
//   GEMM_CPLX_T_PLANES: as GEMM_CPLX_T, written as the three BF16 planes
//                       outp[p] (row j, columns 2m, 2m + 1; row stride ldp).
enum { GEMM_REAL = 0, GEMM_REAL_T = 1, GEMM_CPLX_T = 2, GEMM_CPLX_T_PLANES = 3 };
struct GemmTc {
  const uint16_t* A[3];
  const uint16_t* B[3];
  int M, N, K;
  int64_t lda, ldb;
  void* out;
  int mode;
  int64_t ldo;
  void* outp[3];
  int64_t ldp;
  int* status;
};
void gemm_tc(const GemmTc& g, cudaStream_t st);
// The three BF16 planes of a complex matrix X (rows x cols, leading
// dimension ldx complex) with row stride ldk (>= 2 cols, a multiple of 8;
// the padding is zeroed).
void split_planes(const void* X, int64_t rows, int cols, int64_t ldx, void* const planes[3],
                  int64_t ldk, cudaStream_t st);

// Force the module loads of the kernels the allocation-free entry point
// launches (k_masks; k_string_phase and k_phase in both precisions), so
// that none of them loads lazily on a later call.
void preload_mask_kernel();
void preload_phase_kernels();

}  // namespace fs
