// C ABI of libfsgpu.so: argument checks, context and scratch management, and
// the host-side orchestration of the kernels for each gate (§3.2) and for
// the LUCJ ansatz (§4.3, §4.5.1).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "fs_internal.h"

namespace fs {

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }

Ctx*& current_ctx() {
  static thread_local Ctx* c = nullptr;
  return c;
}
void prof_begin(cudaStream_t st, cudaEvent_t* a) {
  Ctx* c = current_ctx();
  *a = nullptr;
  if (!c || !c->prof_on) return;
  if (cudaEventCreate(a) != cudaSuccess || cudaEventRecord(*a, st) != cudaSuccess) *a = nullptr;
}
void prof_end(const char* name, cudaStream_t st, cudaEvent_t a, int kernels) {
  Ctx* c = current_ctx();
  if (!a || !c) return;
  cudaEvent_t b;
  if (cudaEventCreate(&b) != cudaSuccess) return;
  cudaEventRecord(b, st);
  c->prof.push_back(ProfRec{name, a, b, kernels});
}

void* scratch(Ctx* ctx, const std::string& name, size_t bytes) {
  Scratch& s = ctx->scratch[name];
  if (s.bytes < bytes) {
    if (s.ptr) FS_CUDA(cudaFree(s.ptr));
    s.ptr = nullptr;
    s.bytes = 0;
    cudaError_t e = cudaMalloc(&s.ptr, bytes);
    if (e != cudaSuccess) {
      set_error("scratch allocation of " + std::to_string(bytes) + " bytes failed: " +
                cudaGetErrorString(e));
      throw Fail{FS_ERR_NOMEM};
    }
    s.bytes = bytes;
  }
  return s.ptr;
}

static std::vector<zd> load_cmat(const double* p, int n) {
  std::vector<zd> m((size_t)n * n);
  for (size_t k = 0; k < m.size(); ++k) m[k] = zd(p[2 * k], p[2 * k + 1]);
  return m;
}

static void check_unitary(const std::vector<zd>& U, int n, const char* what) {
  double e = unitarity_error(n, U.data());
  FS_REQUIRE(e <= 1e-10, FS_ERR_NOT_UNITARY,
             std::string(what) + " is not unitary (max |U^dag U - I| = " +
                 std::to_string(e) + ")");
}

static void check_sector(Ctx* ctx, void* vec, int dtype, int norb, int na, int nb) {
  FS_REQUIRE(ctx != nullptr, FS_ERR_ARG, "null context");
  FS_REQUIRE(dtype == FS_C64 || dtype == FS_C128, FS_ERR_ARG, "dtype must be FS_C64 or FS_C128");
  FS_REQUIRE(norb >= 1 && norb <= kMaxNorb, FS_ERR_ARG, "norb must be in [1, 32]");
  FS_REQUIRE(na >= 0 && na <= norb && nb >= 0 && nb <= norb, FS_ERR_ARG,
             "electron counts must be in [0, norb]");
  FS_REQUIRE(vec != nullptr, FS_ERR_ARG, "null state pointer");
  FS_REQUIRE(((uintptr_t)vec & 15u) == 0, FS_ERR_ARG, "state pointer must be 16-byte aligned");
}

static Mat real_mat(const double* p, int n, double scale) {
  Mat m;
  for (int k = 0; k < n * n; ++k) m.v[k] = scale * p[k];
  return m;
}

static StrPhase phase_of(const RotProgram* rp, const double* J, double t, const double* lam,
                         int n) {
  StrPhase f;
  f.t = t;
  if (rp) {
    f.use_d = 1;
    for (int p = 0; p < n; ++p) {
      f.d[2 * p] = rp->phase[p].real();
      f.d[2 * p + 1] = rp->phase[p].imag();
    }
  }
  if (J) {
    f.use_j = 1;
    for (int k = 0; k < n * n; ++k) f.J.v[k] = J[k];
  }
  if (lam) {
    f.use_lam = 1;
    for (int p = 0; p < n; ++p) f.lam[p] = lam[p];
  }
  return f;
}

// A diagonal-Coulomb evolution fused into the epilogue of a beta sweep:
// same-spin matrix J (J_bb = J_aa), mixed matrix J_ab, time t.
struct Fused {
  const double* J_aa = nullptr;  // host, N x N
  const double* J_ab = nullptr;  // host, N x N
  const double* J_bb = nullptr;  // host, N x N; null means J_aa
  double t = 0;
};

// Orbital rotation with programs pa (alpha) and pb (beta): one sweep per
// spin.  The beta sweep's epilogue also applies the optional fused
// diagonal-Coulomb evolution `dc`.
static void rotate(Ctx* ctx, Space* sa, Space* sb, void* v0, void* v1, int nst, int dtype,
                   const RotProgram& pa, const RotProgram& pb, const Fused* dc,
                   cudaStream_t st) {
  const int n = sa->norb;
  const size_t csz = dtype == FS_C64 ? 8 : 16;
  void* ea_a = scratch(ctx, "ea_a", sa->dim * csz);
  void* ea_b = scratch(ctx, "ea_b", sb->dim * csz);
  void* ea_o = scratch(ctx, "ea_o", sa->dim * csz);
  launch_string_phase(sa, ea_a, dtype, phase_of(&pa, nullptr, 0, nullptr, n), st);
  PhaseDev ph;
  ph.ea_a = ea_a;
  launch_sweep(ctx, sa, sb, 0, v0, v1, nst, dtype, pa, ph, st);
  PhaseDev phb;
  if (dc) {
    launch_string_phase(sb, ea_b, dtype,
                        phase_of(&pb, dc->J_bb ? dc->J_bb : dc->J_aa, dc->t, nullptr, n), st);
    launch_string_phase(sa, ea_o, dtype, phase_of(nullptr, dc->J_aa, dc->t, nullptr, n), st);
    phb.ea_a = ea_o;
    phb.has_x = 1;
    // mixed terms (p in I_a, q in I_b) and (p in I_b, q in I_a), J_ba = J_ab^T
    phb.X = real_mat(dc->J_ab, n, -dc->t);
  } else {
    launch_string_phase(sb, ea_b, dtype, phase_of(&pb, nullptr, 0, nullptr, n), st);
  }
  phb.ea_b = ea_b;
  launch_sweep(ctx, sa, sb, 1, v0, v1, nst, dtype, pb, phb, st);
}

// The same rotation (and fused diagonal-Coulomb evolution) with every sweep a
// row sweep: the state alternates between vec (row-major, alpha strings on
// rows) and tv = vec^T (beta strings on rows).  From vec (trans false): the
// beta sweep on rows of vec, one transpose, then the alpha sweep on rows of
// tv with the evolution in its epilogue; from tv the other way round.  The
// two spin parts commute, so the order is free; each rotation costs one
// transpose instead of a column sweep.  `trans` is flipped.
static void rotate_alternating(Ctx* ctx, Space* sa, Space* sb, void* vec, void* tv, bool& trans,
                               int dtype, const RotProgram& pa, const RotProgram& pb,
                               const Fused* dc, cudaStream_t st) {
  const int n = sa->norb;
  const size_t csz = dtype == FS_C64 ? 8 : 16;
  void* ea_a = scratch(ctx, "ea_a", sa->dim * csz);
  void* ea_b = scratch(ctx, "ea_b", sb->dim * csz);
  void* eo_a = scratch(ctx, "alt_eo_a", sa->dim * csz);
  void* eo_b = scratch(ctx, "alt_eo_b", sb->dim * csz);
  const double* Jbb = dc ? (dc->J_bb ? dc->J_bb : dc->J_aa) : nullptr;
  if (!trans) {
    launch_string_phase(sb, ea_b, dtype, phase_of(&pb, nullptr, 0, nullptr, n), st);
    PhaseDev p1;
    p1.ea_b = ea_b;
    launch_sweep(ctx, sa, sb, 1, vec, nullptr, 1, dtype, pb, p1, st);
    launch_transpose(vec, tv, sa->dim, sb->dim, dtype, st);
    // alpha on rows of tv: spaces swapped, this spin (alpha) in the b slot
    PhaseDev p2;
    if (dc) {
      launch_string_phase(sa, ea_a, dtype, phase_of(&pa, dc->J_aa, dc->t, nullptr, n), st);
      launch_string_phase(sb, eo_b, dtype, phase_of(nullptr, Jbb, dc->t, nullptr, n), st);
      p2.ea_a = eo_b;
      p2.has_x = 1;
      for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) p2.X.v[q * n + p] = -dc->t * dc->J_ab[p * n + q];
    } else {
      launch_string_phase(sa, ea_a, dtype, phase_of(&pa, nullptr, 0, nullptr, n), st);
    }
    p2.ea_b = ea_a;
    launch_sweep(ctx, sb, sa, 1, tv, nullptr, 1, dtype, pa, p2, st);
    trans = true;
  } else {
    launch_string_phase(sa, ea_a, dtype, phase_of(&pa, nullptr, 0, nullptr, n), st);
    PhaseDev p1;
    p1.ea_b = ea_a;
    launch_sweep(ctx, sb, sa, 1, tv, nullptr, 1, dtype, pa, p1, st);
    launch_transpose(tv, vec, sb->dim, sa->dim, dtype, st);
    PhaseDev p2;
    if (dc) {
      launch_string_phase(sb, ea_b, dtype, phase_of(&pb, Jbb, dc->t, nullptr, n), st);
      launch_string_phase(sa, eo_a, dtype, phase_of(nullptr, dc->J_aa, dc->t, nullptr, n), st);
      p2.ea_a = eo_a;
      p2.has_x = 1;
      p2.X = real_mat(dc->J_ab, n, -dc->t);
    } else {
      launch_string_phase(sb, ea_b, dtype, phase_of(&pb, nullptr, 0, nullptr, n), st);
    }
    p2.ea_b = ea_b;
    launch_sweep(ctx, sa, sb, 1, vec, nullptr, 1, dtype, pb, p2, st);
    trans = false;
  }
}

// Whether the LUCJ passes alternate layouts: states larger than L2 (column
// sweeps are strided there) when `extra` more states fit in device memory.
static bool alternate_layouts(Ctx* ctx, Space* sa, Space* sb, int dtype, int extra,
                              const char* const* names) {
  const size_t S = (size_t)sa->dim * sb->dim * (dtype == FS_C64 ? 8 : 16);
  if (S <= (size_t)ctx->prop.l2CacheSize) return false;
  bool have = true;
  for (int k = 0; k < extra; ++k) have = have && ctx->scratch[names[k]].bytes >= S;
  if (have) return true;
  size_t fr = 0, tot = 0;
  return cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr > extra * S + (1ull << 30);
}

// Standalone diagonal phase pass (number-operator sum and/or diagonal Coulomb).
static void phase_pass(Ctx* ctx, Space* sa, Space* sb, void* vec, int dtype,
                       const StrPhase& fa, const StrPhase& fb, const double* J_ab,
                       double xscale, cudaStream_t st) {
  const size_t csz = dtype == FS_C64 ? 8 : 16;
  void* ea_a = scratch(ctx, "ea_a", sa->dim * csz);
  void* ea_b = scratch(ctx, "ea_b", sb->dim * csz);
  launch_string_phase(sa, ea_a, dtype, fa, st);
  launch_string_phase(sb, ea_b, dtype, fb, st);
  PhaseDev ph;
  ph.ea_a = ea_a;
  ph.ea_b = ea_b;
  if (J_ab) {
    ph.has_x = 1;
    ph.X = real_mat(J_ab, sa->norb, xscale);
  }
  if (ph.has_x && phase_tc_supported(dtype, sa, sb, vec))
    launch_phase_tc(ctx, sa, sb, vec, ph, st);
  else
    launch_phase(sa, sb, vec, dtype, ph, st);
}

static CMat cmat_of(const std::vector<zd>& U, int n) {
  CMat m{};
  for (int k = 0; k < n * n; ++k) {
    m.v[2 * k] = U[k].real();
    m.v[2 * k + 1] = U[k].imag();
  }
  return m;
}

// Orbital rotation by the selected method.  FS_ROT_AUTO measures both
// methods once per (sector, dtype) on a scratch copy of the state (the
// first such call synchronizes the stream) and keeps the faster.
static void rotate_any(Ctx* ctx, Space* sa, Space* sb, void* vec, int dtype,
                       const std::vector<zd>& Ua, const std::vector<zd>& Ub,
                       const RotProgram& pa, const RotProgram& pb, cudaStream_t st) {
  const int n = sa->norb;
  int path = ctx->rot_path;
  if (path == FS_ROT_AUTO) {
    if (!minor_path_supported(sa, sb)) {
      path = FS_ROT_GIVENS;
    } else {
      auto key = std::make_tuple(n, sa->nocc, sb->nocc, dtype);
      auto it = ctx->rot_choice.find(key);
      if (it != ctx->rot_choice.end()) {
        path = it->second;
      } else {
        const size_t bytes = sa->dim * sb->dim * (dtype == FS_C64 ? 8 : 16);
        void* tv = scratch(ctx, "autotune_state", bytes);
        FS_CUDA(cudaMemcpyAsync(tv, vec, bytes, cudaMemcpyDeviceToDevice, st));
        cudaEvent_t e[3];
        for (auto& x : e) FS_CUDA(cudaEventCreate(&x));
        float tg = 0, tm = 0;
        for (int rep = 0; rep < 2; ++rep) {  // first round warms up
          FS_CUDA(cudaEventRecord(e[0], st));
          for (int k = 0; k < 3; ++k) rotate(ctx, sa, sb, tv, nullptr, 1, dtype, pa, pb, nullptr, st);
          FS_CUDA(cudaEventRecord(e[1], st));
          for (int k = 0; k < 3; ++k)
            launch_minor_rotation(ctx, sa, sb, tv, dtype, cmat_of(Ua, n), cmat_of(Ub, n), st);
          FS_CUDA(cudaEventRecord(e[2], st));
          FS_CUDA(cudaEventSynchronize(e[2]));
          FS_CUDA(cudaEventElapsedTime(&tg, e[0], e[1]));
          FS_CUDA(cudaEventElapsedTime(&tm, e[1], e[2]));
        }
        for (auto& x : e) cudaEventDestroy(x);
        path = tm < tg ? FS_ROT_MINORS : FS_ROT_GIVENS;
        ctx->rot_choice[key] = path;
      }
    }
  }
  if (path == FS_ROT_MINORS)
    launch_minor_rotation(ctx, sa, sb, vec, dtype, cmat_of(Ua, n), cmat_of(Ub, n), st);
  else
    rotate(ctx, sa, sb, vec, nullptr, 1, dtype, pa, pb, nullptr, st);
}

static void lucj_checks(Ctx* ctx, const fs_lucj* op, void* vec, int dtype) {
  FS_REQUIRE(op != nullptr, FS_ERR_ARG, "null LUCJ operator");
  check_sector(ctx, vec, dtype, op->norb, op->n_alpha, op->n_beta);
  FS_REQUIRE(op->n_reps >= 0, FS_ERR_ARG, "n_reps must be >= 0");
  FS_REQUIRE(op->n_reps == 0 || (op->K && op->J_aa && op->J_ab), FS_ERR_ARG,
             "null LUCJ parameter array");
}

// Merged rotations of the LUCJ circuit: R_0 = U_0^dag, R_k = U_k^dag U_{k-1},
// R_n = U_{n-1}, since U(A) U(B) = U(AB) (§2.3, merging as in §4.3).
static std::vector<std::vector<zd>> lucj_rotations(const fs_lucj* op,
                                                   std::vector<std::vector<zd>>* Us_out) {
  const int n = op->norb, R = op->n_reps;
  const size_t nn = (size_t)n * n;
  std::vector<std::vector<zd>> Us(R), Rs(R + 1, std::vector<zd>(nn));
  for (int k = 0; k < R; ++k) {
    std::vector<zd> K = load_cmat(op->K + 2 * nn * k, n);
    Us[k].resize(nn);
    expm(n, K.data(), Us[k].data());
  }
  std::vector<zd> adj(nn);
  mat_adjoint(n, Us[0].data(), Rs[0].data());
  for (int k = 1; k < R; ++k) {
    mat_adjoint(n, Us[k].data(), adj.data());
    mat_mul(n, adj.data(), Us[k - 1].data(), Rs[k].data());
  }
  Rs[R] = Us[R - 1];
  if (Us_out) *Us_out = Us;
  return Rs;
}

// ------------------------------------------------------------ gate lists
// A circuit of orbital rotations and diagonal-Coulomb evolutions, applied
// with neighbouring rotations multiplied on the host (U(A) U(B) = U(AB),
// §2.3) and every diagonal-Coulomb evolution fused into the beta sweep of
// the rotation before it; one that follows no rotation runs as a phase pass.
struct GateOp {
  int kind = 0;             // 0 orbital rotation, 1 diagonal-Coulomb evolution
  std::vector<zd> Ua, Ub;   // kind 0
  const double *J_aa = nullptr, *J_ab = nullptr, *J_bb = nullptr;  // kind 1
  double t = 0;             // kind 1
};

static void run_gates(Ctx* ctx, Space* sa, Space* sb, void* vec, int dtype,
                      const std::vector<GateOp>& ops, cudaStream_t st) {
  const int n = sa->norb;
  const size_t nn = (size_t)n * n;
  std::vector<zd> I(nn, zd(0)), Pa, Pb, tmp(nn);
  for (int p = 0; p < n; ++p) I[p * n + p] = 1;
  Pa = I;
  Pb = I;
  bool pending = false;
  auto flush = [&](const GateOp* dc) {
    if (pending) {
      RotProgram pa = decompose_adjacent(n, Pa.data());
      RotProgram pb = decompose_adjacent(n, Pb.data());
      Fused f;
      if (dc) {
        f.J_aa = dc->J_aa;
        f.J_ab = dc->J_ab;
        f.J_bb = dc->J_bb;
        f.t = dc->t;
      }
      rotate(ctx, sa, sb, vec, nullptr, 1, dtype, pa, pb, dc ? &f : nullptr, st);
    } else if (dc) {
      phase_pass(ctx, sa, sb, vec, dtype, phase_of(nullptr, dc->J_aa, dc->t, nullptr, n),
                 phase_of(nullptr, dc->J_bb ? dc->J_bb : dc->J_aa, dc->t, nullptr, n), dc->J_ab,
                 -dc->t, st);
    }
    Pa = I;
    Pb = I;
    pending = false;
  };
  for (const GateOp& op : ops) {
    if (op.kind == 0) {
      mat_mul(n, op.Ua.data(), Pa.data(), tmp.data());
      Pa = tmp;
      mat_mul(n, op.Ub.data(), Pb.data(), tmp.data());
      Pb = tmp;
      pending = true;
    } else {
      flush(&op);
    }
  }
  flush(nullptr);
}

// S_order(t) of the Trotter-Suzuki product formulas (Hamiltonian time
// evolution section) as (term, time) pairs, first factor first:
// S_0 = H_1 .. H_L, S_1 = H_1/2 .. H_L/2 H_L/2 .. H_1/2,
// S_k = S_{k-1}(u t)^2 S_{k-1}((1 - 4u) t) S_{k-1}(u t)^2, u = 1/(4 - 4^{1/(2k-1)}).
static void product_formula(int L, double t, int order,
                            std::vector<std::pair<int, double>>& out) {
  if (order == 0) {
    for (int j = 0; j < L; ++j) out.emplace_back(j, t);
  } else if (order == 1) {
    for (int j = 0; j < L; ++j) out.emplace_back(j, t / 2);
    for (int j = L - 1; j >= 0; --j) out.emplace_back(j, t / 2);
  } else {
    const double u = 1.0 / (4.0 - std::pow(4.0, 1.0 / (2 * order - 1)));
    for (int r = 0; r < 2; ++r) product_formula(L, u * t, order - 1, out);
    product_formula(L, (1 - 4 * u) * t, order - 1, out);
    for (int r = 0; r < 2; ++r) product_formula(L, u * t, order - 1, out);
  }
}

// The (term, time) sequence of n_steps steps of S_order(time / n_steps),
// with neighbouring factors of the same term joined (exp(-i H_j a)
// exp(-i H_j b) = exp(-i H_j (a + b)), exact).
static std::vector<std::pair<int, double>> trotter_sequence(int L, double time, int n_steps,
                                                            int order) {
  std::vector<std::pair<int, double>> one, all;
  product_formula(L, time / n_steps, order, one);
  for (int r = 0; r < n_steps; ++r)
    for (const auto& f : one) {
      if (!all.empty() && all.back().first == f.first)
        all.back().second += f.second;
      else
        all.push_back(f);
    }
  return all;
}

// exp(-i t M) for an N x N Hermitian M (host, FP64).
static std::vector<zd> expm_minus_i(int n, const std::vector<zd>& M, double t) {
  std::vector<zd> K(M.size()), U(M.size());
  for (size_t q = 0; q < M.size(); ++q) K[q] = zd(0, -t) * M[q];
  expm(n, K.data(), U.data());
  return U;
}

static std::vector<zd> adjoint_of(int n, const std::vector<zd>& U) {
  std::vector<zd> A(U.size());
  mat_adjoint(n, U.data(), A.data());
  return A;
}

static void check_hermitian(const std::vector<zd>& M, int n, const char* what) {
  double err = 0, scale = 1;
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      err = std::max(err, std::abs(M[p * n + q] - std::conj(M[q * n + p])));
      scale = std::max(scale, std::abs(M[p * n + q]));
    }
  if (err > 1e-10 * scale) {
    set_error(std::string(what) + " is not Hermitian");
    throw Fail{FS_ERR_ARG};
  }
}

}  // namespace fs

using namespace fs;

struct fs_ctx : public fs::Ctx {};

extern "C" {

const char* fs_last_error(void) { return g_err.c_str(); }

int fs_create(fs_ctx** out, int device) {
  return guarded([&] {
    FS_REQUIRE(out != nullptr, FS_ERR_ARG, "null output pointer");
    int n = 0;
    FS_CUDA(cudaGetDeviceCount(&n));
    FS_REQUIRE(device >= 0 && device < n, FS_ERR_ARG, "device index out of range");
    FS_CUDA(cudaSetDevice(device));
    fs_ctx* c = new fs_ctx();
    c->device = device;
    FS_CUDA(cudaGetDeviceProperties(&c->prop, device));
    FS_CUDA(cudaMalloc(&c->d_status, sizeof(int)));
    FS_CUDA(cudaMemset(c->d_status, 0, sizeof(int)));
    *out = c;
  });
}

int fs_destroy(fs_ctx* ctx) {
  return guarded([&] {
    FS_REQUIRE(ctx != nullptr, FS_ERR_ARG, "null context");
    FS_CUDA(cudaSetDevice(ctx->device));
    FS_CUDA(cudaDeviceSynchronize());
    for (auto& kv : ctx->spaces) free_space(kv.second);
    for (auto& kv : ctx->scratch) cudaFree(kv.second.ptr);
    cudaFree(ctx->d_status);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->tune_stream) cudaStreamDestroy(ctx->tune_stream);
    delete ctx;
  });
}

int fs_sync_status(fs_ctx* ctx, void* stream) {
  int code = 0;
  int rc = guarded([&] {
    FS_REQUIRE(ctx != nullptr, FS_ERR_ARG, "null context");
    cudaStream_t st = (cudaStream_t)stream;
    FS_CUDA(cudaMemcpyAsync(&code, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    FS_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
    FS_CUDA(cudaStreamSynchronize(st));
  });
  if (rc != FS_OK) return rc;
  if (code != 0) set_error("device status word reported an error");
  return code;
}

int fs_profile_start(fs_ctx* ctx) {
  return guarded([&] {
    FS_REQUIRE(ctx != nullptr, FS_ERR_ARG, "null context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (auto& r : ctx->prof) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    ctx->prof.clear();
    ctx->prof_on = true;
  });
}

int fs_profile_stop(fs_ctx* ctx, char* out, int64_t cap) {
  return guarded([&] {
    FS_REQUIRE(ctx != nullptr && out != nullptr && cap > 0, FS_ERR_ARG, "bad arguments");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->prof_on = false;
    struct Agg {
      long n = 0, k = 0;
      double ms = 0;
    };
    std::map<std::string, Agg> agg;
    for (auto& r : ctx->prof) {
      FS_CUDA(cudaEventSynchronize(r.b));
      float ms = 0;
      FS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      auto& x = agg[r.name];
      x.n += 1;
      x.k += r.kernels;
      x.ms += ms;
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    ctx->prof.clear();
    std::string js = "{";
    bool first = true;
    for (auto& kv : agg) {
      char buf[256];
      snprintf(buf, sizeof buf, "%s\"%s\": [%ld, %.6f, %ld]", first ? "" : ", ",
               kv.first.c_str(), kv.second.n, kv.second.ms, kv.second.k);
      js += buf;
      first = false;
    }
    js += "}";
    FS_REQUIRE((int64_t)js.size() < cap, FS_ERR_ARG, "profile buffer too small");
    memcpy(out, js.c_str(), js.size() + 1);
  });
}

int fs_set_rotation_path(fs_ctx* ctx, int path) {
  return guarded([&] {
    FS_REQUIRE(ctx != nullptr, FS_ERR_ARG, "null context");
    FS_REQUIRE(path >= FS_ROT_AUTO && path <= FS_ROT_MINORS, FS_ERR_ARG, "unknown rotation path");
    ctx->rot_path = path;
  });
}

int fs_set_sweep_engine(fs_ctx* ctx, int engine) {
  return guarded([&] {
    FS_REQUIRE(ctx != nullptr, FS_ERR_ARG, "null context");
    FS_REQUIRE(engine >= FS_SWEEP_AUTO && engine <= FS_SWEEP_TENSOR, FS_ERR_ARG,
               "unknown sweep engine");
    ctx->sweep_engine = engine;
  });
}

int fs_set_batch_tuning(fs_ctx* ctx, int on) {
  return guarded([&] {
    FS_REQUIRE(ctx != nullptr, FS_ERR_ARG, "null context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->batch_tuning = on ? 1 : 0;
    if (!on) {
      ctx->sweep_tune.clear();
      ctx->sweep_tune_ms.clear();
    }
  });
}

int fs_tuning_report(fs_ctx* ctx, char* out, int64_t cap) {
  return guarded([&] {
    FS_REQUIRE(ctx != nullptr && out != nullptr && cap > 0, FS_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::string js = "[";
    for (const auto& kv : ctx->sweep_tune) {
      const auto& k = kv.first;
      if (js.size() > 1) js += ",";
      js += "{\"norb\":" + std::to_string(k[0]) + ",\"n_this\":" + std::to_string(k[1]) +
            ",\"n_other\":" + std::to_string(k[2]) + ",\"dtype\":" + std::to_string(k[3]) +
            ",\"states\":" + std::to_string(k[4]) + ",\"reverse\":" + std::to_string(k[5]) +
            ",\"cross\":" + std::to_string(k[6]) + ",\"budget_kb\":" + std::to_string(k[7]) +
            ",\"vectors_per_cta\":" + std::to_string(1 << kv.second);
      // the timed widths (a zero time marks a width that was not a candidate)
      std::string w = ",\"widths\":[", t = ",\"ms\":[";
      const auto m = ctx->sweep_tune_ms.find(k);
      if (m != ctx->sweep_tune_ms.end())
        for (size_t i = 0, n = 0; i < m->second.size(); ++i) {
          if (!(m->second[i] > 0.f)) continue;
          w += (n ? "," : "") + std::to_string(1 << i);
          t += (n ? "," : "") + std::to_string(m->second[i]);
          ++n;
        }
      js += w + "]" + t + "]}";
    }
    js += "]";
    FS_REQUIRE((int64_t)js.size() < cap, FS_ERR_ARG, "report buffer too small");
    memcpy(out, js.c_str(), js.size() + 1);
  });
}

int fs_string_table(fs_ctx* ctx, int norb, int nocc, uint32_t* masks_host, int64_t dim) {
  return guarded([&] {
    FS_REQUIRE(ctx != nullptr && masks_host != nullptr, FS_ERR_ARG, "null pointer");
    FS_REQUIRE(norb >= 0 && norb <= kMaxNorb && nocc >= 0 && nocc <= norb, FS_ERR_ARG,
               "bad (norb, nocc)");
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    Space* s = get_space(ctx, norb, nocc, 0);
    FS_REQUIRE(dim == s->dim, FS_ERR_ARG, "dim must equal C(norb, nocc)");
    FS_CUDA(cudaMemcpy(masks_host, s->masks, dim * 4, cudaMemcpyDeviceToHost));
  });
}

int fs_excitation_table(fs_ctx* ctx, int norb, int nocc, uint32_t* out_host, int64_t n) {
  return guarded([&] {
    FS_REQUIRE(ctx != nullptr && out_host != nullptr, FS_ERR_ARG, "null pointer");
    FS_REQUIRE(norb >= 1 && norb <= kMaxNorb && nocc >= 0 && nocc <= norb, FS_ERR_ARG,
               "bad (norb, nocc)");
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    Space* s = get_space(ctx, norb, nocc, 0);
    FS_REQUIRE(n == s->dim * norb * norb, FS_ERR_ARG, "n_entries must be dim*norb*norb");
    uint32_t* d = (uint32_t*)scratch(ctx, "exc", n * 4);
    launch_exc_table(s, d, 0);
    FS_CUDA(cudaMemcpy(out_host, d, n * 4, cudaMemcpyDeviceToHost));
  });
}

int fs_apply_orbital_rotation(fs_ctx* ctx, void* vec, int dtype, const double* U_a,
                              const double* U_b, int norb, int na, int nb, void* stream) {
  return guarded([&] {
    check_sector(ctx, vec, dtype, norb, na, nb);
    FS_REQUIRE(U_a != nullptr, FS_ERR_ARG, "null U_a");
    std::vector<zd> Ua = load_cmat(U_a, norb);
    std::vector<zd> Ub = U_b ? load_cmat(U_b, norb) : Ua;
    check_unitary(Ua, norb, "U_a");
    if (U_b) check_unitary(Ub, norb, "U_b");
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Space* sa = get_space(ctx, norb, na, st);
    Space* sb = get_space(ctx, norb, nb, st);
    RotProgram pa = decompose_adjacent(norb, Ua.data());
    RotProgram pb = U_b ? decompose_adjacent(norb, Ub.data()) : pa;
    rotate_any(ctx, sa, sb, vec, dtype, Ua, Ub, pa, pb, st);
  });
}

int fs_apply_num_op_sum_evolution(fs_ctx* ctx, void* vec, int dtype, const double* lam_a,
                                  const double* lam_b, double t, int norb, int na, int nb,
                                  void* stream) {
  return guarded([&] {
    check_sector(ctx, vec, dtype, norb, na, nb);
    FS_REQUIRE(lam_a != nullptr, FS_ERR_ARG, "null lam_a");
    FS_REQUIRE(std::isfinite(t), FS_ERR_ARG, "t must be finite");
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Space* sa = get_space(ctx, norb, na, st);
    Space* sb = get_space(ctx, norb, nb, st);
    phase_pass(ctx, sa, sb, vec, dtype, phase_of(nullptr, nullptr, t, lam_a, norb),
               phase_of(nullptr, nullptr, t, lam_b ? lam_b : lam_a, norb), nullptr, 0, st);
  });
}

int fs_apply_diag_coulomb_evolution(fs_ctx* ctx, void* vec, int dtype, const double* J_aa,
                                    const double* J_ab, const double* J_bb, double t,
                                    int norb, int na, int nb, void* stream) {
  return guarded([&] {
    check_sector(ctx, vec, dtype, norb, na, nb);
    FS_REQUIRE(J_aa != nullptr && J_ab != nullptr, FS_ERR_ARG, "null J_aa or J_ab");
    FS_REQUIRE(std::isfinite(t), FS_ERR_ARG, "t must be finite");
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Space* sa = get_space(ctx, norb, na, st);
    Space* sb = get_space(ctx, norb, nb, st);
    // theta = -(t/2)[sum_{I_a} J_aa + sum_{I_b} J_bb + 2 sum_{p in I_a, q in I_b} J_ab]
    phase_pass(ctx, sa, sb, vec, dtype, phase_of(nullptr, J_aa, t, nullptr, norb),
               phase_of(nullptr, J_bb ? J_bb : J_aa, t, nullptr, norb), J_ab, -t, st);
  });
}

int fs_lucj_forward(fs_ctx* ctx, const fs_lucj* op, void* vec, int dtype, void* stream) {
  return guarded([&] {
    lucj_checks(ctx, op, vec, dtype);
    const int n = op->norb, R = op->n_reps;
    const size_t nn = (size_t)n * n;
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Space* sa = get_space(ctx, n, op->n_alpha, st);
    Space* sb = get_space(ctx, n, op->n_beta, st);
    if (R == 0) {
      if (op->from_hf) {
        CMat I{};
        for (int p = 0; p < n; ++p) I.v[2 * (p * n + p)] = 1.0;
        launch_slater(ctx, sa, sb, vec, dtype, I, st);
      }
      return;
    }
    auto Rs = lucj_rotations(op, nullptr);
    int k0 = 0;
    if (op->from_hf) {
      // U(R_0)|HF> is a Slater determinant: rank-1 closed form (§2.4)
      CMat Rm{};
      for (size_t q = 0; q < nn; ++q) {
        Rm.v[2 * q] = Rs[0][q].real();
        Rm.v[2 * q + 1] = Rs[0][q].imag();
      }
      launch_slater(ctx, sa, sb, vec, dtype, Rm, st);
      phase_pass(ctx, sa, sb, vec, dtype, phase_of(nullptr, op->J_aa, 1.0, nullptr, n),
                 phase_of(nullptr, op->J_aa, 1.0, nullptr, n), op->J_ab, -1.0, st);
      k0 = 1;
    }
    static const char* const kFwdT[] = {"vjp_tpsi"};
    const bool alt = k0 <= R && alternate_layouts(ctx, sa, sb, dtype, 1, kFwdT);
    void* tv = nullptr;
    if (alt) {
      const size_t S = (size_t)sa->dim * sb->dim * (dtype == FS_C64 ? 8 : 16);
      tv = scratch(ctx, "vjp_tpsi", S);
    }
    bool trans = false;
    for (int k = k0; k <= R; ++k) {
      RotProgram p = decompose_adjacent(n, Rs[k].data());
      Fused dc;
      dc.J_aa = op->J_aa + k * nn;
      dc.J_ab = op->J_ab + k * nn;
      dc.t = 1.0;
      const Fused* f = k < R ? &dc : nullptr;
      if (alt)
        rotate_alternating(ctx, sa, sb, vec, tv, trans, dtype, p, p, f, st);
      else
        rotate(ctx, sa, sb, vec, nullptr, 1, dtype, p, p, f, st);
    }
    if (trans) launch_transpose(tv, vec, sb->dim, sa->dim, dtype, st);
  });
}

// ------------------------------------------------- remaining Table 1 gates
static void spin_mask_check(int spins) {
  FS_REQUIRE(spins >= 1 && spins <= 3, FS_ERR_ARG, "spin mask must be 1 (alpha), 2 (beta) or 3");
}

static void orb_check(int p, int norb) {
  FS_REQUIRE(p >= 0 && p < norb, FS_ERR_ARG, "orbital index out of range");
}

int fs_apply_num_interaction(fs_ctx* ctx, void* vec, int dtype, double theta, int p, int spins,
                             int norb, int na, int nb, void* stream) {
  return guarded([&] {
    check_sector(ctx, vec, dtype, norb, na, nb);
    spin_mask_check(spins);
    orb_check(p, norb);
    FS_REQUIRE(std::isfinite(theta), FS_ERR_ARG, "theta must be finite");
    // exp(i theta n_p) = number-operator-sum evolution with lambda = e_p, t = -theta
    std::vector<double> la(norb, 0.0), lb(norb, 0.0);
    if (spins & 1) la[p] = 1;
    if (spins & 2) lb[p] = 1;
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Space* sa = get_space(ctx, norb, na, st);
    Space* sb = get_space(ctx, norb, nb, st);
    phase_pass(ctx, sa, sb, vec, dtype, phase_of(nullptr, nullptr, -theta, la.data(), norb),
               phase_of(nullptr, nullptr, -theta, lb.data(), norb), nullptr, 0, st);
  });
}

int fs_apply_num_num_interaction(fs_ctx* ctx, void* vec, int dtype, double theta, int p,
                                 int sigma, int q, int tau, int norb, int na, int nb,
                                 void* stream) {
  return guarded([&] {
    check_sector(ctx, vec, dtype, norb, na, nb);
    orb_check(p, norb);
    orb_check(q, norb);
    FS_REQUIRE((sigma == 0 || sigma == 1) && (tau == 0 || tau == 1), FS_ERR_ARG,
               "spins must be 0 (alpha) or 1 (beta)");
    FS_REQUIRE(std::isfinite(theta), FS_ERR_ARG, "theta must be finite");
    // diagonal-Coulomb evolution at t = -theta whose exponent is n_{p sigma} n_{q tau}
    const size_t nn = (size_t)norb * norb;
    std::vector<double> Jaa(nn, 0.0), Jab(nn, 0.0), Jbb(nn, 0.0);
    if (sigma == tau) {
      std::vector<double>& J = sigma == 0 ? Jaa : Jbb;
      if (p == q) {
        J[p * norb + p] = 2;  // -1/2 t J_pp n_p n_p with n_p^2 = n_p
      } else {
        J[p * norb + q] = 1;
        J[q * norb + p] = 1;
      }
    } else if (sigma == 0) {
      Jab[p * norb + q] = 1;  // the mixed term counts J_ab twice
    } else {
      Jab[q * norb + p] = 1;
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Space* sa = get_space(ctx, norb, na, st);
    Space* sb = get_space(ctx, norb, nb, st);
    phase_pass(ctx, sa, sb, vec, dtype, phase_of(nullptr, Jaa.data(), -theta, nullptr, norb),
               phase_of(nullptr, Jbb.data(), -theta, nullptr, norb),
               sigma == tau ? nullptr : Jab.data(), theta, st);
  });
}

// Orbital rotation by expm(K) on the spins of the mask (identity on the
// others), K the one-body generator of a Table 1 gate.
static void generator_rotation(fs_ctx* ctx, void* vec, int dtype, const std::vector<zd>& K,
                               int spins, int norb, int na, int nb, void* stream) {
  const size_t nn = (size_t)norb * norb;
  std::vector<zd> U(nn), I(nn, zd(0));
  for (int p = 0; p < norb; ++p) I[p * norb + p] = 1;
  expm(norb, K.data(), U.data());
  const std::vector<zd>& Ua = (spins & 1) ? U : I;
  const std::vector<zd>& Ub = (spins & 2) ? U : I;
  std::lock_guard<std::mutex> lk(ctx->mu);
  current_ctx() = ctx;
  FS_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  Space* sa = get_space(ctx, norb, na, st);
  Space* sb = get_space(ctx, norb, nb, st);
  RotProgram pa = decompose_adjacent(norb, Ua.data());
  RotProgram pb = decompose_adjacent(norb, Ub.data());
  rotate_any(ctx, sa, sb, vec, dtype, Ua, Ub, pa, pb, st);
}

int fs_apply_givens_rotation(fs_ctx* ctx, void* vec, int dtype, double theta, int p, int q,
                             int spins, int norb, int na, int nb, void* stream) {
  return guarded([&] {
    check_sector(ctx, vec, dtype, norb, na, nb);
    spin_mask_check(spins);
    orb_check(p, norb);
    orb_check(q, norb);
    FS_REQUIRE(p != q, FS_ERR_ARG, "a Givens rotation needs two distinct orbitals");
    FS_REQUIRE(std::isfinite(theta), FS_ERR_ARG, "theta must be finite");
    // theta (a^dag_p a_q - a^dag_q a_p) = sum K_rs a^dag_r a_s
    std::vector<zd> K((size_t)norb * norb, zd(0));
    K[p * norb + q] = theta;
    K[q * norb + p] = -theta;
    generator_rotation(ctx, vec, dtype, K, spins, norb, na, nb, stream);
  });
}

int fs_apply_tunneling_interaction(fs_ctx* ctx, void* vec, int dtype, double theta, int p,
                                   int q, int spins, int norb, int na, int nb, void* stream) {
  return guarded([&] {
    check_sector(ctx, vec, dtype, norb, na, nb);
    spin_mask_check(spins);
    orb_check(p, norb);
    orb_check(q, norb);
    FS_REQUIRE(p != q, FS_ERR_ARG, "a tunneling interaction needs two distinct orbitals");
    FS_REQUIRE(std::isfinite(theta), FS_ERR_ARG, "theta must be finite");
    // i theta (a^dag_p a_q + a^dag_q a_p) = sum K_rs a^dag_r a_s
    std::vector<zd> K((size_t)norb * norb, zd(0));
    K[p * norb + q] = zd(0, theta);
    K[q * norb + p] = zd(0, theta);
    generator_rotation(ctx, vec, dtype, K, spins, norb, na, nb, stream);
  });
}

int fs_apply_quad_ham_evolution(fs_ctx* ctx, void* vec, int dtype, const double* M_a,
                                const double* M_b, double t, int norb, int na, int nb,
                                void* stream) {
  return guarded([&] {
    check_sector(ctx, vec, dtype, norb, na, nb);
    FS_REQUIRE(M_a != nullptr, FS_ERR_ARG, "null M_a");
    FS_REQUIRE(std::isfinite(t), FS_ERR_ARG, "t must be finite");
    std::vector<zd> Ma = load_cmat(M_a, norb);
    std::vector<zd> Mb = M_b ? load_cmat(M_b, norb) : Ma;
    check_hermitian(Ma, norb, "M_a");
    if (M_b) check_hermitian(Mb, norb, "M_b");
    // exp(-i t sum M_pq a^dag_p a_q) = U(expm(-i M t)) per spin
    std::vector<zd> Ua = expm_minus_i(norb, Ma, t);
    std::vector<zd> Ub = M_b ? expm_minus_i(norb, Mb, t) : Ua;
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Space* sa = get_space(ctx, norb, na, st);
    Space* sb = get_space(ctx, norb, nb, st);
    RotProgram pa = decompose_adjacent(norb, Ua.data());
    RotProgram pb = M_b ? decompose_adjacent(norb, Ub.data()) : pa;
    rotate_any(ctx, sa, sb, vec, dtype, Ua, Ub, pa, pb, st);
  });
}

// ------------------------------------------------------ operator action
int fs_apply_molecular_hamiltonian(fs_ctx* ctx, const void* vec, void* out, int dtype,
                                   const double* one_body, const double* two_body,
                                   double constant, int64_t workspace_bytes, int norb, int na,
                                   int nb, void* stream) {
  return guarded([&] {
    check_sector(ctx, const_cast<void*>(vec), dtype, norb, na, nb);
    check_sector(ctx, out, dtype, norb, na, nb);
    FS_REQUIRE(out != vec, FS_ERR_ARG, "input and output must be distinct buffers");
    FS_REQUIRE(one_body != nullptr && two_body != nullptr, FS_ERR_ARG, "null tensor");
    FS_REQUIRE(std::isfinite(constant), FS_ERR_ARG, "constant must be finite");
    FS_REQUIRE(workspace_bytes >= 0, FS_ERR_ARG, "workspace_bytes must be >= 0");
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Space* sa = get_space(ctx, norb, na, st);
    Space* sb = get_space(ctx, norb, nb, st);
    molecular_hamiltonian(ctx, sa, sb, vec, out, dtype, one_body, two_body, constant,
                          workspace_bytes, st);
  });
}

// ------------------------------------------------------------ sampling
int fs_sample_state(fs_ctx* ctx, const void* vec, int dtype, int norb, int na, int nb,
                    const double* uniforms, int64_t shots, int64_t* out, void* stream) {
  return guarded([&] {
    check_sector(ctx, const_cast<void*>(vec), dtype, norb, na, nb);
    FS_REQUIRE(shots >= 0, FS_ERR_ARG, "shots must be >= 0");
    FS_REQUIRE(shots == 0 || (uniforms != nullptr && out != nullptr), FS_ERR_ARG,
               "null uniforms or output");
    FS_REQUIRE(((uintptr_t)uniforms & 7u) == 0 && ((uintptr_t)out & 7u) == 0, FS_ERR_ARG,
               "uniforms and output must be 8-byte aligned");
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = get_space(ctx, norb, na, st)->dim * get_space(ctx, norb, nb, st)->dim;
    sample_state(ctx, vec, dtype, n, uniforms, shots, out, st);
  });
}

int fs_sample_slater(fs_ctx* ctx, const double* U, int norb, const int* occ, int nocc,
                     const double* uniforms, int64_t shots, uint64_t* out, void* stream) {
  return guarded([&] {
    FS_REQUIRE(ctx != nullptr, FS_ERR_ARG, "null context");
    FS_REQUIRE(norb >= 1 && norb <= 1024, FS_ERR_ARG, "norb must be in [1, 1024]");
    FS_REQUIRE(nocc >= 0 && nocc <= norb, FS_ERR_ARG, "nocc must be in [0, norb]");
    FS_REQUIRE(U != nullptr && (nocc == 0 || occ != nullptr), FS_ERR_ARG,
               "null matrix or occupation list");
    FS_REQUIRE(shots >= 0, FS_ERR_ARG, "shots must be >= 0");
    FS_REQUIRE(shots == 0 || ((nocc == 0 || uniforms != nullptr) && out != nullptr), FS_ERR_ARG,
               "null uniforms or output");
    FS_REQUIRE(((uintptr_t)uniforms & 7u) == 0 && ((uintptr_t)out & 7u) == 0, FS_ERR_ARG,
               "uniforms and output must be 8-byte aligned");
    std::vector<char> seen(norb, 0);
    for (int k = 0; k < nocc; ++k) {
      FS_REQUIRE(occ[k] >= 0 && occ[k] < norb, FS_ERR_ARG, "occupied orbital out of range");
      FS_REQUIRE(!seen[occ[k]], FS_ERR_ARG, "occupied orbitals must be distinct");
      seen[occ[k]] = 1;
    }
    // Phi = U[:, occ]; its columns must be orthonormal (Phi^dag Phi = I)
    std::vector<zd> Phi((size_t)norb * (nocc > 0 ? nocc : 1));
    for (int p = 0; p < norb; ++p)
      for (int j = 0; j < nocc; ++j) {
        const size_t k = (size_t)p * norb + occ[j];
        Phi[(size_t)p * nocc + j] = zd(U[2 * k], U[2 * k + 1]);
      }
    double err = 0;
    for (int a = 0; a < nocc; ++a)
      for (int b = a; b < nocc; ++b) {
        zd g = 0;
        for (int p = 0; p < norb; ++p)
          g += std::conj(Phi[(size_t)p * nocc + a]) * Phi[(size_t)p * nocc + b];
        err = std::max(err, std::abs(g - (a == b ? 1.0 : 0.0)));
      }
    FS_REQUIRE(std::isfinite(err) && err <= 1e-10, FS_ERR_NOT_UNITARY,
               "the occupied columns of U are not orthonormal (max |Phi^dag Phi - I| = " +
                   std::to_string(err) + ")");
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    sample_slater(ctx, Phi, norb, nocc, uniforms, shots, out, (cudaStream_t)stream);
  });
}

// ------------------------------------------------------------ Trotter
static void trotter_checks(double time, int n_steps, int order) {
  FS_REQUIRE(std::isfinite(time), FS_ERR_ARG, "time must be finite");
  FS_REQUIRE(n_steps >= 1, FS_ERR_ARG, "n_steps must be >= 1");
  FS_REQUIRE(order >= 0 && order <= 6, FS_ERR_ARG, "order must be in 0 .. 6");
}

int fs_simulate_trotter_double_factorized(fs_ctx* ctx, void* vec, int dtype,
                                          const double* one_body, int n_terms,
                                          const double* diag_coulomb_mats,
                                          const double* orbital_rotations, double time,
                                          int n_steps, int order, int norb, int na, int nb,
                                          void* stream) {
  return guarded([&] {
    check_sector(ctx, vec, dtype, norb, na, nb);
    trotter_checks(time, n_steps, order);
    FS_REQUIRE(one_body != nullptr, FS_ERR_ARG, "null one-body tensor");
    FS_REQUIRE(n_terms >= 0 && (n_terms == 0 || (diag_coulomb_mats && orbital_rotations)),
               FS_ERR_ARG, "bad two-body terms");
    const size_t nn = (size_t)norb * norb;
    std::vector<zd> h = load_cmat(one_body, norb);
    check_hermitian(h, norb, "one-body tensor");
    std::vector<std::vector<zd>> U(n_terms), Ud(n_terms);
    for (int k = 0; k < n_terms; ++k) {
      U[k] = load_cmat(orbital_rotations + 2 * nn * k, norb);
      check_unitary(U[k], norb, "orbital rotation");
      Ud[k] = adjoint_of(norb, U[k]);
    }
    std::vector<GateOp> ops;
    for (const auto& f : trotter_sequence(1 + n_terms, time, n_steps, order)) {
      if (f.first == 0) {
        GateOp g;
        g.Ua = g.Ub = expm_minus_i(norb, h, f.second);
        ops.push_back(std::move(g));
      } else {
        // U(U_t) DC(J_t on every spin pair, time) U(U_t)^dag
        const int k = f.first - 1;
        const double* J = diag_coulomb_mats + nn * k;
        GateOp r0;
        r0.Ua = r0.Ub = Ud[k];
        ops.push_back(std::move(r0));
        GateOp d;
        d.kind = 1;
        d.J_aa = d.J_ab = d.J_bb = J;
        d.t = f.second;
        ops.push_back(d);
        GateOp r1;
        r1.Ua = r1.Ub = U[k];
        ops.push_back(std::move(r1));
      }
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Space* sa = get_space(ctx, norb, na, st);
    Space* sb = get_space(ctx, norb, nb, st);
    run_gates(ctx, sa, sb, vec, dtype, ops, st);
  });
}

int fs_simulate_trotter_diag_coulomb(fs_ctx* ctx, void* vec, int dtype, const double* one_body,
                                     const double* J_aa, const double* J_ab,
                                     const double* J_bb, double time, int n_steps, int order,
                                     int norb, int na, int nb, void* stream) {
  return guarded([&] {
    check_sector(ctx, vec, dtype, norb, na, nb);
    trotter_checks(time, n_steps, order);
    FS_REQUIRE(one_body != nullptr && J_aa != nullptr && J_ab != nullptr, FS_ERR_ARG,
               "null Hamiltonian array");
    std::vector<zd> h = load_cmat(one_body, norb);
    check_hermitian(h, norb, "one-body tensor");
    std::vector<GateOp> ops;
    for (const auto& f : trotter_sequence(2, time, n_steps, order)) {
      GateOp g;
      if (f.first == 0) {
        g.Ua = g.Ub = expm_minus_i(norb, h, f.second);
      } else {
        g.kind = 1;
        g.J_aa = J_aa;
        g.J_ab = J_ab;
        g.J_bb = J_bb ? J_bb : J_aa;
        g.t = f.second;
      }
      ops.push_back(std::move(g));
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Space* sa = get_space(ctx, norb, na, st);
    Space* sb = get_space(ctx, norb, nb, st);
    run_gates(ctx, sa, sb, vec, dtype, ops, st);
  });
}

}  // extern "C"

namespace fs {

// Reverse sweeps over the merged LUCJ circuit
//   psi_out = U(R_n) D_{n-1} U(R_{n-1}) ... D_0 U(R_0) psi_in.
// For m = n .. 0: undo U(R_m) on psi and g together (beta sweep, then alpha
// sweep), accumulating T^(m)_pq = <g| E_pq |psi> at the input side of U(R_m);
// the alpha sweep also writes W = Im(conj(g) psi) and undoes D_{m-1}.
// With dL = Re sum (R^-1 dR)_pq T_pq, the Euclidean gradient is R conj(T);
// the chain rule through R_m = U_m^dag U_{m-1} and K -> expm(K) is FP64 host
// work.
// The context's mapped pinned staging buffer, grown to at least `bytes`
// (growing allocates and frees pinned memory, which synchronizes the
// device; it happens on the first calls only).
static double* host_stage(Ctx* ctx, size_t bytes) {
  if (ctx->h_stage_bytes < bytes) {
    if (ctx->h_stage) FS_CUDA(cudaFreeHost(ctx->h_stage));
    ctx->h_stage = nullptr;
    ctx->h_stage_dev = nullptr;
    ctx->h_stage_bytes = 0;
    const size_t cap = std::max<size_t>(bytes, 1 << 17);
    void* h = nullptr;
    FS_CUDA(cudaHostAlloc(&h, cap, cudaHostAllocMapped));
    void* d = nullptr;
    const cudaError_t e = cudaHostGetDevicePointer(&d, h, 0);
    if (e != cudaSuccess) {
      cudaFreeHost(h);
      FS_CUDA(e);
    }
    ctx->h_stage = (double*)h;
    ctx->h_stage_dev = (double*)d;
    ctx->h_stage_bytes = cap;
  }
  return ctx->h_stage;
}

static void lucj_vjp_impl(Ctx* ctx, const fs_lucj* op, void* vec, void* cot, int dtype,
                          double* dK, double* dJ_aa, double* dJ_ab, cudaStream_t st) {
  const int n = op->norb, R = op->n_reps;
  const size_t nn = (size_t)n * n;
  Space* sa = get_space(ctx, n, op->n_alpha, st);
  Space* sb = get_space(ctx, n, op->n_beta, st);
  const size_t csz = dtype == FS_C64 ? 8 : 16;
  if (R == 0) {
    if (dK || dJ_aa || dJ_ab) FS_CUDA(cudaStreamSynchronize(st));
    return;
  }
  std::vector<std::vector<zd>> Us;
  auto Rs = lucj_rotations(op, &Us);
  double* Tacc = (double*)scratch(ctx, "vjp_T", (R + 1) * nn * 2 * sizeof(double));
  double* dJd = (double*)scratch(ctx, "vjp_dJ", 2 * R * nn * sizeof(double));
  FS_CUDA(cudaMemsetAsync(Tacc, 0, (R + 1) * nn * 2 * sizeof(double), st));
  FS_CUDA(cudaMemsetAsync(dJd, 0, 2 * R * nn * sizeof(double), st));
  double* dJaa_d = dJd;
  double* dJab_d = dJd + R * nn;
  // Reverse alpha sweeps on a state larger than L2 run on transposed copies
  // of psi and g (alpha strings along rows, so every slab is contiguous)
  // when memory allows two more states; their W comes out transposed and
  // their dJ_ab transposed, accumulated apart and transposed on the host.
  const size_t S = (size_t)sa->dim * sb->dim * csz;
  bool alpha_t = S > (size_t)ctx->prop.l2CacheSize;
  if (alpha_t) {
    size_t fr = 0, tot = 0;
    const bool have = ctx->scratch["vjp_tpsi"].bytes >= S && ctx->scratch["vjp_tg"].bytes >= S;
    if (!have && cudaMemGetInfo(&fr, &tot) == cudaSuccess) alpha_t = fr > 2 * S + (1ull << 30);
  }
  double* dJabT_d = nullptr;
  void *tpsi = nullptr, *tg = nullptr;
  if (alpha_t) {
    tpsi = scratch(ctx, "vjp_tpsi", S);
    tg = scratch(ctx, "vjp_tg", S);
    dJabT_d = (double*)scratch(ctx, "vjp_dJabT", R * nn * sizeof(double));
    FS_CUDA(cudaMemsetAsync(dJabT_d, 0, R * nn * sizeof(double), st));
  }
  void* Wb = scratch(ctx, "vjp_W", sa->dim * sb->dim * (csz / 2));
  void* ea_a = scratch(ctx, "ea_a", sa->dim * csz);
  void* ea_b = scratch(ctx, "ea_b", sb->dim * csz);
  void* e2_a = scratch(ctx, "ea2_a", sa->dim * csz);
  void* e2_b = scratch(ctx, "ea2_b", sb->dim * csz);
  std::vector<zd> adj(nn);
  // With transposed copies the layers alternate: from (vec, cot) the beta
  // undo runs on rows of the states, then both are transposed and the alpha
  // undo runs on rows of the copies, carrying W and D_{m-1}^dag; the next
  // layer starts from the copies with the alpha undo, transposes back, and
  // the beta undo carries W and D^dag.  The spin parts of a rotation commute
  // and T^alpha (T^beta) is unchanged by the beta (alpha) rotation, so the
  // order is free; each layer costs two transposes.
  bool trans = false;
  for (int m = R; m >= 0; --m) {
    mat_adjoint(n, Rs[m].data(), adj.data());
    RotProgram inv = decompose_adjacent(n, adj.data());
    double* Tm = Tacc + (size_t)m * nn * 2;
    const double* Ja = m >= 1 ? op->J_aa + (size_t)(m - 1) * nn : nullptr;
    const double* Jab = m >= 1 ? op->J_ab + (size_t)(m - 1) * nn : nullptr;
    if (m >= 1) {
      launch_string_phase(sa, e2_a, dtype, phase_of(nullptr, Ja, -1.0, nullptr, n), st);
      launch_string_phase(sb, e2_b, dtype, phase_of(nullptr, Ja, -1.0, nullptr, n), st);
    }
    launch_string_phase(sb, ea_b, dtype, phase_of(&inv, nullptr, 0, nullptr, n), st);
    launch_string_phase(sa, ea_a, dtype, phase_of(&inv, nullptr, 0, nullptr, n), st);
    if (alpha_t && trans) {
      // alpha: undo on rows of the copies, T^alpha
      PhaseDev q1;
      q1.ea_b = ea_a;
      RevArgs t1;
      t1.T = Tm;
      launch_sweep(ctx, sb, sa, 1, tpsi, tg, 2, dtype, inv, q1, st, &t1);
      launch_transpose(tpsi, vec, sb->dim, sa->dim, dtype, st);
      launch_transpose(tg, cot, sb->dim, sa->dim, dtype, st);
      // beta: undo, T^beta, W and D_{m-1}^dag
      PhaseDev p2;
      p2.ea_b = ea_b;
      RevArgs r2;
      r2.T = Tm;
      if (m >= 1) {
        r2.ea2_a = e2_a;
        r2.ea2_b = e2_b;
        r2.W = Wb;
        p2.has_x = 1;
        p2.X = real_mat(Jab, n, 1.0);
      }
      launch_sweep(ctx, sa, sb, 1, vec, cot, 2, dtype, inv, p2, st, &r2);
      if (m >= 1)
        launch_dc_grad(ctx, sa, sb, Wb, dtype, dJaa_d + (size_t)(m - 1) * nn,
                       dJab_d + (size_t)(m - 1) * nn, st);
      trans = false;
      continue;
    }
    // beta: undo, T^beta
    PhaseDev p1;
    p1.ea_b = ea_b;
    RevArgs r1;
    r1.T = Tm;
    launch_sweep(ctx, sa, sb, 1, vec, cot, 2, dtype, inv, p1, st, &r1);
    // alpha: undo, T^alpha, W and D_{m-1}^dag
    if (alpha_t) {
      // the same sweep as a row sweep of the transposed states: this spin
      // (alpha) along rows of length dim_a, the cross angles transposed
      launch_transpose(vec, tpsi, sa->dim, sb->dim, dtype, st);
      launch_transpose(cot, tg, sa->dim, sb->dim, dtype, st);
      PhaseDev q2;
      q2.ea_b = ea_a;
      RevArgs t2;
      t2.T = Tm;
      if (m >= 1) {
        t2.ea2_b = e2_a;
        t2.ea2_a = e2_b;
        t2.W = Wb;
        q2.has_x = 1;
        for (int p = 0; p < n; ++p)
          for (int q = 0; q < n; ++q) q2.X.v[q * n + p] = Jab[p * n + q];
      }
      launch_sweep(ctx, sb, sa, 1, tpsi, tg, 2, dtype, inv, q2, st, &t2);
      if (m >= 1)
        launch_dc_grad(ctx, sb, sa, Wb, dtype, dJaa_d + (size_t)(m - 1) * nn,
                       dJabT_d + (size_t)(m - 1) * nn, st);
      trans = true;
    } else {
      PhaseDev p2;
      p2.ea_a = ea_a;
      RevArgs r2;
      r2.T = Tm;
      if (m >= 1) {
        r2.ea2_a = e2_a;
        r2.ea2_b = e2_b;
        r2.W = Wb;
        p2.has_x = 1;
        p2.X = real_mat(Jab, n, 1.0);
      }
      launch_sweep(ctx, sa, sb, 0, vec, cot, 2, dtype, inv, p2, st, &r2);
      if (m >= 1)
        launch_dc_grad(ctx, sa, sb, Wb, dtype, dJaa_d + (size_t)(m - 1) * nn,
                       dJab_d + (size_t)(m - 1) * nn, st);
    }
  }
  if (trans) {
    launch_transpose(tpsi, vec, sb->dim, sa->dim, dtype, st);
    launch_transpose(tg, cot, sb->dim, sa->dim, dtype, st);
  }
  std::vector<double> Th((R + 1) * nn * 2), dJh(2 * R * nn), dJT(alpha_t ? R * nn : 0);
  {
    // one small kernel writes the three results into the mapped host buffer
    const size_t ntot = Th.size() + dJh.size() + dJT.size();
    double* hs = host_stage(ctx, ntot * sizeof(double));
    launch_gather_f64(Tacc, (int64_t)Th.size(), dJd, (int64_t)dJh.size(),
                      alpha_t ? dJabT_d : nullptr, (int64_t)dJT.size(), ctx->h_stage_dev, st);
    FS_CUDA(cudaStreamSynchronize(st));
    std::copy(hs, hs + Th.size(), Th.begin());
    std::copy(hs + Th.size(), hs + Th.size() + dJh.size(), dJh.begin());
    std::copy(hs + Th.size() + dJh.size(), hs + ntot, dJT.begin());
  }
  if (alpha_t)
    for (int k = 0; k < R; ++k)
      for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
          dJh[R * nn + k * nn + p * n + q] += dJT[k * nn + q * n + p];
  if (dJ_aa) std::copy(dJh.begin(), dJh.begin() + R * nn, dJ_aa);
  if (dJ_ab) std::copy(dJh.begin() + R * nn, dJh.end(), dJ_ab);
  if (!dK) return;
  std::vector<std::vector<zd>> gU(R, std::vector<zd>(nn, zd(0)));
  std::vector<zd> gR(nn), cT(nn), tmp(nn), tmp2(nn);
  for (int m = 0; m <= R; ++m) {
    for (size_t q = 0; q < nn; ++q)
      cT[q] = zd(Th[2 * (m * nn + q)], -Th[2 * (m * nn + q) + 1]);
    mat_mul(n, Rs[m].data(), cT.data(), gR.data());  // R conj(T)
    if (m == 0) {
      mat_adjoint(n, gR.data(), tmp.data());
      for (size_t q = 0; q < nn; ++q) gU[0][q] += tmp[q];
    }
    if (m == R) {
      for (size_t q = 0; q < nn; ++q) gU[R - 1][q] += gR[q];
    }
    if (m >= 1 && m <= R - 1) {
      mat_mul(n, Us[m].data(), gR.data(), tmp.data());
      for (size_t q = 0; q < nn; ++q) gU[m - 1][q] += tmp[q];
      mat_adjoint(n, gR.data(), tmp2.data());
      mat_mul(n, Us[m - 1].data(), tmp2.data(), tmp.data());
      for (size_t q = 0; q < nn; ++q) gU[m][q] += tmp[q];
    }
  }
  for (int k = 0; k < R; ++k) {
    std::vector<zd> K = load_cmat(op->K + 2 * nn * k, n), out(nn);
    expm_frechet_adjoint(n, K.data(), gU[k].data(), out.data());
    for (size_t q = 0; q < nn; ++q) {
      dK[2 * (k * nn + q)] = out[q].real();
      dK[2 * (k * nn + q) + 1] = out[q].imag();
    }
  }
}

}  // namespace fs

extern "C" int fs_lucj_vjp(fs_ctx* ctx, const fs_lucj* op, void* vec, void* cot, int dtype,
                           double* dK, double* dJ_aa, double* dJ_ab, void* stream) {
  return guarded([&] {
    lucj_checks(ctx, op, vec, dtype);
    FS_REQUIRE(cot != nullptr && ((uintptr_t)cot & 15u) == 0, FS_ERR_ARG,
               "cotangent pointer must be non-null and 16-byte aligned");
    FS_REQUIRE(cot != vec, FS_ERR_ARG, "state and cotangent must be distinct buffers");
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    lucj_vjp_impl(ctx, op, vec, cot, dtype, dK, dJ_aa, dJ_ab, (cudaStream_t)stream);
  });
}

extern "C" int fs_lucj_batch(fs_ctx* ctx, int n_circuits, const fs_lucj* ops, void* const* vecs,
                             void* const* cots, int dtype, int do_vjp, double* const* dK,
                             double* const* dJ_aa, double* const* dJ_ab, void* stream) {
  return guarded([&] {
    FS_REQUIRE(ctx != nullptr && ops != nullptr && vecs != nullptr, FS_ERR_ARG, "null argument");
    FS_REQUIRE(n_circuits >= 1, FS_ERR_ARG, "n_circuits must be >= 1");
    FS_REQUIRE(dtype == FS_C64 || dtype == FS_C128, FS_ERR_ARG, "dtype must be FS_C64 or FS_C128");
    FS_REQUIRE(!do_vjp || cots != nullptr, FS_ERR_ARG, "null cotangent array");
    for (int c = 0; c < n_circuits; ++c) {
      const fs_lucj* op = &ops[c];
      FS_REQUIRE(op->norb >= 1 && op->norb <= kMaxNorb && op->n_alpha >= 0 &&
                     op->n_alpha <= op->norb && op->n_beta >= 0 && op->n_beta <= op->norb &&
                     op->n_reps >= 0 && (op->n_reps == 0 || (op->K && op->J_aa && op->J_ab)),
                 FS_ERR_ARG, "bad circuit description");
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    current_ctx() = ctx;
    FS_CUDA(cudaSetDevice(ctx->device));
    lucj_batch(ctx, n_circuits, ops, vecs, cots, dtype, do_vjp, dK, dJ_aa, dJ_ab,
               (cudaStream_t)stream);
  });
}
