// Batched LUCJ forward + VJP over many independent circuits with uneven
// sectors (§4.3, §4.5.1 per circuit).
//
// Every stage of the circuit (per-string phase tables, one sweep, one
// reduction) runs once for all circuits: the sweeps as one persistent launch
// over a work queue of (circuit, slab) items, largest circuits first; the
// small kernels over flattened (circuit, element) ranges.  The whole stage
// sequence is captured into one CUDA graph and launched once.  All small
// per-circuit data (Givens programs, phase recipes, coupling matrices) is
// prepared on the host and uploaded in one copy before the capture.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

// ------------------------------------------------------- batched kernels
template <typename Job>
__device__ __forceinline__ int find_job(const Job* jobs, int njobs, int64_t it) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].item0 <= it) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Per-string factors (see launch_string_phase), one recipe per job.
struct BStr {
  const uint32_t* masks;
  void* out;
  const double* J;  // device, norb x norb, or null
  int64_t item0;
  int norb, use_d;
  double t;
  double d[2 * kMaxOrb];
};

template <typename R>
__global__ void k_string_phase_batch(const BStr* jobs, int njobs, int64_t total) {
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total;
       it += (int64_t)gridDim.x * blockDim.x) {
    const BStr& J = jobs[find_job(jobs, njobs, it)];
    const int64_t e = it - J.item0;
    const uint32_t m = J.masks[e];
    double re = 1, im = 0, ang = 0;
    for (int p = 0; p < J.norb; ++p) {
      if (!((m >> p) & 1u)) continue;
      if (J.use_d) {
        const double dr = J.d[2 * p], di = J.d[2 * p + 1];
        const double nr = re * dr - im * di;
        im = re * di + im * dr;
        re = nr;
      }
      if (J.J)
        for (int q = 0; q < J.norb; ++q)
          if ((m >> q) & 1u) ang -= 0.5 * J.t * J.J[p * J.norb + q];
    }
    const double r = ang - 6.283185307179586 * rint(ang * 0.15915494309189535);
    double s, c;
    sincos(r, &s, &c);
    reinterpret_cast<cx_t<R>*>(J.out)[e] = mk<R>((R)(re * c - im * s), (R)(re * s + im * c));
  }
}

// Hartree-Fock initial states: psi = e_0.
struct BVec {
  void* vec;
  int64_t item0;
};
template <typename R>
__global__ void k_hf_batch(const BVec* jobs, int njobs, int64_t total) {
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total;
       it += (int64_t)gridDim.x * blockDim.x) {
    const BVec& J = jobs[find_job(jobs, njobs, it)];
    const int64_t e = it - J.item0;
    reinterpret_cast<cx_t<R>*>(J.vec)[e] = mk<R>(e == 0 ? R(1) : R(0), R(0));
  }
}

// Slater start of a circuit from Hartree-Fock (§2.4): the first merged
// rotation R_0 maps HF to a Slater determinant, psi = a b^T with
// a[I] = det(R_0[I, {0..n_a-1}]) (likewise b); one job per (circuit, spin).
struct BSl {
  const uint32_t* masks;
  double2* out;
  const CMat* R;  // device
  int64_t item0;
  int norb, n;
};
__global__ void k_slater_batch(const BSl* jobs, int njobs, int64_t total) {
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total;
       it += (int64_t)gridDim.x * blockDim.x) {
    const BSl& J = jobs[find_job(jobs, njobs, it)];
    const int64_t e = it - J.item0;
    J.out[e] = slater_minor(J.masks[e], J.norb, J.n, J.R->v);
  }
}

// psi = a b^T followed by the first diagonal-Coulomb gate: one CTA per
// (circuit, alpha row); the row's cross angles w[q] = sum_{p in I_a} X[p][q]
// become 8-bit subset tables, the same-spin parts arrive as string factors.
struct BSd {
  void* vec;
  const double2* va;
  const double2* vb;
  const void* ea_a;
  const void* ea_b;
  const Mat* X;  // device: -J_ab of the first gate
  const uint32_t* ma;
  const uint32_t* mb;
  int64_t db;
  int norb;
  int64_t item0;  // alpha rows
};
template <typename R>
__global__ void __launch_bounds__(256) k_slater_dc_batch(const BSd* jobs, int njobs,
                                                         int64_t total) {
  using C = cx_t<R>;
  __shared__ double w[32];
  __shared__ C tab[4 * 256];
  for (int64_t it = blockIdx.x; it < total; it += gridDim.x) {
    const BSd& J = jobs[find_job(jobs, njobs, it)];
    const int64_t i = it - J.item0;
    const uint32_t mi = J.ma[i];
    const int N = J.norb, nch = (N + 7) / 8;
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
      double sum = 0;
      for (uint32_t m = mi; m; m &= m - 1) sum += J.X->v[(__ffs(m) - 1) * N + q];
      w[q] = sum;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nch * 256; idx += blockDim.x) {
      const int c = idx >> 8;
      double sum = 0;
      for (int v = idx & 255; v; v &= v - 1) {
        const int x = 8 * c + __ffs(v) - 1;
        if (x < N) sum += w[x];
      }
      tab[idx] = expi<R>(sum);
    }
    __syncthreads();
    const double2 a = J.va[i];
    const C ea = reinterpret_cast<const C*>(J.ea_a)[i];
    C* row = reinterpret_cast<C*>(J.vec) + i * J.db;
    for (int64_t j = threadIdx.x; j < J.db; j += blockDim.x) {
      const double2 b = J.vb[j];
      C f = mk<R>((R)(a.x * b.x - a.y * b.y), (R)(a.x * b.y + a.y * b.x));
      f = cmul<R>(f, cmul<R>(ea, reinterpret_cast<const C*>(J.ea_b)[j]));
      const uint32_t m = __ldg(J.mb + j);
      for (int c = 0; c < nch; ++c) f = cmul<R>(f, tab[c * 256 + ((m >> (8 * c)) & 255)]);
      row[j] = f;
    }
    __syncthreads();
  }
}

// Gradient of one diagonal-Coulomb gate per job from W (as fs_reduce.cu):
// rows give Occ_a^T W Occ_b and the alpha part of dJ_aa, columns the beta
// part.
struct BDc {
  const void* W;
  const uint32_t* ma;
  const uint32_t* mb;
  double* dJaa;
  double* dJab;
  double* c;  // column sums, dim_b
  int64_t da, db;
  int norb;
  int64_t item0;  // rows, columns or (p, q) items, per kernel
};

// Rows in contiguous chunks per CTA; partial sums per CTA in shared memory,
// flushed to the job's accumulators when the job changes and at the end.
template <typename R>
__global__ void __launch_bounds__(128)
    k_dc_rows_batch(const BDc* jobs, int njobs, int64_t total) {
  __shared__ double red[4][kMaxOrb + 1];
  __shared__ double sab[kMaxOrb * kMaxOrb], saa[kMaxOrb * kMaxOrb];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * per, b1 = min(total, b0 + per);
  int cur = -1;
  for (int k = threadIdx.x; k < kMaxOrb * kMaxOrb; k += 128) sab[k] = saa[k] = 0;
  __syncthreads();
  for (int64_t it = b0; it < b1; ++it) {
    const int jb = find_job(jobs, njobs, it);
    if (jb != cur) {
      if (cur >= 0) {
        const BDc& P = jobs[cur];
        for (int k = threadIdx.x; k < P.norb * P.norb; k += 128) {
          if (sab[k] != 0) atomicAdd(P.dJab + k, sab[k]);
          if (saa[k] != 0) atomicAdd(P.dJaa + k, saa[k]);
          sab[k] = saa[k] = 0;
        }
        __syncthreads();
      }
      cur = jb;
    }
    const BDc& J = jobs[jb];
    const int64_t i = it - J.item0;
    const R* row = reinterpret_cast<const R*>(J.W) + i * J.db;
    R acc[kMaxOrb + 1];
#pragma unroll
    for (int q = 0; q <= kMaxOrb; ++q) acc[q] = 0;
    for (int64_t j = threadIdx.x; j < J.db; j += 128) {
      const R w = row[j];
      const uint32_t m = __ldg(J.mb + j);
      acc[kMaxOrb] += w;
#pragma unroll
      for (int q = 0; q < kMaxOrb; ++q) acc[q] += ((m >> q) & 1u) ? w : R(0);
    }
#pragma unroll
    for (int q = 0; q <= kMaxOrb; ++q) {
      double v = (double)acc[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
      if (lane == 0) red[wid][q] = v;
    }
    __syncthreads();
    const uint32_t mi = J.ma[i];
    const double ri = red[0][kMaxOrb] + red[1][kMaxOrb] + red[2][kMaxOrb] + red[3][kMaxOrb];
    for (int k = threadIdx.x; k < J.norb * J.norb; k += 128) {
      const int p = k / J.norb, q = k - p * J.norb;
      if (!((mi >> p) & 1u)) continue;
      sab[k] += red[0][q] + red[1][q] + red[2][q] + red[3][q];
      if ((mi >> q) & 1u) saa[k] += 0.5 * ri;
    }
    __syncthreads();
  }
  if (cur >= 0) {
    const BDc& P = jobs[cur];
    for (int k = threadIdx.x; k < P.norb * P.norb; k += 128) {
      if (sab[k] != 0) atomicAdd(P.dJab + k, sab[k]);
      if (saa[k] != 0) atomicAdd(P.dJaa + k, saa[k]);
    }
  }
}

template <typename R>
__global__ void k_dc_cols_batch(const BDc* jobs, int njobs, int64_t total) {
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total;
       it += (int64_t)gridDim.x * blockDim.x) {
    const BDc& J = jobs[find_job(jobs, njobs, it)];
    const int64_t j = it - J.item0;
    const R* w = reinterpret_cast<const R*>(J.W) + j;
    double s = 0;
    for (int64_t i = 0; i < J.da; ++i) s += (double)w[i * J.db];
    J.c[j] = s;
  }
}

__global__ void __launch_bounds__(128)
    k_dc_beta_aa_batch(const BDc* jobs, int njobs, int64_t total) {
  __shared__ double red[4];
  for (int64_t it = blockIdx.x; it < total; it += gridDim.x) {
    const BDc& J = jobs[find_job(jobs, njobs, it)];
    const int k = (int)(it - J.item0), p = k / J.norb, q = k - p * J.norb;
    const uint32_t want = (1u << p) | (1u << q);
    double s = 0;
    for (int64_t j = threadIdx.x; j < J.db; j += 128)
      if ((__ldg(J.mb + j) & want) == want) s += J.c[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) J.dJaa[k] += 0.5 * (red[0] + red[1] + red[2] + red[3]);
    __syncthreads();
  }
}

// ------------------------------------------------------------ host side
namespace {

// A growing byte image of device-side parameters, uploaded in one copy.
struct Image {
  std::vector<unsigned char> bytes;
  size_t add(const void* p, size_t n, size_t align = 256) {
    size_t o = (bytes.size() + align - 1) / align * align;
    bytes.resize(o + n);
    if (p) memcpy(bytes.data() + o, p, n);
    return o;
  }
};

struct Circuit {
  int idx;
  const fs_lucj* op;
  Space* sa;
  Space* sb;
  std::vector<std::vector<zd>> Us, Rs;
  std::vector<RotProgram> fwd, rev;
  // device pointers (scratch arena)
  void *ea_a, *ea_b, *ea_o, *e2_a, *e2_b, *W;
  double *T, *dJ, *colsum;
  double2 *sl_a, *sl_b;     // Slater start vectors (from Hartree-Fock only)
  size_t jaa_off, xab_off;  // image offsets: J_aa (R x N x N), X mats (2R Mat)
  size_t r0_off;            // image offset of R_0 (CMat, from Hartree-Fock only)
  bool hf() const { return op->from_hf != 0; }
};

// A stage: kernel launches recorded into the graph.
struct Stage {
  int kind;  // 0 string phases, 1 sweep, 2 hf init, 3 dc gradient, 4 Slater
             // minors, 5 Slater product + first diagonal-Coulomb gate
  int nst = 1;
  size_t jobs_off = 0;
  int njobs = 0;
  int64_t total = 0, total2 = 0, total3 = 0;
  size_t smem = 0;
  int counter = -1;
  bool pk = false;
};

}  // namespace

static void lucj_batch_impl(Ctx* ctx, int n, const fs_lucj* ops, void* const* vecs,
                            void* const* cots, int dtype, int do_vjp, double* const* dK,
                            double* const* dJaa, double* const* dJab, cudaStream_t st) {
  const size_t csz = dtype == FS_C64 ? 8 : 16;
  const int R = ops[0].n_reps;
  // ---- circuits, largest first (work-queue order)
  std::vector<Circuit> cs(n);
  for (int c = 0; c < n; ++c) {
    const fs_lucj* op = &ops[c];
    FS_REQUIRE(op->n_reps == R, FS_ERR_ARG, "all circuits of a batch need the same n_reps");
    FS_REQUIRE(op->norb >= 6 && op->norb <= 32, FS_ERR_UNSUPPORTED,
               "batched circuits need 6 <= norb <= 32");
    FS_REQUIRE(vecs[c] && ((uintptr_t)vecs[c] & 15u) == 0, FS_ERR_ARG, "bad state pointer");
    FS_REQUIRE(!do_vjp || (cots[c] && ((uintptr_t)cots[c] & 15u) == 0 && cots[c] != vecs[c]),
               FS_ERR_ARG, "bad cotangent pointer");
    Circuit& C = cs[c];
    C.idx = c;
    C.op = op;
    C.sa = get_space(ctx, op->norb, op->n_alpha, st);
    C.sb = get_space(ctx, op->norb, op->n_beta, st);
    FS_REQUIRE(C.sa->dim >= 2 && C.sb->dim >= 2, FS_ERR_UNSUPPORTED,
               "batched circuits need at least two strings per spin");
  }
  std::stable_sort(cs.begin(), cs.end(), [](const Circuit& a, const Circuit& b) {
    return a.sa->dim * a.sb->dim > b.sa->dim * b.sb->dim;
  });
  // ---- host FP64 work: merged rotations and their Givens programs
  for (auto& C : cs) {
    if (R == 0) continue;
    const fs_lucj* op = C.op;
    const int N = op->norb;
    C.Rs = std::vector<std::vector<zd>>();
    {
      // R_0 = U_0^dag, R_k = U_k^dag U_{k-1}, R_n = U_{n-1}
      const size_t nn = (size_t)N * N;
      std::vector<std::vector<zd>> Us(R), Rs(R + 1, std::vector<zd>(nn));
      for (int k = 0; k < R; ++k) {
        std::vector<zd> K(nn);
        for (size_t q = 0; q < nn; ++q) K[q] = zd(op->K[2 * (k * nn + q)], op->K[2 * (k * nn + q) + 1]);
        Us[k].resize(nn);
        expm(N, K.data(), Us[k].data());
      }
      std::vector<zd> adj(nn);
      mat_adjoint(N, Us[0].data(), Rs[0].data());
      for (int k = 1; k < R; ++k) {
        mat_adjoint(N, Us[k].data(), adj.data());
        mat_mul(N, adj.data(), Us[k - 1].data(), Rs[k].data());
      }
      Rs[R] = Us[R - 1];
      C.Us = Us;
      C.Rs = Rs;
    }
    std::vector<zd> adj((size_t)N * N);
    for (int k = 0; k <= R; ++k) {
      C.fwd.push_back(decompose_adjacent(N, C.Rs[k].data()));
      mat_adjoint(N, C.Rs[k].data(), adj.data());
      C.rev.push_back(decompose_adjacent(N, adj.data()));
    }
  }
  // ---- device scratch arena
  size_t arena = 0;
  auto take = [&](size_t bytes) {
    size_t o = (arena + 255) / 256 * 256;
    arena = o + bytes;
    return o;
  };
  std::vector<size_t> o_ea(n), o_w(n), o_t(n), o_dj(n), o_cs(n), o_sl(n);
  for (int c = 0; c < n; ++c) {
    const Circuit& C = cs[c];
    const int N = C.op->norb;
    const size_t dmax = std::max(C.sa->dim, C.sb->dim);
    o_ea[c] = take(5 * dmax * csz);
    o_sl[c] = C.hf() && R > 0 ? take((C.sa->dim + C.sb->dim) * sizeof(double2)) : 0;
    o_w[c] = do_vjp && R > 0 ? take(C.sa->dim * C.sb->dim * csz / 2) : 0;
    o_t[c] = take((size_t)(R + 1) * N * N * 2 * sizeof(double));
    o_dj[c] = take((size_t)2 * std::max(R, 1) * N * N * sizeof(double));
    o_cs[c] = take(C.sb->dim * sizeof(double));
  }
  const size_t acc_begin = std::min(o_t.empty() ? arena : o_t[0], arena);
  unsigned char* base = (unsigned char*)scratch(ctx, "batch_arena", std::max<size_t>(arena, 256));
  for (int c = 0; c < n; ++c) {
    Circuit& C = cs[c];
    const size_t dmax = std::max(C.sa->dim, C.sb->dim);
    C.ea_a = base + o_ea[c];
    C.ea_b = base + o_ea[c] + dmax * csz;
    C.ea_o = base + o_ea[c] + 2 * dmax * csz;
    C.e2_a = base + o_ea[c] + 3 * dmax * csz;
    C.e2_b = base + o_ea[c] + 4 * dmax * csz;
    C.W = do_vjp && R > 0 ? base + o_w[c] : nullptr;
    C.T = (double*)(base + o_t[c]);
    C.dJ = (double*)(base + o_dj[c]);
    C.colsum = (double*)(base + o_cs[c]);
    C.sl_a = C.hf() && R > 0 ? (double2*)(base + o_sl[c]) : nullptr;
    C.sl_b = C.hf() && R > 0 ? C.sl_a + C.sa->dim : nullptr;
  }
  // ---- parameter image: J_aa arrays, X matrices, programs, jobs
  Image img;
  for (auto& C : cs) {
    const int N = C.op->norb;
    const size_t nn = (size_t)N * N;
    C.jaa_off = img.add(C.op->J_aa, std::max<size_t>(R, 1) * nn * sizeof(double) * (R > 0));
    std::vector<Mat> X(2 * std::max(R, 1));
    for (int k = 0; k < R; ++k)
      for (size_t q = 0; q < nn; ++q) {
        X[k].v[q] = -C.op->J_ab[k * nn + q];     // forward D_k
        X[R + k].v[q] = C.op->J_ab[k * nn + q];  // reverse D_k^dag
      }
    C.xab_off = img.add(X.data(), X.size() * sizeof(Mat));
    C.r0_off = 0;
    if (C.hf() && R > 0) {
      CMat R0{};
      for (size_t q = 0; q < nn; ++q) {
        R0.v[2 * q] = C.Rs[0][q].real();
        R0.v[2 * q + 1] = C.Rs[0][q].imag();
      }
      C.r0_off = img.add(&R0, sizeof(CMat));
    }
  }
  const size_t maxsm = (size_t)ctx->prop.sharedMemPerBlockOptin;
  const size_t half_sm = (size_t)ctx->prop.sharedMemPerMultiprocessor / 2 - 1024;
  std::vector<Stage> stages;
  int ncounters = 0;
  unsigned char* dimg = nullptr;  // set after the image is complete
  // string-phase stage: recipes (masks, out, J, use_d with program phase)
  auto phase_stage = [&](auto&& recipe) {
    std::vector<BStr> js;
    int64_t tot = 0;
    for (auto& C : cs) {
      std::vector<BStr> r = recipe(C);
      for (auto& b : r) {
        b.item0 = tot;
        tot += (b.masks == C.sa->masks) ? C.sa->dim : C.sb->dim;
        js.push_back(b);
      }
    }
    Stage S;
    S.kind = 0;
    S.njobs = (int)js.size();
    S.total = tot;
    S.jobs_off = img.add(js.data(), js.size() * sizeof(BStr));
    stages.push_back(S);
  };
  auto recipe_of = [&](const Space* sp, void* out, const RotProgram* rp, size_t jaa_off, bool use_j,
                       int k, double t, int N) {
    BStr b{};
    b.masks = sp->masks;
    b.out = out;
    b.norb = N;
    b.t = t;
    if (rp) {
      b.use_d = 1;
      for (int p = 0; p < N; ++p) {
        b.d[2 * p] = rp->phase[p].real();
        b.d[2 * p + 1] = rp->phase[p].imag();
      }
    }
    // J pointer patched after upload: store the image offset for now
    b.J = use_j ? (const double*)(uintptr_t)(jaa_off + (size_t)k * N * N * sizeof(double) + 1) : nullptr;
    return b;
  };
  // sweep stage: one job per circuit
  struct PendingSweep {
    size_t stage;
    std::vector<SweepJob> jobs;
    std::vector<size_t> prog_off, x_off;
  };
  std::vector<PendingSweep> pend;
  auto sweep_stage = [&](int dir, int nst, auto&& use, auto&& setup) {
    PendingSweep P;
    P.stage = stages.size();
    Stage S;
    S.kind = 1;
    S.nst = nst;
    int64_t items = 0;
    size_t smem = 0;
    bool pk = true;
    const size_t budget = nst == 1 ? half_sm : maxsm;
    for (auto& C : cs) {
      if (!use(C)) continue;
      PhaseDev ph;
      RevArgs rv;
      const RotProgram* rp = nullptr;
      long xk = -1;
      bool has_rev = false;
      setup(C, ph, rv, rp, xk, has_rev);
      BatchSweepPlan plan;
      plan_batch_sweep(ctx, C.sa, C.sb, dir, C.op ? vecs[C.idx] : nullptr,
                       nst == 2 ? cots[C.idx] : nullptr, nst, dtype, *rp, ph,
                       has_rev ? &rv : nullptr, budget, plan);
      SweepJob j{};
      j.g = plan.g;
      j.item0 = (int)items;
      items += plan.nslabs;
      smem = std::max(smem, plan.smem);
      pk = pk && plan.pk;
      P.jobs.push_back(j);
      P.prog_off.push_back(img.add(plan.prog.data(), plan.prog.size()));
      P.x_off.push_back(xk >= 0 ? C.xab_off + (size_t)xk * sizeof(Mat) : (size_t)-1);
    }
    if (P.jobs.empty()) return;
    S.counter = ncounters++;
    S.njobs = (int)P.jobs.size();
    S.total = items;
    S.smem = smem;
    S.pk = pk;
    stages.push_back(S);
    pend.push_back(std::move(P));
  };
  auto all = [](const Circuit&) { return true; };
  Mat zero{};
  const size_t zero_off = img.add(&zero, sizeof(Mat));

  // ---------------- forward
  {
    std::vector<BVec> hv;
    int64_t tot = 0;
    for (auto& C : cs)
      if (C.hf() && R == 0) {  // with rotations the Slater start writes the state
        hv.push_back(BVec{vecs[C.idx], tot});
        tot += C.sa->dim * C.sb->dim;
      }
    if (!hv.empty()) {
      Stage S;
      S.kind = 2;
      S.njobs = (int)hv.size();
      S.total = tot;
      S.jobs_off = img.add(hv.data(), hv.size() * sizeof(BVec));
      stages.push_back(S);
    }
  }
  bool any_hf = false;
  for (auto& C : cs) any_hf = any_hf || C.hf();
  auto sweeps_k = [&](int k) {
    // circuits from Hartree-Fock replace the first rotation (and gate) by
    // the Slater start
    return [k](const Circuit& C) { return k > 0 || !C.hf(); };
  };
  for (int k = 0; k <= R && R > 0; ++k) {
    phase_stage([&](Circuit& C) {
      const int N = C.op->norb;
      std::vector<BStr> r;
      if (k == 0 && C.hf()) {  // same-spin parts of the first gate
        r.push_back(recipe_of(C.sa, C.ea_a, nullptr, C.jaa_off, true, 0, 1.0, N));
        r.push_back(recipe_of(C.sb, C.ea_b, nullptr, C.jaa_off, true, 0, 1.0, N));
        return r;
      }
      r.push_back(recipe_of(C.sa, C.ea_a, &C.fwd[k], 0, false, 0, 0.0, N));
      r.push_back(recipe_of(C.sb, C.ea_b, &C.fwd[k], C.jaa_off, k < R, k, 1.0, N));
      if (k < R) r.push_back(recipe_of(C.sa, C.ea_o, nullptr, C.jaa_off, true, k, 1.0, N));
      return r;
    });
    if (k == 0 && any_hf) {
      std::vector<BSl> sl;
      std::vector<BSd> sd;
      int64_t ts = 0, tr = 0;
      for (auto& C : cs) {
        if (!C.hf()) continue;
        const int N = C.op->norb;
        // R and X pointers are image offsets + 1 until the image is placed
        const CMat* r0 = (const CMat*)(uintptr_t)(C.r0_off + 1);
        sl.push_back(BSl{C.sa->masks, C.sl_a, r0, ts, N, C.op->n_alpha});
        ts += C.sa->dim;
        sl.push_back(BSl{C.sb->masks, C.sl_b, r0, ts, N, C.op->n_beta});
        ts += C.sb->dim;
        BSd d{};
        d.vec = vecs[C.idx];
        d.va = C.sl_a;
        d.vb = C.sl_b;
        d.ea_a = C.ea_a;
        d.ea_b = C.ea_b;
        d.X = (const Mat*)(uintptr_t)(C.xab_off + 1);
        d.ma = C.sa->masks;
        d.mb = C.sb->masks;
        d.db = C.sb->dim;
        d.norb = N;
        d.item0 = tr;
        tr += C.sa->dim;
        sd.push_back(d);
      }
      Stage S4;
      S4.kind = 4;
      S4.njobs = (int)sl.size();
      S4.total = ts;
      S4.jobs_off = img.add(sl.data(), sl.size() * sizeof(BSl));
      stages.push_back(S4);
      Stage S5;
      S5.kind = 5;
      S5.njobs = (int)sd.size();
      S5.total = tr;
      S5.jobs_off = img.add(sd.data(), sd.size() * sizeof(BSd));
      stages.push_back(S5);
    }
    sweep_stage(0, 1, sweeps_k(k), [&](Circuit& C, PhaseDev& ph, RevArgs&, const RotProgram*& rp, long& xk,
                          bool&) {
      ph.ea_a = C.ea_a;
      rp = &C.fwd[k];
      xk = -1;
    });
    sweep_stage(1, 1, sweeps_k(k), [&](Circuit& C, PhaseDev& ph, RevArgs&, const RotProgram*& rp, long& xk,
                          bool&) {
      ph.ea_b = C.ea_b;
      rp = &C.fwd[k];
      if (k < R) {
        ph.ea_a = C.ea_o;
        ph.has_x = 1;
        xk = k;
      } else {
        xk = -1;
      }
    });
  }
  // ---------------- reverse
  if (do_vjp && R > 0) {
    for (int m = R; m >= 0; --m) {
      phase_stage([&](Circuit& C) {
        const int N = C.op->norb;
        std::vector<BStr> r;
        r.push_back(recipe_of(C.sb, C.ea_b, &C.rev[m], 0, false, 0, 0.0, N));
        return r;
      });
      sweep_stage(1, 2, all, [&](Circuit& C, PhaseDev& ph, RevArgs& rv, const RotProgram*& rp, long& xk,
                            bool& has_rev) {
        const int N = C.op->norb;
        ph.ea_b = C.ea_b;
        rp = &C.rev[m];
        rv.T = C.T + (size_t)m * N * N * 2;
        has_rev = true;
        xk = -1;
      });
      phase_stage([&](Circuit& C) {
        const int N = C.op->norb;
        std::vector<BStr> r;
        r.push_back(recipe_of(C.sa, C.ea_a, &C.rev[m], 0, false, 0, 0.0, N));
        if (m >= 1) {
          r.push_back(recipe_of(C.sa, C.e2_a, nullptr, C.jaa_off, true, m - 1, -1.0, N));
          r.push_back(recipe_of(C.sb, C.e2_b, nullptr, C.jaa_off, true, m - 1, -1.0, N));
        }
        return r;
      });
      sweep_stage(0, 2, all, [&](Circuit& C, PhaseDev& ph, RevArgs& rv, const RotProgram*& rp, long& xk,
                            bool& has_rev) {
        const int N = C.op->norb;
        ph.ea_a = C.ea_a;
        rp = &C.rev[m];
        rv.T = C.T + (size_t)m * N * N * 2;
        has_rev = true;
        xk = -1;
        if (m >= 1) {
          rv.ea2_a = C.e2_a;
          rv.ea2_b = C.e2_b;
          rv.W = C.W;
          ph.has_x = 1;
          xk = R + (m - 1);
        }
      });
      if (m >= 1) {
        std::vector<BDc> js;
        int64_t rows = 0, cols = 0, pqs = 0;
        for (auto& C : cs) {
          const int N = C.op->norb;
          BDc b{};
          b.W = C.W;
          b.ma = C.sa->masks;
          b.mb = C.sb->masks;
          b.dJaa = C.dJ + (size_t)(m - 1) * N * N;
          b.dJab = C.dJ + (size_t)(R + m - 1) * N * N;
          b.c = C.colsum;
          b.da = C.sa->dim;
          b.db = C.sb->dim;
          b.norb = N;
          js.push_back(b);
          rows += b.da;
          cols += b.db;
          pqs += N * N;
        }
        // three kernels, three item numberings: rows, columns, (p, q)
        std::vector<BDc> jr = js, jc = js, jp = js;
        int64_t a = 0, b2 = 0, c3 = 0;
        for (size_t i = 0; i < js.size(); ++i) {
          jr[i].item0 = a;
          a += js[i].da;
          jc[i].item0 = b2;
          b2 += js[i].db;
          jp[i].item0 = c3;
          c3 += js[i].norb * js[i].norb;
        }
        Stage S;
        S.kind = 3;
        S.njobs = (int)js.size();
        S.total = rows;
        S.total2 = cols;
        S.total3 = pqs;
        S.jobs_off = img.add(jr.data(), jr.size() * sizeof(BDc));
        img.add(jc.data(), jc.size() * sizeof(BDc), 1);
        img.add(jp.data(), jp.size() * sizeof(BDc), 1);
        stages.push_back(S);
      }
    }
  }
  // sweep jobs: patch program/X pointers after the image layout is fixed
  std::vector<size_t> job_offs(pend.size());
  for (size_t i = 0; i < pend.size(); ++i)
    job_offs[i] = img.add(nullptr, pend[i].jobs.size() * sizeof(SweepJob));
  const size_t counters_off = img.add(nullptr, std::max(ncounters, 1) * sizeof(int));
  dimg = (unsigned char*)scratch(ctx, "batch_image", img.bytes.size());
  for (size_t i = 0; i < pend.size(); ++i) {
    for (size_t j = 0; j < pend[i].jobs.size(); ++j) {
      SweepJob& J = pend[i].jobs[j];
      J.prog = dimg + pend[i].prog_off[j];
      J.X = (const Mat*)(dimg + (pend[i].x_off[j] == (size_t)-1 ? zero_off : pend[i].x_off[j]));
    }
    memcpy(img.bytes.data() + job_offs[i], pend[i].jobs.data(),
           pend[i].jobs.size() * sizeof(SweepJob));
    stages[pend[i].stage].jobs_off = job_offs[i];
  }
  // string-phase recipes and Slater jobs: image offsets -> device pointers
  for (auto& S : stages) {
    if (S.kind == 0) {
      BStr* b = (BStr*)(img.bytes.data() + S.jobs_off);
      for (int i = 0; i < S.njobs; ++i)
        if (b[i].J) b[i].J = (const double*)(dimg + ((uintptr_t)b[i].J - 1));
    } else if (S.kind == 4) {
      BSl* b = (BSl*)(img.bytes.data() + S.jobs_off);
      for (int i = 0; i < S.njobs; ++i) b[i].R = (const CMat*)(dimg + ((uintptr_t)b[i].R - 1));
    } else if (S.kind == 5) {
      BSd* b = (BSd*)(img.bytes.data() + S.jobs_off);
      for (int i = 0; i < S.njobs; ++i) b[i].X = (const Mat*)(dimg + ((uintptr_t)b[i].X - 1));
    }
  }
  memset(img.bytes.data() + counters_off, 0, std::max(ncounters, 1) * sizeof(int));
  FS_CUDA(cudaMemcpyAsync(dimg, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice, st));
  // accumulators start at zero
  for (int c = 0; c < n; ++c) {
    const int N = cs[c].op->norb;
    FS_CUDA(cudaMemsetAsync(cs[c].T, 0, (size_t)(R + 1) * N * N * 2 * sizeof(double), st));
    FS_CUDA(cudaMemsetAsync(cs[c].dJ, 0, (size_t)2 * std::max(R, 1) * N * N * sizeof(double), st));
  }
  (void)acc_begin;
  int* counters = (int*)(dimg + counters_off);

  // kernel attributes are set before the capture starts
  for (auto& S : stages)
    if (S.kind == 1) launch_sweep_batch(ctx, dtype, S.nst, nullptr, 0, 0, nullptr, S.smem, st, S.pk);
  // ---- record the stages into one graph and launch it on `st`
  if (!ctx->capture_stream)
    FS_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
  cudaStream_t cst = ctx->capture_stream;
  const bool prof = ctx->prof_on;
  ctx->prof_on = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  FS_CUDA(cudaStreamBeginCapture(cst, cudaStreamCaptureModeThreadLocal));
  try {
    const int sms = ctx->prop.multiProcessorCount;
    for (auto& S : stages) {
      const unsigned char* jp = dimg + S.jobs_off;
      if (S.kind == 0) {
        unsigned grid = (unsigned)std::min<int64_t>((S.total + 255) / 256, 16 * sms);
        if (dtype == FS_C64)
          k_string_phase_batch<float><<<grid, 256, 0, cst>>>((const BStr*)jp, S.njobs, S.total);
        else
          k_string_phase_batch<double><<<grid, 256, 0, cst>>>((const BStr*)jp, S.njobs, S.total);
      } else if (S.kind == 2) {
        unsigned grid = (unsigned)std::min<int64_t>((S.total + 255) / 256, 32 * sms);
        if (dtype == FS_C64)
          k_hf_batch<float><<<grid, 256, 0, cst>>>((const BVec*)jp, S.njobs, S.total);
        else
          k_hf_batch<double><<<grid, 256, 0, cst>>>((const BVec*)jp, S.njobs, S.total);
      } else if (S.kind == 1) {
        launch_sweep_batch(ctx, dtype, S.nst, (const SweepJob*)jp, S.njobs, (int)S.total,
                           counters + S.counter, S.smem, cst, S.pk);
      } else if (S.kind == 4) {
        unsigned grid = (unsigned)std::min<int64_t>((S.total + 63) / 64, 16 * sms);
        k_slater_batch<<<grid, 64, 0, cst>>>((const BSl*)jp, S.njobs, S.total);
      } else if (S.kind == 5) {
        unsigned grid = (unsigned)std::min<int64_t>(S.total, 16 * sms);
        if (dtype == FS_C64)
          k_slater_dc_batch<float><<<grid, 256, 0, cst>>>((const BSd*)jp, S.njobs, S.total);
        else
          k_slater_dc_batch<double><<<grid, 256, 0, cst>>>((const BSd*)jp, S.njobs, S.total);
      } else {
        const BDc* jr = (const BDc*)jp;
        const BDc* jc = jr + S.njobs;
        const BDc* jq = jc + S.njobs;
        unsigned g1 = (unsigned)std::min<int64_t>(S.total, 8 * sms);
        unsigned g2 = (unsigned)std::min<int64_t>((S.total2 + 127) / 128, 16 * sms);
        unsigned g3 = (unsigned)std::min<int64_t>(S.total3, 8 * sms);
        if (dtype == FS_C64) {
          k_dc_rows_batch<float><<<g1, 128, 0, cst>>>(jr, S.njobs, S.total);
          k_dc_cols_batch<float><<<g2, 128, 0, cst>>>(jc, S.njobs, S.total2);
        } else {
          k_dc_rows_batch<double><<<g1, 128, 0, cst>>>(jr, S.njobs, S.total);
          k_dc_cols_batch<double><<<g2, 128, 0, cst>>>(jc, S.njobs, S.total2);
        }
        k_dc_beta_aa_batch<<<g3, 128, 0, cst>>>(jq, S.njobs, S.total3);
      }
      FS_CUDA(cudaGetLastError());
    }
  } catch (...) {
    cudaGraph_t g2 = nullptr;
    cudaStreamEndCapture(cst, &g2);
    if (g2) cudaGraphDestroy(g2);
    ctx->prof_on = prof;
    throw;
  }
  FS_CUDA(cudaStreamEndCapture(cst, &graph));
  ctx->prof_on = prof;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    FS_CUDA(e);
  }
  {
    ProfScope ps("lucj_batch_graph", st, (int)stages.size());
    e = cudaGraphLaunch(exec, st);
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  FS_CUDA(e);
  if (!do_vjp || R == 0) return;
  // ---- gradients: T and dJ to the host, chain rule in FP64
  for (auto& C : cs) {
    const int N = C.op->norb;
    const size_t nn = (size_t)N * N;
    std::vector<double> Th((R + 1) * nn * 2), dJh(2 * R * nn);
    FS_CUDA(cudaMemcpyAsync(Th.data(), C.T, Th.size() * 8, cudaMemcpyDeviceToHost, st));
    FS_CUDA(cudaMemcpyAsync(dJh.data(), C.dJ, dJh.size() * 8, cudaMemcpyDeviceToHost, st));
    FS_CUDA(cudaStreamSynchronize(st));
    if (dJaa && dJaa[C.idx]) std::copy(dJh.begin(), dJh.begin() + R * nn, dJaa[C.idx]);
    if (dJab && dJab[C.idx]) std::copy(dJh.begin() + R * nn, dJh.end(), dJab[C.idx]);
    if (!dK || !dK[C.idx]) continue;
    std::vector<std::vector<zd>> gU(R, std::vector<zd>(nn, zd(0)));
    std::vector<zd> gR(nn), cT(nn), tmp(nn), tmp2(nn);
    for (int m = 0; m <= R; ++m) {
      for (size_t q = 0; q < nn; ++q) cT[q] = zd(Th[2 * (m * nn + q)], -Th[2 * (m * nn + q) + 1]);
      mat_mul(N, C.Rs[m].data(), cT.data(), gR.data());
      if (m == 0) {
        mat_adjoint(N, gR.data(), tmp.data());
        for (size_t q = 0; q < nn; ++q) gU[0][q] += tmp[q];
      }
      if (m == R)
        for (size_t q = 0; q < nn; ++q) gU[R - 1][q] += gR[q];
      if (m >= 1 && m <= R - 1) {
        mat_mul(N, C.Us[m].data(), gR.data(), tmp.data());
        for (size_t q = 0; q < nn; ++q) gU[m - 1][q] += tmp[q];
        mat_adjoint(N, gR.data(), tmp2.data());
        mat_mul(N, C.Us[m - 1].data(), tmp2.data(), tmp.data());
        for (size_t q = 0; q < nn; ++q) gU[m][q] += tmp[q];
      }
    }
    for (int k = 0; k < R; ++k) {
      std::vector<zd> K(nn), out(nn);
      for (size_t q = 0; q < nn; ++q)
        K[q] = zd(C.op->K[2 * (k * nn + q)], C.op->K[2 * (k * nn + q) + 1]);
      expm_frechet_adjoint(N, K.data(), gU[k].data(), out.data());
      for (size_t q = 0; q < nn; ++q) {
        dK[C.idx][2 * (k * nn + q)] = out[q].real();
        dK[C.idx][2 * (k * nn + q) + 1] = out[q].imag();
      }
    }
  }
}

void lucj_batch(Ctx* ctx, int n, const fs_lucj* ops, void* const* vecs, void* const* cots,
                int dtype, int do_vjp, double* const* dK, double* const* dJaa,
                double* const* dJab, cudaStream_t st) {
  lucj_batch_impl(ctx, n, ops, vecs, cots, dtype, do_vjp, dK, dJaa, dJab, st);
}

}  // namespace fs
