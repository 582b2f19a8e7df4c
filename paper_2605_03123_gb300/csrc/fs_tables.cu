// String tables built on the device with the combinatorial number system:
// the string of address r has the occupied orbitals o_0 < ... < o_{n-1}
// with r = sum_k C(o_k, k+1) (§3.1 addressing, ascending-mask order).
#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

__constant__ uint32_t c_binom[kMaxOrb + 1][kMaxOrb + 1];

// Constant memory is per device: upload the table once for each device
// this process uses (the current device at the time of the call).
static void upload_binomials() {
  static std::mutex m;
  static bool done[256] = {};
  int dev = 0;
  FS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(m);
  if (dev >= 0 && dev < 256 && done[dev]) return;
  uint32_t h[kMaxOrb + 1][kMaxOrb + 1];
  for (int n = 0; n <= kMaxOrb; ++n)
    for (int k = 0; k <= kMaxOrb; ++k) h[n][k] = (uint32_t)binom_host(n, k);
  FS_CUDA(cudaMemcpyToSymbol(c_binom, h, sizeof(h)));
  if (dev >= 0 && dev < 256) done[dev] = true;
}

__device__ __forceinline__ uint32_t cns_rank(uint32_t mask) {
  uint32_t r = 0;
  int k = 0;
  while (mask) {
    int o = __ffs(mask) - 1;
    r += c_binom[o][k + 1];
    ++k;
    mask &= mask - 1;
  }
  return r;
}

// The string of address r among strings of n electrons in `norb` orbitals:
// choose the occupied orbitals from the top, o = largest with C(o, k) <= r.
__device__ __forceinline__ uint32_t cns_unrank(uint32_t r, int n, int norb) {
  uint32_t mask = 0;
  int o = norb - 1;
  for (int k = n; k >= 1; --k) {
    while (c_binom[o][k] > r) --o;
    mask |= 1u << o;
    r -= c_binom[o][k];
    --o;
  }
  return mask;
}

// Insert zero bits at positions lo < hi into an (norb-2)-bit mask.
__device__ __forceinline__ uint32_t expand2(uint32_t m, int lo, int hi) {
  uint32_t low = m & ((1u << lo) - 1u);
  uint32_t rest = (m >> lo) << (lo + 1);  // zero at lo
  m = low | rest;
  low = m & ((1u << hi) - 1u);
  rest = (m >> hi) << (hi + 1);  // zero at hi
  return low | rest;
}
__device__ __forceinline__ uint32_t expand1(uint32_t m, int pos) {
  uint32_t low = m & ((1u << pos) - 1u);
  return low | ((m >> pos) << (pos + 1));
}

__global__ void k_masks(uint32_t* masks, int64_t dim, int n, int norb) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < dim) masks[r] = cns_unrank((uint32_t)r, n, norb);
}

// Adjacent pair lists: for p = 0..norb-2 and t < npp, the t-th string with
// p occupied and p+1 empty; entry = src | dst << 16 with dst = I^{p->p+1}.
__global__ void k_adjacent_pairs(uint32_t* pairs, int npp, int n, int norb) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int p = blockIdx.y;
  if (t >= npp) return;
  uint32_t m = expand2(cns_unrank((uint32_t)t, n - 1, norb - 2), p, p + 1);
  uint32_t src = cns_rank(m | (1u << p));
  uint32_t dst = cns_rank(m | (1u << (p + 1)));
  pairs[(int64_t)p * npp + t] = src | (dst << 16);
}

// Ordered-pair lists for E_pq = a^dag_p a_q: strings with q occupied and p
// empty (p != q), src = I, dst = I^{q->p}, sign bit set when the number of
// occupied orbitals strictly between p and q is odd.  Diagonal lists (p == q)
// hold the strings with p occupied, src = dst, sign 0.
__global__ void k_cross_pairs(uint32_t* xp, uint32_t* xs, int* cnt, int nx,
                              int n, int norb) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int p = blockIdx.y / norb, q = blockIdx.y % norb;
  int64_t base = (int64_t)blockIdx.y * nx;
  int nw = (nx + 31) / 32;
  if (p == q) {
    int count = (n >= 1) ? (int)c_binom[norb - 1][n - 1] : 0;
    if (t == 0) cnt[blockIdx.y] = count;
    if (t >= count) return;
    uint32_t m = expand1(cns_unrank((uint32_t)t, n - 1, norb - 1), p) | (1u << p);
    uint32_t r = cns_rank(m);
    xp[base + t] = r | (r << 16);
    return;
  }
  int count = (n >= 1 && norb >= 2) ? (int)c_binom[norb - 2][n - 1] : 0;
  if (t == 0) cnt[blockIdx.y] = count;
  if (t >= count) return;
  int lo = min(p, q), hi = max(p, q);
  uint32_t m = expand2(cns_unrank((uint32_t)t, n - 1, norb - 2), lo, hi);
  uint32_t src = cns_rank(m | (1u << q));
  uint32_t dst = cns_rank(m | (1u << p));
  uint32_t between = ((1u << hi) - 1u) & ~((2u << lo) - 1u);
  uint32_t sgn = __popc(m & between) & 1u;
  xp[base + t] = src | (dst << 16);
  if (sgn) atomicOr(&xs[(int64_t)blockIdx.y * nw + t / 32], 1u << (t % 32));
}

// Full excitation table for the C ABI: out[(i*norb + p)*norb + q].
__global__ void k_exc_table(uint32_t* out, const uint32_t* masks, int64_t dim,
                            int norb) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= dim) return;
  uint32_t m = masks[i];
  for (int p = 0; p < norb; ++p)
    for (int q = 0; q < norb; ++q) {
      uint32_t v = 0xFFFFFFFFu;
      if ((m >> q) & 1u) {
        if (p == q) {
          v = (uint32_t)i;
        } else if (!((m >> p) & 1u)) {
          int lo = min(p, q), hi = max(p, q);
          uint32_t between = ((1u << hi) - 1u) & ~((2u << lo) - 1u);
          uint32_t m2 = (m & ~(1u << q)) | (1u << p);
          v = cns_rank(m2) | ((uint32_t)(__popc(m & between) & 1) << 31);
        }
      }
      out[(i * norb + p) * norb + q] = v;
    }
}

// Gather table of the single excitations of each string t: for every
// p in t and q not in t or q == p, in (p, q) order, the entry
// pq = p * norb + q and src = E_qp t with sign bit 31 = the sign of
// a^dag_q a_p |t> (equal to <t| a^dag_p a_q |src>).  ne = n(N - n) + n
// entries per string.
__global__ void k_gather_table(uint16_t* pq_out, uint32_t* src_out, const uint32_t* masks,
                               int64_t dim, int norb, int ne) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= dim) return;
  const uint32_t m = masks[t];
  int k = 0;
  for (int p = 0; p < norb; ++p) {
    if (!((m >> p) & 1u)) continue;
    for (int q = 0; q < norb; ++q) {
      uint32_t v;
      if (q == p) {
        v = (uint32_t)t;
      } else if (!((m >> q) & 1u)) {
        const int lo = min(p, q), hi = max(p, q);
        const uint32_t between = ((1u << hi) - 1u) & ~((2u << lo) - 1u);
        const uint32_t m2 = (m & ~(1u << p)) | (1u << q);
        v = cns_rank(m2) | ((uint32_t)(__popc(m & between) & 1) << 31);
      } else {
        continue;
      }
      if (k < ne) {
        pq_out[t * ne + k] = (uint16_t)(p * norb + q);
        src_out[t * ne + k] = v;
      }
      ++k;
    }
  }
}

static int64_t choose(int n, int k) { return (int64_t)binom_host(n, k); }

void build_gather_table(Space* sp, cudaStream_t st) {
  if (sp->gpq) return;
  const int n = sp->nocc, N = sp->norb;
  sp->ne = n * (N - n) + n;
  const size_t cnt = (size_t)sp->dim * std::max(sp->ne, 1);
  FS_CUDA(cudaMalloc(&sp->gpq, cnt * sizeof(uint16_t)));
  FS_CUDA(cudaMalloc(&sp->gsrc, cnt * sizeof(uint32_t)));
  if (sp->ne > 0) {
    k_gather_table<<<(unsigned)((sp->dim + 127) / 128), 128, 0, st>>>(sp->gpq, sp->gsrc,
                                                                    sp->masks, sp->dim, N,
                                                                    sp->ne);
    FS_CUDA(cudaGetLastError());
  }
}

Space* get_space(Ctx* ctx, int norb, int nocc, cudaStream_t st) {
  auto key = std::make_pair(norb, nocc);
  auto it = ctx->spaces.find(key);
  if (it != ctx->spaces.end()) return it->second;
  upload_binomials();
  Space* s = new Space();
  s->norb = norb;
  s->nocc = nocc;
  s->dim = choose(norb, nocc);
  try {
    FS_CUDA(cudaMalloc(&s->masks, s->dim * sizeof(uint32_t)));
    k_masks<<<(unsigned)((s->dim + 255) / 256), 256, 0, st>>>(s->masks, s->dim,
                                                               nocc, norb);
    FS_CUDA(cudaGetLastError());
    if (s->dim <= kMaxSweepDim) {
      s->npp = (norb >= 2 && nocc >= 1) ? (int)choose(norb - 2, nocc - 1) : 0;
      if (s->npp > 0) {
        FS_CUDA(cudaMalloc(&s->pairs, (size_t)(norb - 1) * s->npp * 4));
        dim3 g((s->npp + 255) / 256, norb - 1);
        k_adjacent_pairs<<<g, 256, 0, st>>>(s->pairs, s->npp, nocc, norb);
        FS_CUDA(cudaGetLastError());
      }
      s->nx = nocc >= 1 ? (int)choose(norb - 1, nocc - 1) : 0;
      if (s->nx > 0) {
        size_t nlist = (size_t)norb * norb;
        int nw = (s->nx + 31) / 32;
        FS_CUDA(cudaMalloc(&s->xpairs, nlist * s->nx * 4));
        FS_CUDA(cudaMalloc(&s->xsign, nlist * nw * 4));
        FS_CUDA(cudaMalloc(&s->xcount, nlist * sizeof(int)));
        FS_CUDA(cudaMemsetAsync(s->xsign, 0, nlist * nw * 4, st));
        dim3 g((s->nx + 255) / 256, (unsigned)nlist);
        k_cross_pairs<<<g, 256, 0, st>>>(s->xpairs, s->xsign, s->xcount, s->nx,
                                         nocc, norb);
        FS_CUDA(cudaGetLastError());
      }
    }
  } catch (...) {
    free_space(s);
    throw;
  }
  ctx->spaces[key] = s;
  return s;
}

void free_space(Space* s) {
  if (!s) return;
  cudaFree(s->masks);
  cudaFree(s->pairs);
  cudaFree(s->xpairs);
  cudaFree(s->xsign);
  cudaFree(s->xcount);
  cudaFree(s->tpass);
  cudaFree(s->trec);
  cudaFree(s->gpq);
  cudaFree(s->gsrc);
  for (int b = 0; b < 4; ++b) {
    cudaFree(s->tgrec[b]);
    cudaFree(s->tgoff[b]);
  }
  for (auto& w : s->win) {
    cudaFree(w.orbits);
    cudaFree(w.off);
    cudaFree(w.offs);
    for (int b = 0; b < 4; ++b) {
      cudaFree(w.gorb[b]);
      cudaFree(w.goff[b]);
    }
  }
  delete s;
}

void preload_mask_kernel() {
  cudaFuncAttributes fa;
  FS_CUDA(cudaFuncGetAttributes(&fa, k_masks));
}

void launch_masks(uint32_t* out, int norb, int nocc, cudaStream_t st) {
  upload_binomials();
  int64_t dim = choose(norb, nocc);
  k_masks<<<(unsigned)((dim + 255) / 256), 256, 0, st>>>(out, dim, nocc, norb);
  FS_CUDA(cudaGetLastError());
}

void launch_exc_table(const Space* sp, uint32_t* out, cudaStream_t st) {
  k_exc_table<<<(unsigned)((sp->dim + 127) / 128), 128, 0, st>>>(
      out, sp->masks, sp->dim, sp->norb);
  FS_CUDA(cudaGetLastError());
}

}  // namespace fs
