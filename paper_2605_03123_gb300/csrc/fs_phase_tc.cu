// Diagonal-Coulomb phase of a complex64 state in one streaming pass, with
// the alpha-beta cross term on the tcgen05 tensor cores and the state moved
// by the tensor memory accelerator.
//
// theta(i, j) = A_i + B_j + sum_{p in I_a(i), q in I_b(j)} X[p][q]  (§3.2.2,
// X = -t J_ab).  With Y[p][j] = sum_{q in I_b(j)} X[p][q] (formed in FP64 and
// reduced mod 2 pi), the cross term of a tile of 128 alpha x 16 beta strings
// is Z = Occ_a Y: a 128 x K 0/1 matrix times K x 16 (K = 16 or 32 orbitals).
// Y is split into three BF16 pieces (24 significand bits) and occupations
// are exact in BF16, so the three products per tile are exact and only the
// FP32 accumulation of at most 3K terms rounds.  A_i and B_j arrive as
// per-string factors.
//
// A CTA walks its tiles through an STAGES-deep ring in shared memory: one
// thread loads a stage with a 2-D TMA copy of the state tile (128 rows x 128
// bytes, 128-byte swizzle) and bulk copies of the tile's occupations, Y
// pieces and factors, all completing on the stage's mbarrier; issues the
// three MMAs into a TMEM accumulator (double buffered); after the 128
// threads (thread = row = TMEM lane) have applied the phases in place, it
// stores the tile back with a 2-D TMA copy.  Waits are bounded; the TMEM is
// always freed.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "fs_common.cuh"
#include "fs_internal.h"
#include "fs_tc.cuh"

namespace fs {
namespace dct {

constexpr int TI = 128, TJ = 16;            // tile: alpha rows x beta columns
constexpr int STAGES = 4, THREADS = 128;
constexpr int STATE_BYTES = TI * TJ * 8;    // 16 KB, 128-byte rows, swizzled
__host__ __device__ constexpr int occ_bytes(int nk) { return TI * nk * 2; }
__host__ __device__ constexpr int y_bytes(int nk) { return 3 * TJ * nk * 2; }
__host__ __device__ constexpr int stage_bytes(int nk) {
  return STATE_BYTES + occ_bytes(nk) + y_bytes(nk) + TI * 8 + TJ * 8;
}
// byte offset of (row r, k) in a K-major no-swizzle core-matrix layout
__host__ __device__ inline int core_offset(int r, int k, int nk) {
  return ((r >> 3) * (nk >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

}  // namespace dct

// Occupations of the alpha strings, per tile of 128 rows in the MMA layout
// (rows past dim_a zero), and the alpha factors padded to whole tiles.
__global__ void k_dc_occ(__nv_bfloat16* occ, float2* eaa, const uint32_t* ma, const float2* ea,
                         int64_t da, int64_t nti, int nk) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nti * dct::TI) return;
  const uint32_t m = r < da ? ma[r] : 0u;
  __nv_bfloat16* t = occ + (r / dct::TI) * (dct::occ_bytes(nk) / 2);
  const int rr = (int)(r % dct::TI);
  for (int k = 0; k < nk; ++k)
    t[dct::core_offset(rr, k, nk) / 2] = __float2bfloat16_rn(((m >> k) & 1u) ? 1.f : 0.f);
  eaa[r] = r < da ? (ea ? ea[r] : make_float2(1.f, 0.f)) : make_float2(0.f, 0.f);
}

// Y[p][j] = sum_{q in I_b(j)} X[p][q] reduced mod 2 pi in FP64, as three
// BF16 pieces per tile of 16 columns in the MMA layout (rows j, K = p), and
// the beta factors padded to whole tiles.
__global__ void k_dc_ypieces(__nv_bfloat16* y, float2* eab, const uint32_t* mb, const float2* eb,
                             int64_t db, int64_t ntj, int norb, int nk,
                             const __grid_constant__ Mat X) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= ntj * dct::TJ) return;
  const uint32_t m = j < db ? mb[j] : 0u;
  __nv_bfloat16* t = y + (j / dct::TJ) * (dct::y_bytes(nk) / 2);
  const int jj = (int)(j % dct::TJ);
  for (int p = 0; p < nk; ++p) {
    double v = 0;
    if (p < norb && j < db)
      for (uint32_t b = m; b; b &= b - 1) v += X.v[p * norb + (__ffs(b) - 1)];
    v -= 6.283185307179586 * rint(v * 0.15915494309189535);
    double r = v;
    for (int pc = 0; pc < 3; ++pc) {
      const __nv_bfloat16 h = __float2bfloat16_rn((float)r);
      t[pc * dct::TJ * nk + dct::core_offset(jj, p, nk) / 2] = h;
      r -= (double)__bfloat162float(h);
    }
  }
  eab[j] = j < db ? (eb ? eb[j] : make_float2(1.f, 0.f)) : make_float2(0.f, 0.f);
}

template <int NK>
__global__ void __launch_bounds__(dct::THREADS, 1)
    k_phase_tc(const __grid_constant__ CUtensorMap map, const __nv_bfloat16* occ,
               const float2* eaa, const __nv_bfloat16* ypc, const float2* eab, int64_t nti,
               int64_t ntj, int* status) {
  using namespace dct;
  constexpr int SB = stage_bytes(NK);
  constexpr int OFF_OCC = STATE_BYTES, OFF_Y = OFF_OCC + occ_bytes(NK);
  constexpr int OFF_EA = OFF_Y + y_bytes(NK), OFF_EB = OFF_EA + TI * 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(8) uint64_t s_full[STAGES];
  __shared__ __align__(8) uint64_t s_mma[2];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sraw = tc::smem_u32(smraw);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;
  constexpr int SSTRIDE = (SB + 1023) / 1024 * 1024;  // stages 1024-byte aligned (swizzle)
  unsigned char* sgen = smraw + (sbase - sraw);
  const int64_t ntiles = nti * ntj;
  // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
  const int64_t mine = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) tc::mbar_init(tc::smem_u32(&s_full[s]), 1);
    for (int s = 0; s < 2; ++s) tc::mbar_init(tc::smem_u32(&s_mma[s]), 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&s_tmem), 32);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = s_tmem;
  auto timeout = [&]() {
    if (status) atomicCAS(status, 0, (int)FS_ERR_TIMEOUT);
  };
  auto load = [&](int64_t u) {  // thread 0: tile u of this CTA into stage u % STAGES
    const int s = (int)(u % STAGES);
    const int64_t t = blockIdx.x + u * gridDim.x;
    const int64_t ti = t / ntj, tj = t - ti * ntj;
    const uint32_t st = sbase + (uint32_t)(s * SSTRIDE);
    const uint32_t mb = tc::smem_u32(&s_full[s]);
    tc::mbar_expect_tx(mb, (uint32_t)SB);
    tc::tma_load_2d(st, &map, (int)(tj * TJ), (int)(ti * TI), mb);
    tc::bulk_g2s(st + OFF_OCC, occ + ti * (occ_bytes(NK) / 2), occ_bytes(NK), mb);
    tc::bulk_g2s(st + OFF_Y, ypc + tj * (y_bytes(NK) / 2), y_bytes(NK), mb);
    tc::bulk_g2s(st + OFF_EA, eaa + ti * TI, TI * 8, mb);
    tc::bulk_g2s(st + OFF_EB, eab + tj * TJ, TJ * 8, mb);
  };
  if (tid == 0)
    for (int64_t u = 0; u < STAGES - 1 && u < mine; ++u) load(u);
  for (int64_t u = 0; u < mine; ++u) {
    const int s = (int)(u % STAGES), b = (int)(u & 1);
    const uint32_t st = sbase + (uint32_t)(s * SSTRIDE);
    unsigned char* sg = sgen + s * SSTRIDE;
    if (!tc::mbar_wait(tc::smem_u32(&s_full[s]), (uint32_t)(u / STAGES) & 1u)) timeout();
    if (tid == 0) {
      tc::fence_after();
      constexpr uint32_t ID = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TJ >> 3) << 17) |
                              ((uint32_t)(TI >> 4) << 24);
      constexpr uint32_t SBO = (NK / 8) * 128;
#pragma unroll
      for (int pc = 2; pc >= 0; --pc)
#pragma unroll
        for (int ks = 0; ks < NK / 16; ++ks) {
          const uint64_t ad = tc::sdesc(st + OFF_OCC + ks * 256, 128, SBO);
          const uint64_t bd = tc::sdesc(st + OFF_Y + pc * (TJ * NK * 2) + ks * 256, 128, SBO);
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tm + 16 * b),
              "l"(ad), "l"(bd), "r"(ID), "r"((pc < 2 || ks > 0) ? 1u : 0u)
              : "memory");
        }
      tc::mma_commit(tc::smem_u32(&s_mma[b]));
      // refill: tile u + STAGES - 1 into the stage of tile u - 1, once the
      // store of tile u - 1 has read it
      if (u + STAGES - 1 < mine) {
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        load(u + STAGES - 1);
      }
    }
    __syncwarp();
    if (!tc::mbar_wait(tc::smem_u32(&s_mma[b]), (uint32_t)(u >> 1) & 1u)) timeout();
    tc::fence_after();
    // thread = row: 16 angles from TMEM, 16 amplitudes from the swizzled tile
    uint32_t z[16];
    {
      uint32_t lo[8], hi[8];
      const uint32_t ta = tm + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * b);
      tc::tmem_ld8(ta, lo);
      tc::tmem_ld8(ta + 8, hi);
      tc::wait_ld();
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        z[c] = lo[c];
        z[8 + c] = hi[c];
      }
    }
    const int r = 32 * warp + lane;
    const float2 fa = reinterpret_cast<const float2*>(sg + OFF_EA)[r];
    const float2* fbv = reinterpret_cast<const float2*>(sg + OFF_EB);
    unsigned char* row = sg + r * 128;
#pragma unroll
    for (int c = 0; c < 8; ++c) {  // 16-byte chunk c holds columns 2c, 2c+1
      float4* p = reinterpret_cast<float4*>(row + ((c ^ (r & 7)) << 4));
      float4 v = *p;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        // the angle is a sum of at most 3K terms reduced to [-pi, pi]:
        // bring it back to [-pi, pi] (2 pi in two parts), hardware sincos
        const float zz = __uint_as_float(z[2 * c + h]);
        const float kq = rintf(zz * 0.15915494f);
        const float rr = fmaf(kq, 1.7484555e-07f, fmaf(-kq, 6.28318548f, zz));
        float sn, co;
        __sincosf(rr, &sn, &co);
        const float2 fb = fbv[2 * c + h];
        const float2 fab = make_float2(fa.x * fb.x - fa.y * fb.y, fa.x * fb.y + fa.y * fb.x);
        const float2 f = make_float2(fab.x * co - fab.y * sn, fab.x * sn + fab.y * co);
        float& xr = h ? v.z : v.x;
        float& xi = h ? v.w : v.y;
        const float nr = f.x * xr - f.y * xi, ni = f.x * xi + f.y * xr;
        xr = nr;
        xi = ni;
      }
      *p = v;
    }
    // the TMA store reads through the async proxy: publish the writes, then
    // one thread stores once every row is done
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      const int64_t t = blockIdx.x + u * gridDim.x;
      const int64_t ti = t / ntj, tj = t - ti * ntj;
      tc::tma_store_2d(&map, (int)(tj * TJ), (int)(ti * TI), st);
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tm, 32);
  }
}

bool phase_tc_supported(int dtype, const Space* sa, const Space* sb, const void* vec) {
  // the TMA tensor map needs 16-byte row strides: an even beta dimension
  return dtype == FS_C64 && sa->norb <= 32 && sb->dim % 2 == 0 && ((uintptr_t)vec & 15u) == 0;
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_tiled() {
  static std::mutex m;
  static EncodeTiled fn = nullptr;
  std::lock_guard<std::mutex> g(m);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    FS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q));
    FS_REQUIRE(p != nullptr && q == cudaDriverEntryPointSuccess, FS_ERR_CUDA,
               "cuTensorMapEncodeTiled is not available from the driver");
    fn = (EncodeTiled)p;
  }
  return fn;
}

CUresult tc::encode_map_2d(CUtensorMap* map, CUtensorMapDataType type, void* base, uint64_t inner,
                          uint64_t outer, uint64_t row_bytes, uint32_t box_inner,
                          uint32_t box_outer, CUtensorMapSwizzle swizzle) {
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return encode_tiled()(map, type, 2, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

void launch_phase_tc(Ctx* ctx, const Space* sa, const Space* sb, void* vec, const PhaseDev& ph,
                     cudaStream_t st) {
  using namespace dct;
  const int nk = sa->norb <= 16 ? 16 : 32;
  const int64_t da = sa->dim, db = sb->dim;
  const int64_t nti = (da + TI - 1) / TI, ntj = (db + TJ - 1) / TJ;
  FS_REQUIRE(phase_tc_supported(FS_C64, sa, sb, vec), FS_ERR_UNSUPPORTED,
             "the TMA pass needs 16-byte aligned rows (an even beta dimension)");
  __nv_bfloat16* occ = (__nv_bfloat16*)scratch(ctx, "dc_occ", (size_t)nti * occ_bytes(nk));
  float2* eaa = (float2*)scratch(ctx, "dc_eaa", (size_t)nti * TI * 8);
  __nv_bfloat16* ypc = (__nv_bfloat16*)scratch(ctx, "dc_y", (size_t)ntj * y_bytes(nk));
  float2* eab = (float2*)scratch(ctx, "dc_eab", (size_t)ntj * TJ * 8);
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)db, (cuuint64_t)da};
  const cuuint64_t strides[1] = {(cuuint64_t)db * 8};
  const cuuint32_t box[2] = {TJ, TI};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_tiled()(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, vec, dims, strides,
                                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  FS_REQUIRE(r == CUDA_SUCCESS, FS_ERR_CUDA, "cuTensorMapEncodeTiled failed for the state");
  {
  ProfScope ps("dc_tables", st, 2);
  k_dc_occ<<<(unsigned)((nti * TI + 127) / 128), 128, 0, st>>>(
      occ, eaa, sa->masks, (const float2*)ph.ea_a, da, nti, nk);
  FS_CUDA(cudaGetLastError());
  k_dc_ypieces<<<(unsigned)((ntj * TJ + 127) / 128), 128, 0, st>>>(
      ypc, eab, sb->masks, (const float2*)ph.ea_b, db, ntj, sa->norb, nk, ph.X);
  FS_CUDA(cudaGetLastError());
  }
  ProfScope ps("phase_tc_f32", st);
  const int sstride = (stage_bytes(nk) + 1023) / 1024 * 1024;
  const size_t smem = (size_t)STAGES * sstride + 1024;
  const int64_t ntiles = nti * ntj;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, 2 * ctx->prop.multiProcessorCount);
  if (nk == 16) {
    FS_CUDA(cudaFuncSetAttribute(k_phase_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    k_phase_tc<16><<<grid, THREADS, smem, st>>>(map, occ, eaa, ypc, eab, nti, ntj,
                                                ctx->d_status);
  } else {
    FS_CUDA(cudaFuncSetAttribute(k_phase_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    k_phase_tc<32><<<grid, THREADS, smem, st>>>(map, occ, eaa, ypc, eab, nti, ntj,
                                                ctx->d_status);
  }
  FS_CUDA(cudaGetLastError());
}

}  // namespace fs
