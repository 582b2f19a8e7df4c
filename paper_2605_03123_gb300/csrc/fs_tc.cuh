// Tensor-core window steps of the Givens sweeps (tcgen05, sm_103a).
//
// A window step applies the Givens rotations of W adjacent orbitals
// [a, a+W) (§3.2.3).  Their product V (a W x W unitary) acts on the C(W, m)
// strings that share one occupation outside the window (an orbit, m
// electrons inside) as the compound matrix C_m(V)[S', S] = det V[S', S]
// (§2.3: U a^dag_p U^dag = sum_q U_qp a^dag_q applied to the creation
// operators inside the window; the adjacent pairs carry no sign from outside
// orbitals).  So a step is, per class m, one dense product
//     X' = X C_m(V)^T,    X: orbits x C(W, m) amplitudes,
// done here on the tensor cores:
//   * a tile is 128 orbits (rows); each thread gathers its orbit's
//     amplitudes from the shared-memory slab, splits every real part exactly
//     into three BF16 pieces (x = x1 + x2 + x3: x1 = x truncated to 8
//     significant bits, x2 the next 8 of the remainder, x3 the rest, which
//     fits; both subtractions are exact), and stores [x1 | x2 | x3] into its
//     TMEM lane: the A operand (K = 2 C(W, m) reals, re/im interleaved, two
//     BF16 per 32-bit column);
//   * B = the real form of C_m(V) in three BF16 pieces (from FP64), staged
//     per step in shared memory by a bulk copy, K-major, no swizzle: 8-row x
//     16-byte core matrices, LBO = 128 B between core matrices along K, SBO
//     between 8-row groups along N;
//   * D = sum of the six products A_i B_j with i + j <= 4 (pieces 1..3),
//     smallest first, accumulates in TMEM (FP32): the dropped products are
//     below 2^-24 of the result, so a step is as accurate as FP32
//     arithmetic;
//   * each thread reads its lane of D back and scatters the new amplitudes
//     to the slab.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fs {
namespace tc {

constexpr int kW = 6;          // window width of the tensor-core steps
constexpr int kRows = 128;     // MMA tile rows (M)
constexpr int kWg = 4;         // warpgroups per CTA
constexpr int kThreads = kWg * 128;
constexpr int kWgCols = 128;   // TMEM columns per warpgroup
constexpr int kTmemCols = kWg * kWgCols;

constexpr int kPieces = 3;      // BF16 pieces of every operand

__host__ __device__ constexpr int binom6(int m) {
  return m == 0 || m == 6 ? 1 : m == 1 || m == 5 ? 6 : m == 2 || m == 4 ? 15 : 20;
}
// real K (re/im interleaved) and N, padded to the BF16 K step and to 16
__host__ __device__ constexpr int kp(int m) { return (2 * binom6(m) + 15) / 16 * 16; }
__host__ __device__ constexpr int np(int m) { return (2 * binom6(m) + 15) / 16 * 16; }
// bytes of one BF16 piece of the B image of class m
__host__ __device__ constexpr int piece_bytes(int m) { return np(m) * kp(m) * 2; }
// byte offset of class m's image (pieces 1, 2, 3) in a step image
__host__ __device__ constexpr int class_offset(int m) {
  int o = 0;
  for (int k = 1; k < m; ++k) o += kPieces * piece_bytes(k);
  return o;
}
constexpr int kStepBytes = class_offset(kW);   // classes 1 .. W-1
static_assert(kStepBytes % 128 == 0, "step image must stay 128-byte aligned");
// TMEM columns of a tile: the A pieces (two BF16 per column), then D
__host__ __device__ constexpr int a_cols(int m) { return kp(m) / 2; }
static_assert(kPieces * a_cols(3) + np(3) <= kWgCols, "class 3 tile must fit a warpgroup's TMEM");
// byte offset of element (n, k) in a K-major, no-swizzle BF16 piece with K
// padded to kpad
__host__ __device__ inline int b_offset(int n, int k, int kpad) {
  return ((n >> 3) * (kpad >> 3) + (k >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2;
}
// instruction descriptor (kind::f16): D f32, A and B bf16, K-major both, N, M = 128
__host__ __device__ constexpr uint32_t idesc(int m) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(np(m) >> 3) << 17) |
         ((uint32_t)(kRows >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
// Bounded wait for phase `parity` of an mbarrier: about one second of
// clock cycles at most; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > 2000000000ll) return false;
  }
}
// Bulk copy global -> shared (16-byte aligned, multiple of 16 bytes),
// completing `bytes` transactions on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}
// 2-D TMA tile load global -> shared, completing on the mbarrier; x is the
// inner (contiguous) coordinate, x * element size a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
// 2-D TMA tile store shared -> global (bulk group of the issuing thread);
// x, y must not be negative.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(map), "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(slot), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
               "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
      : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&v)[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// D (+)= A B^T with A in TMEM, B in shared memory (descriptor), BF16 in,
// FP32 accumulate; `acc` = 0 overwrites D.
__device__ __forceinline__ void mma_bf16(uint32_t d, uint32_t a, uint64_t b, uint32_t id,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}
__device__ __forceinline__ void wg_bar(int id) {
  asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory");
}
// Exact three-piece BF16 split of a complex amplitude (re, im), packed two
// BF16 per word (re in the low half, k even; im in the high half): each
// piece is the leading 16 bits of the remainder so far (truncation, so the
// subtractions are exact by Sterbenz's lemma, and the last remainder has at
// most 8 significant bits).
__device__ __forceinline__ void split_bf16x3(float re, float im, uint32_t& p1, uint32_t& p2,
                                             uint32_t& p3) {
  const uint32_t ur = __float_as_uint(re), ui = __float_as_uint(im);
  const float r1 = re - __uint_as_float(ur & 0xFFFF0000u);
  const float i1 = im - __uint_as_float(ui & 0xFFFF0000u);
  const uint32_t ur1 = __float_as_uint(r1), ui1 = __float_as_uint(i1);
  const float r2 = r1 - __uint_as_float(ur1 & 0xFFFF0000u);
  const float i2 = i1 - __uint_as_float(ui1 & 0xFFFF0000u);
  p1 = __byte_perm(ur, ui, 0x7632);
  p2 = __byte_perm(ur1, ui1, 0x7632);
  p3 = __byte_perm(__float_as_uint(r2), __float_as_uint(i2), 0x7632);
}

// Host: a 2-D tensor map (inner extent x outer extent elements, rows
// row_bytes apart, boxes box_inner x box_outer) through the driver's
// cuTensorMapEncodeTiled; out-of-range elements of a box read as zeros.
CUresult encode_map_2d(CUtensorMap* map, CUtensorMapDataType type, void* base, uint64_t inner,
                       uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
                       CUtensorMapSwizzle swizzle);

}  // namespace tc
}  // namespace fs
