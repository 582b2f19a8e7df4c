// Diagonal-Coulomb evolution for callers that must not allocate device
// memory: callers whose device memory is owned by a pool or arena that the
// library may not bypass, and callers that cannot afford the device-wide
// synchronization a cudaMalloc or cudaFree can cause.  The scratch this
// path needs (string masks and per-string phase factors of both spins) lives
// in one file-scope device array instead of in a context.
#include <cmath>
#include <mutex>

#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

// Largest string dimension per spin this entry point accepts.
constexpr int64_t kNoAllocMaxDim = 16384;
constexpr size_t kNoAllocMasks = kNoAllocMaxDim * sizeof(uint32_t);  // 64 KiB per spin
constexpr size_t kNoAllocFactors = kNoAllocMaxDim * 16;             // 256 KiB per spin
constexpr size_t kNoAllocBytes = 2 * kNoAllocMasks + 2 * kNoAllocFactors;  // 640 KiB

// Every device that loads the library holds this array until the process
// exits.  All calls share it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.  The same first
// call also loads every kernel this entry point launches, so no module
// loads lazily on a later call (for instance inside a stream capture).
static unsigned char* noalloc_scratch_address(int dev) {
  static std::mutex m;
  static unsigned char* addr[256] = {};
  FS_REQUIRE(dev >= 0 && dev < 256, FS_ERR_UNSUPPORTED, "device index above 255");
  std::lock_guard<std::mutex> g(m);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error(std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                cudaGetErrorString(e));
      throw Fail{FS_ERR_CUDA};
    }
    preload_mask_kernel();
    preload_phase_kernels();
    addr[dev] = (unsigned char*)p;
  }
  return addr[dev];
}

// The state must be device memory of the current device: the kernels run
// there, and a pointer into another GPU's memory would be dereferenced
// across devices.  cudaPointerGetAttributes allocates nothing.
static void require_current_device_memory(const void* vec, int dev) {
  cudaPointerAttributes pa;
  const cudaError_t e = cudaPointerGetAttributes(&pa, vec);
  if (e != cudaSuccess) {
    cudaGetLastError();  // not sticky; clear it
    set_error(std::string("the state pointer is not a CUDA pointer: ") + cudaGetErrorString(e));
    throw Fail{FS_ERR_ARG};
  }
  FS_REQUIRE(pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged, FS_ERR_ARG,
             "the state must be device memory");
  FS_REQUIRE(pa.device == dev, FS_ERR_ARG,
             "the state lives on another device than the current one");
}

static int64_t dim_of(int norb, int nocc) { return (int64_t)binom_host(norb, nocc); }

}  // namespace fs

using namespace fs;

extern "C" int fs_apply_diag_coulomb_evolution_noalloc(void* vec, int dtype, const double* J_aa,
                                                       const double* J_ab, const double* J_bb,
                                                       double t, int norb, int n_alpha,
                                                       int n_beta, void* stream) {
  return guarded([&] {
    FS_REQUIRE(dtype == FS_C64 || dtype == FS_C128, FS_ERR_ARG,
               "dtype must be FS_C64 or FS_C128");
    FS_REQUIRE(norb >= 1 && norb <= kMaxNorb, FS_ERR_ARG, "norb must be in [1, 32]");
    FS_REQUIRE(n_alpha >= 0 && n_alpha <= norb && n_beta >= 0 && n_beta <= norb, FS_ERR_ARG,
               "electron counts must be in [0, norb]");
    FS_REQUIRE(vec != nullptr && ((uintptr_t)vec & 15u) == 0, FS_ERR_ARG,
               "state pointer must be non-null and 16-byte aligned");
    FS_REQUIRE(J_aa != nullptr && J_ab != nullptr, FS_ERR_ARG, "null J_aa or J_ab");
    FS_REQUIRE(std::isfinite(t), FS_ERR_ARG, "t must be finite");
    const int64_t da = dim_of(norb, n_alpha), db = dim_of(norb, n_beta);
    FS_REQUIRE(da <= kNoAllocMaxDim && db <= kNoAllocMaxDim, FS_ERR_UNSUPPORTED,
               "fs_apply_diag_coulomb_evolution_noalloc accepts at most 16384 strings per "
               "spin; use fs_apply_diag_coulomb_evolution for larger sectors");
    int dev = 0;
    FS_CUDA(cudaGetDevice(&dev));
    require_current_device_memory(vec, dev);
    current_ctx() = nullptr;  // no tracing on this path
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = noalloc_scratch_address(dev);
    Space sa, sb;
    sa.norb = sb.norb = norb;
    sa.nocc = n_alpha;
    sb.nocc = n_beta;
    sa.dim = da;
    sb.dim = db;
    sa.masks = (uint32_t*)base;
    sb.masks = (uint32_t*)(base + kNoAllocMasks);
    void* fa = base + 2 * kNoAllocMasks;
    void* fb = base + 2 * kNoAllocMasks + kNoAllocFactors;
    launch_masks(sa.masks, norb, n_alpha, st);
    launch_masks(sb.masks, norb, n_beta, st);
    // theta = -(t/2)[sum_{I_a} J_aa + sum_{I_b} J_bb + 2 sum_{p in I_a, q in I_b} J_ab]
    StrPhase pa, pb;
    pa.use_j = pb.use_j = 1;
    pa.t = pb.t = t;
    for (int k = 0; k < norb * norb; ++k) {
      pa.J.v[k] = J_aa[k];
      pb.J.v[k] = (J_bb ? J_bb : J_aa)[k];
    }
    launch_string_phase(&sa, fa, dtype, pa, st);
    launch_string_phase(&sb, fb, dtype, pb, st);
    PhaseDev ph;
    ph.ea_a = fa;
    ph.ea_b = fb;
    ph.has_x = 1;
    for (int k = 0; k < norb * norb; ++k) ph.X.v[k] = -t * J_ab[k];
    launch_phase(&sa, &sb, vec, dtype, ph, st);
  });
}
