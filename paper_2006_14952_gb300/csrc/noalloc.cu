// hfmm_morton_sort_noalloc: the first steps of hfmm_build_tree (periodic wrap,
// 63-bit Morton keys, stable sort by (key, input index)) for callers that may
// not allocate device memory.  All scratch lives in one file-scope __device__
// array of fixed size, so the call never reaches cudaMalloc or cudaFree.
#include <cuda.h>  // driver-API types only; the functions are fetched through the runtime

#include <mutex>

#include "common.cuh"

namespace hfmm {
namespace {

constexpr int64_t kNoAllocMaxN = HFMM_NOALLOC_MAX_N;
constexpr size_t kAltKeyBytes = (size_t)kNoAllocMaxN * sizeof(uint64_t);
constexpr size_t kAltIdxBytes = (size_t)kNoAllocMaxN * sizeof(uint32_t);
// sort histograms / offsets / scan partials for kNoAllocMaxN keys, rounded up
constexpr size_t kSortScratchBytes = (size_t)2 * 256 * ((kNoAllocMaxN + 2047) / 2048) * sizeof(uint32_t) + 4096;
constexpr size_t kScratchBytes = kAltKeyBytes + kAltIdxBytes + kSortScratchBytes;

// Shared by every call on a device; held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The device address of g_noalloc_scratch belongs to the CUDA context that
// loaded this module: another context on the same device (a driver-API
// context, or the primary context re-created after cudaDeviceReset) has its
// own copy.  The address is therefore cached per context, keyed by the
// context's process-unique id (cuCtxGetId), and looked up again for a context
// not seen before.  The two driver functions are fetched through the runtime,
// so the library does not link the driver library itself.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

constexpr int kCacheSlots = 64;
struct ScratchCache {
  std::mutex mu;
  bool resolved = false;
  CtxGetCurrentFn get_current = nullptr;
  CtxGetIdFn get_id = nullptr;
  int used = 0, next = 0;
  unsigned long long id[kCacheSlots] = {};
  void *ptr[kCacheSlots] = {};
};
ScratchCache g_cache;

bool resolve_driver_functions() {
  if (g_cache.resolved) return g_cache.get_current && g_cache.get_id;
  g_cache.resolved = true;
  void *f0 = nullptr, *f1 = nullptr;
  cudaDriverEntryPointQueryResult q0 = cudaDriverEntryPointSymbolNotFound, q1 = q0;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
      cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
      q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess)
    return false;
  g_cache.get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
  g_cache.get_id = reinterpret_cast<CtxGetIdFn>(f1);
  return true;
}

// Id of the current context, 0 when there is none yet.
bool current_context_id(unsigned long long *id) {
  CUcontext ctx = nullptr;
  if (g_cache.get_current(&ctx) != CUDA_SUCCESS) return false;
  *id = 0;
  return !ctx || g_cache.get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_noalloc_scratch in the current context.
cudaError_t scratch_address(void **out) {
  std::lock_guard<std::mutex> lock(g_cache.mu);
  if (!resolve_driver_functions()) return cudaErrorNotSupported;
  unsigned long long id = 0;
  if (!current_context_id(&id)) return cudaErrorContextIsDestroyed;
  for (int i = 0; id && i < g_cache.used; ++i)
    if (g_cache.id[i] == id) {
      *out = g_cache.ptr[i];
      return cudaSuccess;
    }
  // First call in this context: the lookup also makes the runtime's context
  // current when the thread had none (the id is read again below).
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  if (!current_context_id(&id) || !id) return cudaErrorContextIsDestroyed;
  const int slot = g_cache.used < kCacheSlots ? g_cache.used++ : (g_cache.next++ % kCacheSlots);
  g_cache.id[slot] = id;
  g_cache.ptr[slot] = p;
  *out = p;
  return cudaSuccess;
}

__global__ void k_keys_noalloc(const double *__restrict__ pos, int64_t n, double box, double inv_pow2,
                               uint64_t *__restrict__ key, uint32_t *__restrict__ idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  key[i] = morton_key(pos[i], pos[n + i], pos[2 * n + i], box, inv_pow2);
  idx[i] = (uint32_t)i;
}

}  // namespace
}  // namespace hfmm

using namespace hfmm;

extern "C" int hfmm_morton_sort_noalloc(const double *pos_soa, int64_t n, double box, uint64_t *keys_out,
                                        uint32_t *perm_out, void *stream) {
  if (n < 0 || !(box > 0)) return HFMM_ERR_ARG;
  if (n > kNoAllocMaxN) return HFMM_ERR_CAPACITY;
  if (n == 0) return HFMM_OK;
  if (!pos_soa || !keys_out || !perm_out) return HFMM_ERR_ARG;
  // An error left by an earlier call of the caller's stays theirs: report it
  // without launching and without clearing it, so that the launch checks
  // below see this call's own launches only.
  if (cudaPeekAtLastError() != cudaSuccess) return HFMM_ERR_CUDA;
  void *base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return HFMM_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char *sp = static_cast<unsigned char *>(base);
  uint64_t *keys_alt = reinterpret_cast<uint64_t *>(sp);
  uint32_t *idx_alt = reinterpret_cast<uint32_t *>(sp + kAltKeyBytes);
  void *sort_scratch = sp + kAltKeyBytes + kAltIdxBytes;
  k_keys_noalloc<<<blocks_for(n, 256), 256, 0, st>>>(pos_soa, n, box, box_inverse_if_pow2(box), keys_out, perm_out);
  note_launch();
  if (cudaGetLastError() != cudaSuccess) return HFMM_ERR_CUDA;
  bool alt = false;
  if (radix_sort_u64_into(keys_out, perm_out, keys_alt, idx_alt, (size_t)n, 0, 63, &alt, sort_scratch,
                          kSortScratchBytes, st) != cudaSuccess)
    return HFMM_ERR_CUDA;
  if (alt) {  // an odd number of passes would leave the result in the scratch copy
    if (cudaMemcpyAsync(keys_out, keys_alt, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(perm_out, idx_alt, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return HFMM_ERR_CUDA;
  }
  return HFMM_OK;
}
