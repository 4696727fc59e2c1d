// hfmm_morton_sort_noalloc: the first steps of hfmm_build_tree (periodic wrap,
// 63-bit Morton keys, stable sort by (key, input index)) for callers that may
// not allocate device memory.  All scratch lives in one file-scope __device__
// array of fixed size, so the call never reaches cudaMalloc or cudaFree.
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

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// x / L: when L is a power of two, x * (1/L) is the same correctly rounded
// quotient (1/L exact), without an FP64 division
__device__ __forceinline__ double div_box(double x, double box, double inv_pow2) {
  return inv_pow2 != 0.0 ? __dmul_rn(x, inv_pow2) : __ddiv_rn(x, box);
}

__device__ __forceinline__ double wrap_box(double x, double box, double inv_pow2) {
  double q = floor(div_box(x, box, inv_pow2));
  return __dsub_rn(x, __dmul_rn(box, q));
}

__device__ __forceinline__ uint32_t grid_coord(double w, double box, double inv_pow2) {
  double t = floor(__dmul_rn(div_box(w, box, inv_pow2), 2097152.0));
  t = fmax(0.0, fmin(t, 2097151.0));
  return (uint32_t)t;
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__global__ void k_keys_noalloc(const double *__restrict__ pos, int64_t n, double box, double inv_pow2,
                               uint64_t *__restrict__ key, uint32_t *__restrict__ idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t k0 = grid_coord(wrap_box(pos[i], box, inv_pow2), box, inv_pow2);
  uint32_t k1 = grid_coord(wrap_box(pos[n + i], box, inv_pow2), box, inv_pow2);
  uint32_t k2 = grid_coord(wrap_box(pos[2 * n + i], box, inv_pow2), box, inv_pow2);
  key[i] = (spread3(k0) << 2) | (spread3(k1) << 1) | spread3(k2);
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
