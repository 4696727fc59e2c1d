// Device primitives: buffer growth, exclusive scan and a stable LSD radix sort.
// Used by the tree build (Morton-key sort) and the list grouping by sink.
#include <vector>

#include "common.cuh"

namespace hfmm {

std::atomic<long long> g_launches{0};
thread_local std::vector<void *> *g_deferred_free = nullptr;

cudaError_t ensure(DBuf &b, size_t bytes) {
  if (bytes <= b.cap) return cudaSuccess;
  size_t want = bytes + bytes / 4 + 256;
  if (b.p && g_deferred_free) {  // stream capture in progress: free after it ends
    g_deferred_free->push_back(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  if (b.p) {
    cudaError_t e = cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return e;
  }
  b.cap = want;
  return cudaSuccess;
}

cudaError_t ensure_keep(DBuf &b, size_t bytes, size_t keep, cudaStream_t st) {
  if (bytes <= b.cap) return cudaSuccess;
  size_t want = bytes + bytes / 2 + 256;
  void *np = nullptr;
  cudaError_t e = cudaMalloc(&np, want);
  if (e != cudaSuccess) return e;
  if (b.p && keep) {
    e = cudaMemcpyAsync(np, b.p, keep, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
      cudaFree(np);
      return e;
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaFree(np);
      return e;
    }
  }
  if (b.p) cudaFree(b.p);
  b.p = np;
  b.cap = want;
  return cudaSuccess;
}

void release(DBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

// ------------------------------------------------------------------ scan
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ T block_exclusive_scan(T v, T *total) {
  __shared__ T warp_tot[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    T t = lane < nw ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;  // inclusive
  }
  __syncthreads();
  T base = w ? warp_tot[w - 1] : T(0);
  if (total) *total = warp_tot[(blockDim.x >> 5) - 1];
  T r = base + x - v;
  __syncthreads();
  return r;
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ in, size_t n, uint64_t *__restrict__ bsum) {
  size_t base = (size_t)blockIdx.x * kScanTile;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    size_t j = base + (size_t)i * kScanThreads + threadIdx.x;
    if (j < n) s += in[j];
  }
  uint64_t tot;
  block_exclusive_scan<uint64_t>(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block sums (any count), total at the end.
__global__ void k_scan_bsum(uint64_t *bsum, size_t nb, uint64_t *total) {
  uint64_t carry = 0;
  for (size_t base = 0; base < nb; base += blockDim.x) {
    size_t j = base + threadIdx.x;
    uint64_t v = j < nb ? bsum[j] : 0;
    uint64_t tot;
    uint64_t ex = block_exclusive_scan<uint64_t>(v, &tot);
    if (j < nb) bsum[j] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, size_t n,
                             const uint64_t *__restrict__ bsum) {
  __shared__ uint32_t tile[kScanTile];
  size_t base = (size_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    size_t j = base + (size_t)i * kScanThreads + threadIdx.x;
    tile[i * kScanThreads + threadIdx.x] = j < n ? in[j] : 0u;
  }
  __syncthreads();
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = tile[threadIdx.x * kScanItems + i];
    s += v[i];
  }
  uint32_t ex = block_exclusive_scan<uint32_t>(s, nullptr);
  uint32_t b = (uint32_t)bsum[blockIdx.x] + ex;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    tile[threadIdx.x * kScanItems + i] = b;
    b += v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    size_t j = base + (size_t)i * kScanThreads + threadIdx.x;
    if (j < n) out[j] = tile[i * kScanThreads + threadIdx.x];
  }
}

}  // namespace

cudaError_t scan_u32(const uint32_t *in, uint32_t *out, uint64_t *total, size_t n, DBuf &tmp, cudaStream_t st) {
  size_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) nb = 1;
  cudaError_t e = ensure(tmp, nb * sizeof(uint64_t));
  if (e != cudaSuccess) return e;
  uint64_t *bsum = P<uint64_t>(tmp);
  if (n == 0) return cudaMemsetAsync(total, 0, sizeof(uint64_t), st);
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, bsum);
  note_launch();
  k_scan_bsum<<<1, 1024, 0, st>>>(bsum, nb, total);
  note_launch();
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, bsum);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ radix sort
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;

__global__ void k_radix_hist(const uint64_t *__restrict__ keys, size_t n, int shift, uint32_t mask,
                             uint32_t *__restrict__ counts, unsigned ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  size_t base = (size_t)blockIdx.x * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    size_t j = base + (size_t)r * kSortThreads + threadIdx.x;
    if (j < n) atomicAdd(&h[(uint32_t)(keys[j] >> shift) & mask], 1u);
  }
  __syncthreads();
  counts[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: elements of a tile are ranked in index order (round, warp,
// lane) among equal digits, offset by the tile's exclusive digit base.
template <bool kVals>
__global__ void k_radix_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, size_t n, int shift,
                                uint32_t mask, const uint32_t *__restrict__ offs, unsigned ntiles) {
  __shared__ uint32_t wh[kSortWarps][256];
  __shared__ uint32_t run[256];
  __shared__ uint32_t gbase[256];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  gbase[tid] = offs[(size_t)tid * ntiles + blockIdx.x];
  run[tid] = 0;
  const size_t base = (size_t)blockIdx.x * kSortTile;
  const uint32_t lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortRounds; ++r) {
    size_t j = base + (size_t)r * kSortThreads + tid;
    bool valid = j < n;
    uint64_t key = valid ? kin[j] : 0ull;
    uint32_t val = (kVals && valid) ? vin[j] : 0u;
    uint32_t d = (uint32_t)(key >> shift) & mask;
#pragma unroll
    for (int q = 0; q < kSortWarps; ++q) wh[q][tid] = 0;
    __syncthreads();
    unsigned act = __ballot_sync(0xffffffffu, valid);
    uint32_t rank = 0;
    if (valid) {
      unsigned peers = __match_any_sync(act, d);
      rank = __popc(peers & lt);
      if (rank == 0) wh[w][d] = __popc(peers);
    }
    __syncthreads();
    {
      uint32_t s = run[tid];
#pragma unroll
      for (int q = 0; q < kSortWarps; ++q) {
        uint32_t t = wh[q][tid];
        wh[q][tid] = s;
        s += t;
      }
      run[tid] = s;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = gbase[d] + wh[w][d] + rank;
      kout[pos] = key;
      if (kVals) vout[pos] = val;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, size_t n,
                           int bit_lo, int bit_hi, bool *in_alt, DBuf &tmp, cudaStream_t st) {
  *in_alt = false;
  if (n <= 1 || bit_hi <= bit_lo) return cudaSuccess;
  unsigned ntiles = (unsigned)((n + kSortTile - 1) / kSortTile);
  size_t m = (size_t)256 * ntiles;
  size_t nb = (m + kScanTile - 1) / kScanTile;
  // tmp layout: counts[m] u32 | offs[m] u32 | bsum[nb] u64 | total u64
  size_t bytes = 2 * m * sizeof(uint32_t) + (nb + 2) * sizeof(uint64_t) + 64;
  cudaError_t e = ensure(tmp, bytes);
  if (e != cudaSuccess) return e;
  uint32_t *counts = P<uint32_t>(tmp);
  uint32_t *offs = counts + m;
  uint64_t *total = reinterpret_cast<uint64_t *>(offs + m + (m & 1));
  DBuf scan_tmp;
  scan_tmp.p = total + 1;
  scan_tmp.cap = (nb + 1) * sizeof(uint64_t);
  uint64_t *ka = keys, *kb = keys_alt;
  uint32_t *va = vals, *vb = vals_alt;
  bool alt = false;
  for (int sh = bit_lo; sh < bit_hi; sh += 8) {
    int bits = bit_hi - sh < 8 ? bit_hi - sh : 8;
    uint32_t mask = (1u << bits) - 1u;
    k_radix_hist<<<ntiles, kSortThreads, 0, st>>>(ka, n, sh, mask, counts, ntiles);
    note_launch();
    e = scan_u32(counts, offs, total, m, scan_tmp, st);
    if (e != cudaSuccess) return e;
    if (vals)
      k_radix_scatter<true><<<ntiles, kSortThreads, 0, st>>>(ka, va, kb, vb, n, sh, mask, offs, ntiles);
    else
      k_radix_scatter<false><<<ntiles, kSortThreads, 0, st>>>(ka, nullptr, kb, nullptr, n, sh, mask, offs, ntiles);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint64_t *tk = ka;
    ka = kb;
    kb = tk;
    uint32_t *tv = va;
    va = vb;
    vb = tv;
    alt = !alt;
  }
  *in_alt = alt;
  return cudaSuccess;
}

}  // namespace hfmm

namespace hfmm {

// ------------------------------------------------------------------ caller-provided scratch
// The same scan and sort as above, with every scratch word taken from a
// caller-provided region instead of a growable buffer (nothing is allocated).

size_t radix_sort_scratch_bytes(size_t n) {
  size_t ntiles = (n + kSortTile - 1) / kSortTile;
  size_t m = 256 * ntiles;
  size_t nb = (m + kScanTile - 1) / kScanTile;
  return 2 * m * sizeof(uint32_t) + (nb + 2) * sizeof(uint64_t) + 64;
}

cudaError_t radix_sort_u64_into(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, size_t n,
                                int bit_lo, int bit_hi, bool *in_alt, void *scratch, size_t scratch_bytes,
                                cudaStream_t st) {
  *in_alt = false;
  if (n <= 1 || bit_hi <= bit_lo) return cudaSuccess;
  if (radix_sort_scratch_bytes(n) > scratch_bytes) return cudaErrorInvalidValue;
  unsigned ntiles = (unsigned)((n + kSortTile - 1) / kSortTile);
  size_t m = (size_t)256 * ntiles;
  size_t nb = (m + kScanTile - 1) / kScanTile;
  uint32_t *counts = static_cast<uint32_t *>(scratch);
  uint32_t *offs = counts + m;
  uint64_t *total = reinterpret_cast<uint64_t *>(offs + m + (m & 1));
  uint64_t *bsum = total + 1;
  uint64_t *ka = keys, *kb = keys_alt;
  uint32_t *va = vals, *vb = vals_alt;
  bool alt = false;
  for (int sh = bit_lo; sh < bit_hi; sh += 8) {
    int bits = bit_hi - sh < 8 ? bit_hi - sh : 8;
    uint32_t mask = (1u << bits) - 1u;
    k_radix_hist<<<ntiles, kSortThreads, 0, st>>>(ka, n, sh, mask, counts, ntiles);
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(counts, m, bsum);
    k_scan_bsum<<<1, 1024, 0, st>>>(bsum, nb, total);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, st>>>(counts, offs, m, bsum);
    if (vals)
      k_radix_scatter<true><<<ntiles, kSortThreads, 0, st>>>(ka, va, kb, vb, n, sh, mask, offs, ntiles);
    else
      k_radix_scatter<false><<<ntiles, kSortThreads, 0, st>>>(ka, nullptr, kb, nullptr, n, sh, mask, offs, ntiles);
    note_launch(5);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint64_t *tk = ka;
    ka = kb;
    kb = tk;
    uint32_t *tv = va;
    va = vb;
    vb = tv;
    alt = !alt;
  }
  *in_alt = alt;
  return cudaSuccess;
}

}  // namespace hfmm
