// M2L as a dense contraction per (level, offset) on the tcgen05 tensor cores
// (m2l_precision 3 = 3xTF32, 4 = BF16x3), with the accumulators resident in
// tensor memory.
//
// Because the expansion centres are the geometric centres, a same-level pair
// at level l whose source is displaced from its sink by the integer cell
// offset o interacts through an operator that depends on (l, o) alone
// (Eq. m2l with the truncated derivative tensors of Sec. 2.2):
//   L~_n(A) += sum_m T_{n+m}(l, o) M~_m(B),   |n| + |m| <= p,
// T the per-(level, offset) table of m2l_table.cu.  A CTA owns a tile of 128
// sinks of one level (consecutive in node order); each offset's contribution
// to their 128 x NC local coefficients is formed in tensor memory and added
// to FP32 accumulators in registers (a thread per sink).  It groups its
// sinks' table pairs by offset (a counting sort in shared memory) and, offset
// by offset, forms
//   A = the sources' multipoles in the rows of the sinks that have a pair with
//       that offset (the other rows zero),
//   B = T(l, o) as the K-major matrix B[n][m] = T_{n+m} (zero where
//       |n| + |m| > p),
// and issues D += A B^T as split products (hi*hi + hi*lo + lo*hi).  The
// operator is degree-blocked: the output columns n, ordered by degree, are
// taken in blocks of 16, and block j only runs the K-steps up to the largest
// ncoef(p - |n|) of its columns, so the MMA covers 2432 operator entries at
// p = 6 for the 924 the contraction uses (of 84 x 84).  Nothing is summed
// across CTAs: after the last offset the accumulators are added to the
// sinks' locals, so the result is deterministic.  Pairs outside the table
// (mixed levels, offsets beyond the table's extent) go to the FP32 per-pair
// kernel.  Waits are bounded; on a timeout the kernel records an error,
// waits (with the full limit) for the MMAs it issued, frees its tensor memory
// and returns.
#include <cuda_bf16.h>

#include <type_traits>

#include "common.cuh"
#include "tc_common.cuh"

namespace hfmm {

cudaError_t m2l_pass(Ctx &c, int q, cudaStream_t st);

namespace {

constexpr int kLoThreads = 128;
constexpr int kLoMaxBins = 1331;  // (2K + 1)^3 offsets of the table, K <= 5
constexpr uint32_t kLoWaitLimit = 1u << 22;
constexpr uint32_t kNoSink = 0xffffffffu;

__host__ __device__ constexpr int lo_ncp(int p) { return (ncoef(p) + 15) / 16 * 16; }
// K (input coefficients m) padded to whole 128-byte swizzle atoms: 32 TF32 or 64 BF16 values
__host__ __device__ constexpr int lo_kpad(int p, bool bf) { return bf ? (ncoef(p) + 63) / 64 * 64 : (ncoef(p) + 31) / 32 * 32; }
__host__ __device__ constexpr int lo_chunks(int p, bool bf) { return lo_kpad(p, bf) / (bf ? 64 : 32); }
// dynamic shared memory: 1 KB alignment slack, A (hi, lo) and B (hi, lo) tiles
__host__ __device__ constexpr size_t lo_smem(int p, bool bf) {
  return 1024 + 2 * (size_t)lo_chunks(p, bf) * 128 * 128 + 2 * (size_t)lo_chunks(p, bf) * lo_ncp(p) * 128;
}

// byte offset of element (row, k) in a K-major, 128-byte-swizzled operand of R rows
template <bool kBF>
__device__ __forceinline__ uint32_t sw_off(int R, int row, int k) {
  constexpr int kPerAtom = kBF ? 64 : 32, kEs = kBF ? 2 : 4;
  const int kc = k / kPerAtom, kb = (k % kPerAtom) * kEs;
  const int u = (kb >> 4) ^ (row & 7);
  return (uint32_t)(kc * R * 128 + row * 128 + u * 16 + (kb & 15));
}

template <bool kBF>
__device__ __forceinline__ void split_store(unsigned char *hi, unsigned char *lo, uint32_t off, float x) {
  if constexpr (kBF) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    *reinterpret_cast<__nv_bfloat16 *>(hi + off) = h;
    *reinterpret_cast<__nv_bfloat16 *>(lo + off) = l;
  } else {
    uint32_t hb;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(x));
    const float h = __uint_as_float(hb);
    uint32_t lb;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"(x - h));
    *reinterpret_cast<uint32_t *>(hi + off) = hb;
    *reinterpret_cast<uint32_t *>(lo + off) = lb;
  }
}

template <bool kBF>
__device__ __forceinline__ void zero_store(unsigned char *hi, unsigned char *lo, uint32_t off) {
  if constexpr (kBF) {
    *reinterpret_cast<uint16_t *>(hi + off) = 0;
    *reinterpret_cast<uint16_t *>(lo + off) = 0;
  } else {
    *reinterpret_cast<uint32_t *>(hi + off) = 0u;
    *reinterpret_cast<uint32_t *>(lo + off) = 0u;
  }
}

struct LoLevels {
  int64_t start[kDepth + 3];  // node index of each level's first node (start[nlevels] = nnodes)
  int nlevels;
};

// flag of each node: it has table pairs in this pass
__global__ void k_lo_flags(const uint32_t *__restrict__ beg, const uint32_t *__restrict__ mid, int64_t nn,
                           uint32_t *__restrict__ flag) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nn) flag[k] = mid[k] > beg[k] ? 1u : 0u;
}

// per level: flagged-node rank at the level start and first tile; total tiles
__global__ void k_lo_levels(const uint32_t *__restrict__ rank, const uint64_t *__restrict__ total, LoLevels lv,
                            int64_t nn, uint32_t *__restrict__ meta) {
  if (threadIdx.x != 0) return;
  uint32_t tiles = 0;
  for (int l = 0; l < lv.nlevels; ++l) {
    const int64_t a = lv.start[l], b = lv.start[l + 1];
    const uint32_t ra = a < nn ? rank[a] : (uint32_t)*total, rb = b < nn ? rank[b] : (uint32_t)*total;
    meta[1 + l] = ra;         // rank of the level's first flagged node
    meta[32 + l] = tiles;     // the level's first tile
    tiles += (rb - ra + 127) / 128;
  }
  meta[0] = tiles;
}

// tile and row of each flagged node: tile_sink[tile * 128 + row] = node
__global__ void k_lo_assign(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ rank,
                            const uint4 *__restrict__ cell, int64_t nn, const uint32_t *__restrict__ meta,
                            uint32_t *__restrict__ tile_sink) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nn || !flag[k]) return;
  const uint32_t l = cell[k].w;
  const uint32_t r = rank[k] - meta[1 + l];
  tile_sink[(size_t)(meta[32 + l] + r / 128) * 128 + (r % 128)] = (uint32_t)k;
}

// table pairs of each tile
__global__ void k_lo_tcount(const uint32_t *__restrict__ tile_sink, const uint32_t *__restrict__ beg,
                            const uint32_t *__restrict__ mid, int64_t ntmax, uint32_t *__restrict__ tcnt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntmax) return;
  uint32_t s = 0;
  for (int r = 0; r < 128; ++r) {
    const uint32_t k = tile_sink[(size_t)t * 128 + r];
    if (k != kNoSink) s += mid[k] - beg[k];
  }
  tcnt[t] = s;
}

template <int P, bool kBF>
__global__ void __launch_bounds__(kLoThreads, 1)
    k_m2l_lo(const uint32_t *__restrict__ meta, const uint32_t *__restrict__ tile_sink,
             const uint32_t *__restrict__ toff, const uint32_t *__restrict__ beg, const uint32_t *__restrict__ mid,
             const uint64_t *__restrict__ lst, const uint4 *__restrict__ cell, const float *__restrict__ M,
             float *__restrict__ L, int ldm, const float *__restrict__ tab, int K, int tab_ld,
             unsigned long long *__restrict__ scratch, int *__restrict__ status, uint32_t group_wait) {
  constexpr int NC = ncoef(P), NCP = lo_ncp(P), KC = lo_chunks(P, kBF);
  constexpr int NBLK = NCP / 16;
  constexpr int KI = kBF ? 16 : 8;  // K per instruction
  constexpr uint32_t TCOLS = NCP <= 32 ? 32 : NCP <= 64 ? 64 : NCP <= 128 ? 128 : 256;
  constexpr uint32_t IDESC = kBF ? idesc_bf16(128, 16) : idesc_tf32(128, 16);
  constexpr int kEs = kBF ? 2 : 4;
  const int t = blockIdx.x;
  if (t >= (int)meta[0]) return;  // more CTAs are launched than tiles (no host read-back)
  extern __shared__ unsigned char lo_raw[];
  __shared__ uint32_t hist[kLoMaxBins], cursor[kLoMaxBins];
  __shared__ uint16_t nz_bin[kLoMaxBins];
  __shared__ uint32_t nz_n;
  __shared__ uint32_t trip[924];  // (n, m, c) with |n| + |m| <= p: C(p + 6, 6) <= 924 (p <= 6)
  __shared__ uint32_t ntrip;
  __shared__ uchar4 mi[kNCMax];
  __shared__ uint32_t s_sink[128];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int kstep[8];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char *base = (unsigned char *)(((uintptr_t)lo_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *a_hi = base, *a_lo = base + KC * 128 * 128;
  unsigned char *b_hi = a_lo + KC * 128 * 128, *b_lo = b_hi + KC * NCP * 128;
  const int W = 2 * K + 1, nbins = W * W * W;

  // ---- set-up: operands zero, multi-indices, operator nonzeros, K-steps per block
  {
    uint32_t *w = reinterpret_cast<uint32_t *>(base);
    const int words = (2 * KC * 128 * 128 + 2 * KC * NCP * 128) / 4;
    for (int i = tid; i < words; i += kLoThreads) w[i] = 0u;
  }
  for (int c = tid; c < NC; c += kLoThreads) {
    int x, y, z;
    mdecode(c, x, y, z);
    mi[c] = make_uchar4((unsigned char)x, (unsigned char)y, (unsigned char)z, (unsigned char)(x + y + z));
  }
  for (int i = tid; i < nbins; i += kLoThreads) hist[i] = 0u;
  s_sink[tid] = tile_sink[(size_t)t * 128 + tid];
  if (tid == 0) {
    ntrip = 0;
    nz_n = 0;
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
  }
  __syncthreads();
  for (int idx = tid; idx < NC * NC; idx += kLoThreads) {
    const int n = idx / NC, m = idx % NC;
    const uchar4 a = mi[n], b = mi[m];
    if (a.w + b.w <= P) {
      const int c = midx(a.x + b.x, a.y + b.y, a.z + b.z);
      trip[atomicAdd(&ntrip, 1u)] = (uint32_t)n | ((uint32_t)m << 8) | ((uint32_t)c << 16);
    }
  }
  if (tid < NBLK) {  // block j: output columns 16j..16j+15; K extent ncoef(P - smallest degree)
    const int n0 = 16 * tid;
    const int kmax = n0 < NC ? ncoef(P - (int)mi[n0].w) : 1;
    kstep[tid] = (kmax + KI - 1) / KI;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t mb = smem_u32(&mbar);

  // ---- group the tile's table pairs by offset (counting sort)
  const uint32_t k0 = s_sink[0];
  const uint4 c0 = cell[k0];
  const int sh = kDepth + 1 - (int)c0.w;  // log2 of the cell side in half units
  auto offset_bin = [&](uint4 ca, uint64_t e) -> int {
    int64_t dd[3];
    half_delta(ca, cell[pair_src(e)], pair_shift(e), dd);
    int o[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int64_t v = dd[d] >> sh;
      o[d] = v > K ? K : v < -K ? -K : (int)v;
    }
    return ((o[0] + K) * W + (o[1] + K)) * W + (o[2] + K);
  };
  const uint32_t my = s_sink[tid];
  uint4 my_cell = make_uint4(0, 0, 0, 0);
  uint32_t my_b = 0, my_m = 0;
  if (my != kNoSink) {
    my_cell = cell[my];
    my_b = beg[my];
    my_m = mid[my];
  }
  for (uint32_t e = my_b; e < my_m; ++e) atomicAdd(&hist[offset_bin(my_cell, lst[e])], 1u);
  __syncthreads();
  if (tid == 0) {  // exclusive offsets and the non-empty bins in bin order
    uint32_t acc = 0, nz = 0;
    for (int i = 0; i < nbins; ++i) {
      const uint32_t h = hist[i];
      cursor[i] = acc;
      if (h) nz_bin[nz++] = (uint16_t)i;
      acc += h;
    }
    nz_n = nz;
  }
  __syncthreads();
  unsigned long long *scr = scratch + toff[t];
  for (uint32_t e = my_b; e < my_m; ++e) {
    const uint64_t le = lst[e];
    const uint32_t pos = atomicAdd(&cursor[offset_bin(my_cell, le)], 1u);
    scr[pos] = ((unsigned long long)tid << 32) | (unsigned long long)pair_src(le);
  }
  __syncthreads();
  // cursor[bin] now holds each bin's end; its start is end - hist

  // ---- one contraction per offset in tensor memory, added to FP32 registers
  // (one row per thread) after each offset: a long chain of MMAs accumulating
  // into one tensor-memory element loses precision with its length (measured:
  // 4.6e-5 relative on the locals when all offsets of a tile accumulate in
  // place, against 4.7e-6 for chains of the per-sink kernel's length)
  float racc[NCP];
#pragma unroll
  for (int i = 0; i < NCP; ++i) racc[i] = 0.f;
  const int64_t lrow = (int64_t)c0.w * nbins;
  uint32_t phase = 0;
  const int ngroups = (int)nz_n;
  constexpr int Q4 = (NC + 3) / 4;  // float4 chunks of a multipole row
  for (int g = 0; g < ngroups; ++g) {
    const int bin = nz_bin[g];
    const uint32_t gend = cursor[bin], gcnt = hist[bin], gbeg = gend - gcnt;
    // B: the operator's nonzero entries (positions fixed, values from the table row)
    const float *T = tab + (lrow + bin) * (int64_t)tab_ld;
    for (uint32_t i = tid; i < ntrip; i += kLoThreads) {
      const uint32_t v = trip[i];
      const int n = (int)(v & 255u), m = (int)((v >> 8) & 255u), c = (int)(v >> 16);
      split_store<kBF>(b_hi, b_lo, sw_off<kBF>(NCP, n, m), __ldg(T + c));
    }
    // A: the sources' multipoles in their sinks' rows
    for (uint32_t i = tid; i < gcnt * Q4; i += kLoThreads) {
      const unsigned long long rs = scr[gbeg + i / Q4];
      const int row = (int)(rs >> 32), q = (int)(i % Q4);
      const float4 v = __ldg(reinterpret_cast<const float4 *>(M + (size_t)(uint32_t)rs * ldm) + q);
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (4 * q + j < NC) split_store<kBF>(a_hi, a_lo, sw_off<kBF>(128, row, 4 * q + j), vv[j]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hs = smem_u32(a_hi), a_ls = smem_u32(a_lo), b_hs = smem_u32(b_hi), b_ls = smem_u32(b_lo);
#pragma unroll
      for (int j = 0; j < NBLK; ++j) {
        const int ns = kstep[j];
        for (int s = 0; s < ns; ++s) {
          const int kk = s * KI;                                 // first K of the step
          const int kc = kk / (kBF ? 64 : 32), kb = (kk % (kBF ? 64 : 32)) * kEs;  // atom and byte in it
          const uint32_t aoff = (uint32_t)(kc * 128 * 128 + kb);
          const uint32_t boff = (uint32_t)(kc * NCP * 128 + 16 * j * 128 + kb);
          const uint64_t ah = desc_sw128(a_hs + aoff), al = desc_sw128(a_ls + aoff);
          const uint64_t bh = desc_sw128(b_hs + boff), bl = desc_sw128(b_ls + boff);
          const uint32_t d = tmem + (uint32_t)(16 * j);
          const uint32_t acc0 = s > 0 ? 1u : 0u;  // each offset starts its accumulator afresh
          if constexpr (kBF) {
            mma_bf16(d, ah, bh, IDESC, acc0);
            mma_bf16(d, ah, bl, IDESC, 1u);
            mma_bf16(d, al, bh, IDESC, 1u);
          } else {
            mma_tf32(d, ah, bh, IDESC, acc0);
            mma_tf32(d, ah, bl, IDESC, 1u);
            mma_tf32(d, al, bh, IDESC, 1u);
          }
        }
      }
      mma_commit(mb);
    }
    const bool ok = mbar_wait(mb, phase, group_wait);
    phase ^= 1u;
    if (!ok && lane == 0) {
      atomicExch(status, 1);
      abort_flag = 1;
    }
    __syncthreads();
    if (abort_flag) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int col = 0; col < NCP; col += 8) {
      float v[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)col, v);
#pragma unroll
      for (int i = 0; i < 8; ++i) racc[col + i] += v[i];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    // the rows written for this offset back to zero (the MMAs that read them are done)
    for (uint32_t i = tid; i < gcnt * Q4; i += kLoThreads) {
      const int row = (int)(scr[gbeg + i / Q4] >> 32), q = (int)(i % Q4);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (4 * q + j < NC) zero_store<kBF>(a_hi, a_lo, sw_off<kBF>(128, row, 4 * q + j));
    }
    __syncthreads();
  }
  if (!abort_flag && ngroups > 0) {
    // thread 32 warp + lane holds row (sink) 32 warp + lane: add its coefficients to the locals
    const uint32_t k = s_sink[warp * 32 + lane];
    if (k != kNoSink) {
#pragma unroll
      for (int i = 0; i < NC; ++i) L[(size_t)k * ldm + i] += racc[i];
    }
  }
  // the MMAs of an abandoned offset may still be running: wait for them with the
  // full limit before the tensor memory they write is freed
  if (abort_flag && tid == 0) mbar_wait(mb, phase ^ 1u, kLoWaitLimit);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

template <int P, bool kBF>
cudaError_t launch_lo(Ctx &c, cudaStream_t st, unsigned ntmax, uint32_t *meta, uint32_t *tile_sink,
                      uint32_t *toff, int *status) {
  const size_t smem = lo_smem(P, kBF);
  cudaError_t e = cudaFuncSetAttribute(k_m2l_lo<P, kBF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const uint32_t wait = c.prm.tc_wait_polls > 0 ? (uint32_t)c.prm.tc_wait_polls
                                                : c.prm.tc_wait_polls < 0 ? 0u : kLoWaitLimit;
  k_m2l_lo<P, kBF><<<ntmax, kLoThreads, smem, st>>>(
      meta, tile_sink, toff, hfmm::P<uint32_t>(c.m2l_beg), hfmm::P<uint32_t>(c.m2l_mid), hfmm::P<uint64_t>(c.m2l),
      hfmm::P<uint4>(c.cell), hfmm::P<float>(c.M), hfmm::P<float>(c.L), c.ldm, hfmm::P<float>(c.tab), c.tab_k,
      c.tab_ld, hfmm::P<unsigned long long>(c.lo_scr), status, wait);
  note_launch();
  return cudaGetLastError();
}

template <int P, bool kBF>
struct LoLaunch {
  static cudaError_t run(Ctx &c, cudaStream_t st, unsigned ntmax, uint32_t *meta, uint32_t *ts, uint32_t *to,
                         int *status) {
    return launch_lo<P, kBF>(c, st, ntmax, meta, ts, to, status);
  }
};

}  // namespace

bool m2l_lo_supported(int p) { return p >= 1 && p <= 6; }

// Table pairs of order q through the tensor-core tiles, the others through the
// FP32 per-pair kernel.
cudaError_t m2l_pass_lo(Ctx &c, int q, cudaStream_t st) {
  if (c.nm2l == 0 || c.nnodes == 0) return cudaSuccess;
  cudaError_t e;
#define TRY(x)                      \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) return e; \
  } while (0)
  if (c.tab_ready && c.tab_k > 0 && (2 * c.tab_k + 1) * (2 * c.tab_k + 1) * (2 * c.tab_k + 1) <= kLoMaxBins) {
    const int T = 256;
    const int64_t nn = c.nnodes;
    const unsigned ntmax = (unsigned)(nn / 128 + c.nlevels + 1);
    TRY(ensure(c.lo_flag, (size_t)nn * 4));
    TRY(ensure(c.lo_rank, (size_t)nn * 4));
    TRY(ensure(c.lo_meta, 64 * 4 + 16));
    TRY(ensure(c.lo_sink, (size_t)ntmax * 128 * 4));
    TRY(ensure(c.lo_tcnt, (size_t)ntmax * 4));
    TRY(ensure(c.lo_toff, (size_t)ntmax * 4));
    TRY(ensure(c.lo_scr, (size_t)(c.nm2l > 0 ? c.nm2l : 1) * 8));
    uint32_t *meta = P<uint32_t>(c.lo_meta);
    uint64_t *total = reinterpret_cast<uint64_t *>(meta + 64);
    TRY(cudaMemsetAsync(c.lo_sink.p, 0xff, (size_t)ntmax * 128 * 4, st));
    k_lo_flags<<<blocks_for(nn, T), T, 0, st>>>(P<uint32_t>(c.m2l_beg), P<uint32_t>(c.m2l_mid), nn,
                                                P<uint32_t>(c.lo_flag));
    note_launch();
    TRY(cudaGetLastError());
    TRY(scan_u32(P<uint32_t>(c.lo_flag), P<uint32_t>(c.lo_rank), total, (size_t)nn, c.tmp, st));
    LoLevels lv{};
    lv.nlevels = c.nlevels;
    for (int l = 0; l <= c.nlevels && l < kDepth + 3; ++l) lv.start[l] = c.level_start[l];
    k_lo_levels<<<1, 32, 0, st>>>(P<uint32_t>(c.lo_rank), total, lv, nn, meta);
    k_lo_assign<<<blocks_for(nn, T), T, 0, st>>>(P<uint32_t>(c.lo_flag), P<uint32_t>(c.lo_rank), P<uint4>(c.cell),
                                                 nn, meta, P<uint32_t>(c.lo_sink));
    k_lo_tcount<<<blocks_for(ntmax, T), T, 0, st>>>(P<uint32_t>(c.lo_sink), P<uint32_t>(c.m2l_beg),
                                                    P<uint32_t>(c.m2l_mid), ntmax, P<uint32_t>(c.lo_tcnt));
    note_launch(3);
    TRY(cudaGetLastError());
    TRY(scan_u32(P<uint32_t>(c.lo_tcnt), P<uint32_t>(c.lo_toff), total, ntmax, c.tmp, st));
    int *status = reinterpret_cast<int *>(P<uint64_t>(c.d_small) + 6);
    uint32_t *ts = P<uint32_t>(c.lo_sink), *to = P<uint32_t>(c.lo_toff);
    const bool bf = c.prm.m2l_precision == 4;
    auto go = [&](auto tf, auto bff) -> cudaError_t {
      return bf ? decltype(bff)::run(c, st, ntmax, meta, ts, to, status)
                : decltype(tf)::run(c, st, ntmax, meta, ts, to, status);
    };
    switch (q) {
      case 1: e = go(LoLaunch<1, false>{}, LoLaunch<1, true>{}); break;
      case 2: e = go(LoLaunch<2, false>{}, LoLaunch<2, true>{}); break;
      case 3: e = go(LoLaunch<3, false>{}, LoLaunch<3, true>{}); break;
      case 4: e = go(LoLaunch<4, false>{}, LoLaunch<4, true>{}); break;
      case 5: e = go(LoLaunch<5, false>{}, LoLaunch<5, true>{}); break;
      case 6: e = go(LoLaunch<6, false>{}, LoLaunch<6, true>{}); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  } else {
    // no usable table: every pair through the per-pair kernel from the list start
    TRY(cudaMemcpyAsync(c.m2l_mid.p, c.m2l_beg.p, (size_t)c.nnodes * 4, cudaMemcpyDeviceToDevice, st));
  }
  return m2l_pass(c, q, st);
#undef TRY
}

}  // namespace hfmm
