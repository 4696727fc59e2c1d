// M2L with split-precision products on the 5th-generation tensor cores
// (tcgen05, accumulator in tensor memory): m2l_precision = 1 (3xTF32) and
// m2l_precision = 2 (BF16x3).
//
// For one sink A with pairs (A, B_k), Eq. m2l in the scaled, per-pair
// normalised form of m2l.cu is
//   L~_n(A) = sum_k u_k^(|n|+1) v_k^|m| sum_m M~_m(B_k) D^_{n+m}(R^_k)
//           = sum_m P[n+m][m],   P[c][m] = sum_k D'_c(k) M'_m(k),
//   D'_c(k) = u_k^(|c|+1) D^_c(R^_k),   M'_m(k) = (v_k / u_k)^|m| M~_m(B_k),
// a GEMM whose contraction dimension is the sink's pair list.  Each FP32
// operand is split x = hi + lo, hi its TF32 rounding (kind::tf32, K = 8 per
// instruction) or its BF16 rounding with lo = bf16(x - hi) (kind::f16 with both
// operands BF16, K = 16); P accumulates hi*hi + hi*lo + lo*hi in FP32.  The
// dropped terms are lo*lo and, for BF16, the rounding of lo: about 2^-21
// relative for TF32 and 2^-16 for BF16 per product.  Only the entries with
// |n|+|m| <= p of P are used, so at most C(p+6,6) / NC^2 of the tensor work is
// algorithmic (462 / 3136 at p = 5).
//
// CTA = 128 threads, one sink at a time (work counter).  A chunk of 128 pairs:
// thread t computes pair t's D' and M' (generated TCStore / TCStoreBF bodies)
// and writes them to the K-major, 128-byte-swizzled tiles (one 128-byte row per
// matrix row holds 32 TF32 or 64 BF16 pairs: 4 or 2 tiles per chunk); one
// thread then issues tiles x 4 K-steps x 3 split products of tcgen05.mma
// (M = 128 rows c, N = NCP columns m) into the sink's TMEM accumulator and
// commits to an mbarrier.  After
// the last chunk the four warps read their 32 TMEM lanes (rows c), stage P in
// shared memory and thread n forms L~_n = sum_m P[n+m][m].  Waits are bounded;
// on a timeout the kernel records an error, waits (with the full limit) for the
// MMAs it already issued, and returns after freeing TMEM.
#include <type_traits>

#include "common.cuh"
#include "gen_bodies.cuh"
#include "tc_common.cuh"

namespace hfmm {
namespace {

constexpr int kThreads = 128;
constexpr int kChunk = 128;  // pairs per chunk (4 tiles of 32)
constexpr uint32_t kWaitLimit = 1u << 22;

__host__ __device__ constexpr int ncp_of(int p) { return (ncoef(p) + 15) / 16 * 16; }
__host__ __device__ constexpr int tmem_cols_of(int p) {
  return ncp_of(p) <= 32 ? 32 : (ncp_of(p) <= 64 ? 64 : (ncp_of(p) <= 128 ? 128 : 256));
}
// 128-byte tiles per 128-pair chunk: 32 TF32 or 64 BF16 pairs per row
__host__ __device__ constexpr int tiles_of(bool bf) { return bf ? 2 : 4; }
// dynamic shared memory: 1 KB alignment slack + A (hi, lo) tiles x 16 KB each + B (hi, lo) tiles x NCP x 128 B each
__host__ __device__ constexpr size_t smem_of(int p, bool bf) {
  return 1024 + 2 * (size_t)tiles_of(bf) * 16384 + 2 * (size_t)tiles_of(bf) * ncp_of(p) * 128;
}

template <int P, bool kBF>
__global__ void __launch_bounds__(kThreads, 1)
    k_m2l_tc(int64_t nn, const uint4 *__restrict__ cell, const uint32_t *__restrict__ beg,
             const uint32_t *__restrict__ end, const uint64_t *__restrict__ lst, const float *__restrict__ M,
             float *__restrict__ L, int ldm, float inv_rs, unsigned long long *__restrict__ ctr,
             int *__restrict__ status, uint32_t chunk_wait) {
  constexpr int NC = ncoef(P);
  constexpr int NCP = ncp_of(P);
  constexpr uint32_t TCOLS = tmem_cols_of(P);
  constexpr uint32_t IDESC = kBF ? idesc_bf16(128, NCP) : idesc_tf32(128, NCP);
  constexpr int kTiles = tiles_of(kBF), kPerRow = kChunk / kTiles;  // tiles per chunk, pairs per 128-byte row
  using T = typename std::conditional<kBF, __nv_bfloat16, float>::type;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ uchar4 mi[kNCMax];
  __shared__ uint32_t next_sink;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  T *a_hi = reinterpret_cast<T *>(base);  // kTiles tiles x 128 rows x kPerRow elements (16 KB each)
  T *a_lo = a_hi + kTiles * 128 * kPerRow;
  T *b_hi = a_lo + kTiles * 128 * kPerRow;  // kTiles tiles x NCP rows x kPerRow elements
  T *b_lo = b_hi + kTiles * NCP * kPerRow;
  float *pbuf = reinterpret_cast<float *>(base);  // P staging after a sink's last chunk (NC^2 floats)

  for (int c = tid; c < NC; c += kThreads) {
    int x, y, z;
    mdecode(c, x, y, z);
    mi[c] = make_uchar4((unsigned char)x, (unsigned char)y, (unsigned char)z, (unsigned char)(x + y + z));
  }
  // operand tiles start at zero.  Rows >= NC of B stay zero; rows >= NC of A may
  // later hold the P staging of a finished sink, which only feeds rows of P
  // that are never read.
  {
    uint32_t *w = reinterpret_cast<uint32_t *>(base);
    for (int i = tid; i < (2 * kTiles * 16384 + 2 * kTiles * NCP * 128) / 4; i += kThreads) w[i] = 0u;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    abort_flag = 0;
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
  uint32_t phase = 0;
  const float kInvSqrtPi = 0.56418958354775628f;

  // this thread's column k within its tile and the swizzled element offsets of
  // that column (16-byte chunks XOR the row mod 8 within each 8-row atom)
  const int kq = tid / kPerRow, kk = tid % kPerRow;
  constexpr int kEl = 16 / (int)sizeof(T);  // elements per 16-byte chunk
  int xo[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) xo[j] = (((kk / kEl) ^ j) * kEl) + (kk % kEl);
  T *my_ahi = a_hi + kq * 128 * kPerRow, *my_alo = a_lo + kq * 128 * kPerRow;
  T *my_bhi = b_hi + kq * NCP * kPerRow, *my_blo = b_lo + kq * NCP * kPerRow;

  for (;;) {
    if (tid == 0) {
      uint32_t s = 0xffffffffu;
      for (;;) {  // next sink with M2L pairs
        unsigned long long t = atomicAdd(ctr, 1ull);
        if ((int64_t)t >= nn) break;
        if (end[t] > beg[t]) {
          s = (uint32_t)t;
          break;
        }
      }
      next_sink = s;
    }
    __syncthreads();
    const uint32_t k = next_sink;
    if (k == 0xffffffffu || abort_flag) break;
    const uint4 ca = cell[k];
    const uint32_t tb = beg[k], te = end[k];
    const uint32_t nch = (te - tb + kChunk - 1) / kChunk;
    for (uint32_t ch = 0; ch < nch; ++ch) {
      const uint32_t t = tb + ch * kChunk + tid;
      const bool valid = t < te;
      float rx = 1.f, ry = 0.f, rz = 0.f, x = 1.f, u = 0.f, vr = 0.f, s = 0.f;
      const float *Mb = M;
      if (valid) {
        const uint64_t e = lst[t];
        const uint32_t b = pair_src(e);
        const uint4 cb = cell[b];
        int64_t dd[3];
        half_delta(ca, cb, pair_shift(e), dd);
        const float Rx = -(float)dd[0], Ry = -(float)dd[1], Rz = -(float)dd[2];
        const float r2 = Rx * Rx + Ry * Ry + Rz * Rz;
        const float rinv = rsqrtf(r2);
        rx = Rx * rinv;
        ry = Ry * rinv;
        rz = Rz * rinv;
        x = r2 * rinv * inv_rs;
        u = (float)(2 * half_width(ca.w)) * rinv;
        vr = (float)half_width(cb.w) / (float)half_width(ca.w);  // v / u = h_B / h_A
        s = 1.f;
        Mb = M + (size_t)b * ldm;
      }
      float f[P + 1];
      f[0] = erfcf(0.5f * x);
      float tk = -x * kInvSqrtPi * __expf(-0.25f * x * x);
      const float hx2 = 0.5f * x * x;
#pragma unroll
      for (int q = 0; q < P; ++q) {
        f[q + 1] = -(float)(2 * q + 1) * f[q] + tk;
        tk = -tk * hx2;
      }
      float U[P + 1];
      U[0] = u;
#pragma unroll
      for (int q = 1; q <= P; ++q) U[q] = U[q - 1] * u;
      if constexpr (kBF) {
        TCStoreBF<P>::store_d(rx, ry, rz, f, U, my_ahi, my_alo, xo);
        TCStoreBF<P>::store_m(Mb, vr, s, my_bhi, my_blo, xo);
      } else {
        TCStore<P>::store_d(rx, ry, rz, f, U, my_ahi, my_alo, xo);
        TCStore<P>::store_m(Mb, vr, s, my_bhi, my_blo, xo);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int q = 0; q < kTiles; ++q) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {  // K-steps of 32 bytes: 8 TF32 or 16 BF16 pairs
            const uint32_t aoff = (uint32_t)(q * 16384 + j * 32), boff = (uint32_t)(q * NCP * 128 + j * 32);
            const uint64_t ah = desc_sw128(smem_u32(a_hi) + aoff), al = desc_sw128(smem_u32(a_lo) + aoff);
            const uint64_t bh = desc_sw128(smem_u32(b_hi) + boff), bl = desc_sw128(smem_u32(b_lo) + boff);
            if constexpr (kBF) {
              mma_bf16(tmem, ah, bh, IDESC, (ch | q | j) ? 1u : 0u);
              mma_bf16(tmem, ah, bl, IDESC, 1u);
              mma_bf16(tmem, al, bh, IDESC, 1u);
            } else {
              mma_tf32(tmem, ah, bh, IDESC, (ch | q | j) ? 1u : 0u);
              mma_tf32(tmem, ah, bl, IDESC, 1u);
              mma_tf32(tmem, al, bh, IDESC, 1u);
            }
          }
        }
        mma_commit(mb);
      }
      const bool ok = mbar_wait(mb, phase, chunk_wait);
      phase ^= 1u;
      if (!ok) {
        if (lane == 0) {
          atomicExch(status, 1);
          abort_flag = 1;
        }
      }
      __syncthreads();
      if (abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (abort_flag) break;
    // TMEM rows 32*warp + lane hold P[c][0..NCP); stage rows c < NC
    const int c = warp * 32 + lane;
#pragma unroll
    for (int col = 0; col < NCP; col += 8) {
      float v[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)col, v);
      if (c < NC) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (col + i < NC) pbuf[c * NC + col + i] = v[i];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid < NC) {
      const uchar4 n = mi[tid];
      float acc = 0.f;
      const int rem = ncoef(P - n.w);
      for (int e = 0; e < rem; ++e) {
        const uchar4 m = mi[e];
        acc += pbuf[midx(n.x + m.x, n.y + m.y, n.z + m.z) * NC + e];
      }
      L[(size_t)k * ldm + tid] += acc;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // the MMAs of an abandoned chunk may still be running: wait for them with the
  // full limit before the tensor memory they write is freed
  if (abort_flag && tid == 0) mbar_wait(mb, phase ^ 1u, kWaitLimit);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

template <int P, bool kBF>
cudaError_t launch_tc(Ctx &c, cudaStream_t st) {
  const size_t smem = smem_of(P, kBF);
  cudaError_t e = cudaFuncSetAttribute(k_m2l_tc<P, kBF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // d_small[5] = work counter, d_small[6] = status word
  unsigned long long *ctr = reinterpret_cast<unsigned long long *>(hfmm::P<uint64_t>(c.d_small) + 5);
  int *status = reinterpret_cast<int *>(hfmm::P<uint64_t>(c.d_small) + 6);
  if ((e = cudaMemsetAsync(ctr, 0, 8, st)) != cudaSuccess) return e;  // the status word is zeroed once per call
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const float inv_rs = (float)(c.prm.box / (double)kHalfBox / c.rs);
  k_m2l_tc<P, kBF><<<nsm > 0 ? nsm : 152, kThreads, smem, st>>>(
      c.nnodes, hfmm::P<uint4>(c.cell), hfmm::P<uint32_t>(c.m2l_beg), hfmm::P<uint32_t>(c.m2l_end),
      hfmm::P<uint64_t>(c.m2l), hfmm::P<float>(c.M), hfmm::P<float>(c.L), c.ldm, inv_rs, ctr, status,
      c.prm.tc_wait_polls > 0 ? (uint32_t)c.prm.tc_wait_polls : c.prm.tc_wait_polls < 0 ? 0u : kWaitLimit);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

bool m2l_tc_supported(int p) { return p >= 1 && p <= 6; }

cudaError_t m2l_pass_tc(Ctx &c, int q, cudaStream_t st) {
  if (c.nm2l == 0 || c.nnodes == 0) return cudaSuccess;
  const bool bf = c.prm.m2l_precision == 2;
  switch (q) {
    case 1: return bf ? launch_tc<1, true>(c, st) : launch_tc<1, false>(c, st);
    case 2: return bf ? launch_tc<2, true>(c, st) : launch_tc<2, false>(c, st);
    case 3: return bf ? launch_tc<3, true>(c, st) : launch_tc<3, false>(c, st);
    case 4: return bf ? launch_tc<4, true>(c, st) : launch_tc<4, false>(c, st);
    case 5: return bf ? launch_tc<5, true>(c, st) : launch_tc<5, false>(c, st);
    case 6: return bf ? launch_tc<6, true>(c, st) : launch_tc<6, false>(c, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hfmm
