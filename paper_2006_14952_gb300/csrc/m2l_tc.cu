// M2L with split-precision products on the 5th-generation tensor cores
// (tcgen05, accumulator in tensor memory), the m2l_precision = 1 path.
//
// For one sink A with pairs (A, B_k), Eq. m2l in the scaled, per-pair
// normalised form of m2l.cu is
//   L~_n(A) = sum_k u_k^(|n|+1) v_k^|m| sum_m M~_m(B_k) D^_{n+m}(R^_k)
//           = sum_m P[n+m][m],   P[c][m] = sum_k D'_c(k) M'_m(k),
//   D'_c(k) = u_k^(|c|+1) D^_c(R^_k),   M'_m(k) = (v_k / u_k)^|m| M~_m(B_k),
// a GEMM whose contraction dimension is the sink's pair list.  Each FP32
// operand is split x = hi + lo with hi its TF32 rounding; P accumulates
// hi*hi + hi*lo + lo*hi in FP32 (3xTF32).  Only the entries with |n|+|m| <= p
// of P are used, so at most C(p+6,6) / NC^2 of the tensor work is algorithmic
// (462 / 3136 at p = 5).
//
// CTA = 128 threads, one sink at a time (work counter).  A chunk of 128 pairs:
// thread t computes pair t's D' and M' (generated TCStore bodies) and writes
// them to the K-major, 128-byte-swizzled tiles of warp t/32 (32 pairs = one
// 128-byte row per matrix row); one thread then issues 4 tiles x 4 K-steps x 3
// split products of tcgen05.mma kind::tf32 (M = 128 rows c, N = NCP columns m,
// K = 8) into the sink's TMEM accumulator and commits to an mbarrier.  After
// the last chunk the four warps read their 32 TMEM lanes (rows c), stage P in
// shared memory and thread n forms L~_n = sum_m P[n+m][m].  Waits are bounded;
// on a timeout the kernel records an error and returns after freeing TMEM.
#include "common.cuh"
#include "gen_bodies.cuh"

namespace hfmm {
namespace {

constexpr int kThreads = 128;
constexpr int kChunk = 128;  // pairs per chunk (4 tiles of 32)
constexpr uint32_t kWaitLimit = 1u << 22;

__host__ __device__ constexpr int ncp_of(int p) { return (ncoef(p) + 15) / 16 * 16; }
__host__ __device__ constexpr int tmem_cols_of(int p) {
  return ncp_of(p) <= 32 ? 32 : (ncp_of(p) <= 64 ? 64 : (ncp_of(p) <= 128 ? 128 : 256));
}
// dynamic shared memory: 1 KB alignment slack + A (hi, lo) 4 x 16 KB each + B (hi, lo) 4 x NCP x 128 B each
__host__ __device__ constexpr size_t smem_of(int p) { return 1024 + 2 * 4 * 16384 + 2 * 4 * (size_t)ncp_of(p) * 128; }

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;   // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1u << 46;             // descriptor version
  d |= (uint64_t)2u << 61;             // 128-byte swizzle
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1)
    k_m2l_tc(int64_t nn, const uint4 *__restrict__ cell, const uint32_t *__restrict__ beg,
             const uint32_t *__restrict__ end, const uint64_t *__restrict__ lst, const float *__restrict__ M,
             float *__restrict__ L, int ldm, float inv_rs, unsigned long long *__restrict__ ctr,
             int *__restrict__ status) {
  constexpr int NC = ncoef(P);
  constexpr int NCP = ncp_of(P);
  constexpr uint32_t TCOLS = tmem_cols_of(P);
  constexpr uint32_t IDESC = idesc_tf32(128, NCP);
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ uchar4 mi[kNCMax];
  __shared__ uint32_t next_sink;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float *a_hi = reinterpret_cast<float *>(base);           // 4 tiles x 4096 floats
  float *a_lo = a_hi + 4 * 4096;
  float *b_hi = a_lo + 4 * 4096;                           // 4 tiles x NCP * 32 floats
  float *b_lo = b_hi + 4 * NCP * 32;
  float *pbuf = a_hi;                                      // P staging after a sink's last chunk

  for (int c = tid; c < NC; c += kThreads) {
    int x, y, z;
    mdecode(c, x, y, z);
    mi[c] = make_uchar4((unsigned char)x, (unsigned char)y, (unsigned char)z, (unsigned char)(x + y + z));
  }
  // operand tiles start at zero.  Rows >= NC of B stay zero; rows >= NC of A may
  // later hold the P staging of a finished sink, which only feeds rows of P
  // that are never read.
  for (int i = tid; i < 2 * 4 * 4096 + 2 * 4 * NCP * 32; i += kThreads) a_hi[i] = 0.f;
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

  // this thread's column k within its tile and the swizzled float offsets of that column
  const int kq = tid >> 5, kk = tid & 31;
  int xo[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) xo[j] = (((kk >> 2) ^ j) << 2) + (kk & 3);
  float *my_ahi = a_hi + kq * 4096, *my_alo = a_lo + kq * 4096;
  float *my_bhi = b_hi + kq * NCP * 32, *my_blo = b_lo + kq * NCP * 32;

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
      TCStore<P>::store_d(rx, ry, rz, f, U, my_ahi, my_alo, xo);
      TCStore<P>::store_m(Mb, vr, s, my_bhi, my_blo, xo);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint32_t aoff = (uint32_t)(q * 4096 * 4 + j * 32), boff = (uint32_t)(q * NCP * 32 * 4 + j * 32);
            const uint64_t ah = desc_sw128(smem_u32(a_hi) + aoff), al = desc_sw128(smem_u32(a_lo) + aoff);
            const uint64_t bh = desc_sw128(smem_u32(b_hi) + boff), bl = desc_sw128(smem_u32(b_lo) + boff);
            mma_tf32(tmem, ah, bh, IDESC, (ch | q | j) ? 1u : 0u);
            mma_tf32(tmem, ah, bl, IDESC, 1u);
            mma_tf32(tmem, al, bh, IDESC, 1u);
          }
        }
        mma_commit(mb);
      }
      const bool ok = mbar_wait(mb, phase);
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
  if (abort_flag && tid == 0) mbar_wait(mb, phase ^ 1u);  // give an overdue commit one more bounded wait
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

template <int P>
cudaError_t launch_tc(Ctx &c, cudaStream_t st) {
  const size_t smem = smem_of(P);
  cudaError_t e = cudaFuncSetAttribute(k_m2l_tc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // d_small[5] = work counter, d_small[6] = status word
  unsigned long long *ctr = reinterpret_cast<unsigned long long *>(hfmm::P<uint64_t>(c.d_small) + 5);
  int *status = reinterpret_cast<int *>(hfmm::P<uint64_t>(c.d_small) + 6);
  if ((e = cudaMemsetAsync(ctr, 0, 8, st)) != cudaSuccess) return e;  // the status word is zeroed once per call
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const float inv_rs = (float)(c.prm.box / (double)kHalfBox / c.rs);
  k_m2l_tc<P><<<nsm > 0 ? nsm : 152, kThreads, smem, st>>>(
      c.nnodes, hfmm::P<uint4>(c.cell), hfmm::P<uint32_t>(c.m2l_beg), hfmm::P<uint32_t>(c.m2l_end),
      hfmm::P<uint64_t>(c.m2l), hfmm::P<float>(c.M), hfmm::P<float>(c.L), c.ldm, inv_rs, ctr, status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

bool m2l_tc_supported(int p) { return p >= 1 && p <= 6; }

cudaError_t m2l_pass_tc(Ctx &c, int q, cudaStream_t st) {
  if (c.nm2l == 0 || c.nnodes == 0) return cudaSuccess;
  switch (q) {
    case 1: return launch_tc<1>(c, st);
    case 2: return launch_tc<2>(c, st);
    case 3: return launch_tc<3>(c, st);
    case 4: return launch_tc<4>(c, st);
    case 5: return launch_tc<5>(c, st);
    case 6: return launch_tc<6>(c, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hfmm
