// Expansion passes in scaled Cartesian form (Sec. 2.1, Eqs. p2m, m2m, m2l, l2l):
//   M~_m = M_m / h^|m|,   L~_n = L_n h^(|n|+1),   h = side of the cell.
// With this scaling the M2M and L2L operators are the same on every level and
// the M2L kernel is a contraction with the derivative tensor of the truncated
// potential erfc(r / 2r_s) / r evaluated in units of the larger cell side.
#include "common.cuh"

namespace hfmm {
namespace {

__device__ __forceinline__ float factf(int k) {
  float f = 1.f;
  for (int i = 2; i <= k; ++i) f *= (float)i;
  return f;
}

__device__ __forceinline__ float powi(float x, int e) {
  float r = 1.f;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// multi-index table in shared memory: {nx, ny, nz, |n|}
__device__ __forceinline__ void build_mi(uchar4 *mi, int nc) {
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    int x, y, z;
    mdecode(c, x, y, z);
    mi[c] = make_uchar4((unsigned char)x, (unsigned char)y, (unsigned char)z, (unsigned char)(x + y + z));
  }
}

__global__ void k_p2m(const uint32_t *__restrict__ leaves, int64_t nl, const uint4 *__restrict__ cell,
                      const uint2 *__restrict__ range, const float4 *__restrict__ pm4, float box, int nc,
                      float *__restrict__ M) {
  __shared__ uchar4 mi[kNCMax];
  build_mi(mi, nc);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nl; t += nw) {
    uint32_t k = leaves[t];
    uint2 r = range[k];
    float inv_h = (float)(1u << cell[k].w) / box;
    for (int c = lane; c < nc; c += 32) {
      uchar4 m = mi[c];
      float s = 0.f;
      for (uint32_t i = r.x; i < r.x + r.y; ++i) {
        float4 q = pm4[i];
        s += q.w * powi(q.x * inv_h, m.x) * powi(q.y * inv_h, m.y) * powi(q.z * inv_h, m.z);
      }
      float coef = ((m.w & 1) ? -1.f : 1.f) / (factf(m.x) * factf(m.y) * factf(m.z));
      M[(size_t)k * nc + c] = coef * s;
    }
  }
}

// M~_m(P) = sum_children sum_{n <= m} (x/H)^n / n! 2^-(|m|-|n|) M~_{m-n}(C),
// x = z_P - z_C = +-H/4 per axis.
__global__ void k_m2m(int64_t lo, int64_t cnt, const uint4 *__restrict__ cell, const int2 *__restrict__ kids, int nc,
                      float *__restrict__ M) {
  __shared__ uchar4 mi[kNCMax];
  build_mi(mi, nc);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < cnt; t += nw) {
    int64_t k = lo + t;
    int2 kd = kids[k];
    if (kd.y == 0) continue;
    for (int c = lane; c < nc; c += 32) {
      uchar4 m = mi[c];
      float acc = 0.f;
      for (int ch = kd.x; ch < kd.x + kd.y; ++ch) {
        uint4 cc = cell[ch];
        float xh[3] = {(cc.x & 1u) ? -0.25f : 0.25f, (cc.y & 1u) ? -0.25f : 0.25f, (cc.z & 1u) ? -0.25f : 0.25f};
        const float *Mc = M + (size_t)ch * nc;
        for (int a = 0; a <= m.x; ++a)
          for (int b = 0; b <= m.y; ++b)
            for (int d = 0; d <= m.z; ++d) {
              int rest = m.w - a - b - d;
              float term = powi(xh[0], a) * powi(xh[1], b) * powi(xh[2], d) /
                           (factf(a) * factf(b) * factf(d)) * ldexpf(1.f, -rest);
              acc += term * Mc[midx(m.x - a, m.y - b, m.z - d)];
            }
      }
      M[(size_t)k * nc + c] = acc;
    }
  }
}

// L~_n(C) += 2^-(|n|+1) sum_{|m| <= p-|n|} (x/H)^m / m! L~_{m+n}(P),  x = z_C - z_P = +-H/4.
__global__ void k_l2l(int64_t lo, int64_t cnt, const uint4 *__restrict__ cell, const int2 *__restrict__ kids, int p,
                      int nc, float *__restrict__ L) {
  __shared__ uchar4 mi[kNCMax];
  build_mi(mi, nc);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < cnt; t += nw) {
    int64_t k = lo + t;
    int2 kd = kids[k];
    if (kd.y == 0) continue;
    const float *Lp = L + (size_t)k * nc;
    for (int ch = kd.x; ch < kd.x + kd.y; ++ch) {
      uint4 cc = cell[ch];
      float xh[3] = {(cc.x & 1u) ? 0.25f : -0.25f, (cc.y & 1u) ? 0.25f : -0.25f, (cc.z & 1u) ? 0.25f : -0.25f};
      for (int c = lane; c < nc; c += 32) {
        uchar4 n = mi[c];
        int rem = p - n.w;
        float s = 0.f;
        for (int e = 0; e < ncoef(rem); ++e) {
          uchar4 m = mi[e];
          s += powi(xh[0], m.x) * powi(xh[1], m.y) * powi(xh[2], m.z) / (factf(m.x) * factf(m.y) * factf(m.z)) *
               Lp[midx(n.x + m.x, n.y + m.y, n.z + m.z)];
        }
        L[(size_t)ch * nc + c] += ldexpf(s, -(n.w + 1));
      }
    }
  }
}

// n! / (2^k k! (n-2k)!)
__device__ __forceinline__ float hcoef(int n, int k) { return factf(n) / (ldexpf(1.f, k) * factf(k) * factf(n - 2 * k)); }

// Generic M2L on CUDA cores, one warp per sink cell, FP32:
//   L~_n(A) += (h_A/h)^(|n|+1) sum_m (h_B/h)^|m| M~_m(B) D^_{n+m}(R / h),   h = max(h_A, h_B),
// with D^ the derivative tensor of erfc(r / 2(r_s/h)) / r (radial form).
__global__ void k_m2l_generic(int64_t nn, const uint4 *__restrict__ cell, const uint32_t *__restrict__ beg,
                              const uint32_t *__restrict__ end, const uint64_t *__restrict__ lst,
                              const float *__restrict__ M, float *__restrict__ L, int p, int nc, float rs_over_box) {
  __shared__ uchar4 mi[kNCMax];
  __shared__ float sM[8][kNCMax];
  __shared__ float sD[8][kNCMax];
  build_mi(mi, nc);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const float kInvSqrtPi = 0.56418958354775628f;
  for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + w; k < nn; k += nw) {
    uint32_t tb = beg[k], te = end[k];
    if (tb == te) continue;
    uint4 ca = cell[k];
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (uint32_t t = tb; t < te; ++t) {
      uint64_t e = lst[t];
      uint32_t b = pair_src(e), s = pair_shift(e);
      uint4 cb = cell[b];
      int64_t dd[3];
      half_delta(ca, cb, s, dd);
      uint32_t lr = ca.w < cb.w ? ca.w : cb.w;  // level of the larger cell
      float inv2w = 1.f / (float)(2 * half_width(lr));
      float R[3] = {-(float)dd[0] * inv2w, -(float)dd[1] * inv2w, -(float)dd[2] * inv2w};
      float sa = ldexpf(1.f, (int)lr - (int)ca.w), sb = ldexpf(1.f, (int)lr - (int)cb.w);
      float rsh = rs_over_box * (float)(1u << lr);
      float r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
      float r = sqrtf(r2), x = r / rsh;
      float f[kPMax + 1];
      f[0] = erfcf(0.5f * x) / r;
      float tk = -expf(-0.25f * x * x) * kInvSqrtPi / rsh;
      float inv2rs2 = 0.5f / (rsh * rsh);
#pragma unroll
      for (int q = 0; q < kPMax; ++q) {
        if (q < p) {
          f[q + 1] = (-(float)(2 * q + 1) * f[q] + tk) / r2;
          tk = -tk * inv2rs2;
        }
      }
      for (int c = lane; c < nc; c += 32) {
        uchar4 n = mi[c];
        float sum = 0.f;
        for (int kx = 0; 2 * kx <= n.x; ++kx)
          for (int ky = 0; 2 * ky <= n.y; ++ky)
            for (int kz = 0; 2 * kz <= n.z; ++kz) {
              float cf = hcoef(n.x, kx) * hcoef(n.y, ky) * hcoef(n.z, kz) * powi(R[0], n.x - 2 * kx) *
                         powi(R[1], n.y - 2 * ky) * powi(R[2], n.z - 2 * kz);
              int o = n.w - kx - ky - kz;
              float fo = f[0];
#pragma unroll
              for (int q = 1; q <= kPMax; ++q)
                if (q == o) fo = f[q];
              sum += cf * fo;
            }
        sD[w][c] = sum;
        sM[w][c] = M[(size_t)b * nc + c] * powi(sb, n.w);
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        int c = lane + 32 * q;
        if (c < nc) {
          uchar4 n = mi[c];
          int rem = p - n.w;
          float sum = 0.f;
          for (int e2 = 0; e2 < ncoef(rem); ++e2) {
            uchar4 m = mi[e2];
            sum += sM[w][e2] * sD[w][midx(n.x + m.x, n.y + m.y, n.z + m.z)];
          }
          acc[q] += sum * powi(sa, n.w + 1);
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      int c = lane + 32 * q;
      if (c < nc) L[(size_t)k * nc + c] += acc[q];
    }
  }
}

}  // namespace

cudaError_t upward(Ctx &c, cudaStream_t st) {
  const int T = 256;
  const float box = (float)c.prm.box;
  if (c.nleaves == 0) return cudaSuccess;
  unsigned g = blocks_for(c.nleaves, 8);
  if (g > 152 * 64) g = 152 * 64;
  k_p2m<<<g, T, 0, st>>>(P<uint32_t>(c.leaves), c.nleaves, P<uint4>(c.cell), P<uint2>(c.range), P<float4>(c.pm4), box,
                         c.nc, P<float>(c.M));
  note_launch();
  for (int l = c.nlevels - 2; l >= 0; --l) {
    int64_t lo = c.level_start[l], cnt = c.level_start[l + 1] - lo;
    unsigned gl = blocks_for(cnt, 8);
    if (gl > 152 * 64) gl = 152 * 64;
    k_m2m<<<gl, T, 0, st>>>(lo, cnt, P<uint4>(c.cell), P<int2>(c.kids), c.nc, P<float>(c.M));
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t m2l_pass(Ctx &c, cudaStream_t st) {
  if (c.nm2l == 0 || c.nnodes == 0) return cudaSuccess;
  const int T = 256;
  unsigned g = blocks_for(c.nnodes, 8);
  if (g > 152 * 32) g = 152 * 32;
  k_m2l_generic<<<g, T, 0, st>>>(c.nnodes, P<uint4>(c.cell), P<uint32_t>(c.m2l_beg), P<uint32_t>(c.m2l_end),
                                 P<uint64_t>(c.m2l), P<float>(c.M), P<float>(c.L), c.p, c.nc,
                                 (float)(c.rs / c.prm.box));
  note_launch();
  return cudaGetLastError();
}

cudaError_t l2l_pass(Ctx &c, cudaStream_t st) {
  const int T = 256;
  for (int l = 0; l + 1 < c.nlevels; ++l) {
    int64_t lo = c.level_start[l], cnt = c.level_start[l + 1] - lo;
    unsigned gl = blocks_for(cnt, 8);
    if (gl > 152 * 64) gl = 152 * 64;
    k_l2l<<<gl, T, 0, st>>>(lo, cnt, P<uint4>(c.cell), P<int2>(c.kids), c.p, c.nc, P<float>(c.L));
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace hfmm
