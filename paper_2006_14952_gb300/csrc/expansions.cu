// Upward and downward translation passes in scaled Cartesian form (Sec. 2.1,
// Eqs. p2m, m2m, l2l):
//   M~_m = M_m / h^|m|,   L~_n = L_n h^(|n|+1),   h = side of the cell.
// With this scaling the M2M and L2L operators are the same on every level.
// (M2L is in m2l.cu.)
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
