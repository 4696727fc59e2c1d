// Fused leaf kernel: cut-off P2P over the sink leaf's P2P list (Sec. 2.1, the
// pair force f_(1)(r) r of Sec. 2.2, kept for 0 < r < R_c), plus L2P of the
// leaf's local expansion (Eq. l2p), written straight to the caller's particle
// order (the un-permute).
//
// One warp per sink leaf: lanes 0..15 own up to 16 sink particles, the two
// half-warps walk alternate source particles of each listed source leaf, and
// a shuffle adds the halves.  Offsets are FP32 relative to leaf centres; the
// centre difference of the two leaves is an exact integer in half units.
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

template <bool kCount>
__global__ void __launch_bounds__(256) k_p2p_l2p(const uint32_t *__restrict__ leaves, int64_t nl,
                                                 const uint4 *__restrict__ cell, const uint2 *__restrict__ range,
                                                 const uint32_t *__restrict__ beg, const uint32_t *__restrict__ end,
                                                 const uint64_t *__restrict__ lst, const float4 *__restrict__ pm4,
                                                 const float *__restrict__ L, const uint32_t *__restrict__ perm,
                                                 int64_t n, int p, int nc, float box, float inv_rs, float rc2, float G,
                                                 float *__restrict__ acc_out,
                                                 unsigned long long *__restrict__ useful) {
  __shared__ uchar4 mi[kNCMax];
  uint32_t n_in = 0;  // pairs inside the cut-off (profile mode only)
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    int x, y, z;
    mdecode(c, x, y, z);
    mi[c] = make_uchar4((unsigned char)x, (unsigned char)y, (unsigned char)z, (unsigned char)(x + y + z));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, half = lane >> 4;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const float kInvSqrtPi = 0.56418958354775628f;
  const float half_unit = box / (float)kHalfBox;
  const int ncl = p >= 1 ? ncoef(p - 1) : 0;
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nl; t += nw) {
    uint32_t k = leaves[t];
    uint4 ca = cell[k];
    uint2 r = range[k];
    uint32_t tb = beg[k], te = end[k];
    float inv_h = (float)(1u << ca.w) / box;
    for (uint32_t base = r.x; base < r.x + r.y; base += 16) {
      uint32_t i = base + (lane & 15);
      bool vi = i < r.x + r.y;
      float4 xi = vi ? pm4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      float ax = 0.f, ay = 0.f, az = 0.f;
      for (uint32_t q = tb; q < te; ++q) {
        uint64_t e = lst[q];
        uint32_t b = pair_src(e), s = pair_shift(e);
        uint4 cb = cell[b];
        uint2 rb = range[b];
        int64_t dd[3];
        half_delta(ca, cb, s, dd);
        // sink offset relative to the (shifted) source leaf centre
        float sx = xi.x - (float)dd[0] * half_unit;
        float sy = xi.y - (float)dd[1] * half_unit;
        float sz = xi.z - (float)dd[2] * half_unit;
        for (uint32_t j = rb.x + half; j < rb.x + rb.y; j += 2) {
          float4 xj = pm4[j];
          float dx = sx - xj.x, dy = sy - xj.y, dz = sz - xj.z;
          float r2 = dx * dx + dy * dy + dz * dz;
          bool in = r2 > 0.f && r2 < rc2;
          if (kCount) n_in += (in && vi);
          float r2s = in ? r2 : 1.f;
          float rinv = rsqrtf(r2s);
          float rr = r2s * rinv;
          float xx = rr * inv_rs;
          float S = erfcf(0.5f * xx) + xx * kInvSqrtPi * expf(-0.25f * xx * xx);
          float f = in ? -S * rinv * rinv * rinv * xj.w : 0.f;
          ax += f * dx;
          ay += f * dy;
          az += f * dz;
        }
      }
      ax += __shfl_xor_sync(0xffffffffu, ax, 16);
      ay += __shfl_xor_sync(0xffffffffu, ay, 16);
      az += __shfl_xor_sync(0xffffffffu, az, 16);
      if (lane < 16 && vi) {
        // L2P: a_d = h^-2 sum_{|n| <= p-1} L~_{n+e_d} u^n / n!, u = offset / h
        const float *Lk = L + (size_t)k * nc;
        float ux = xi.x * inv_h, uy = xi.y * inv_h, uz = xi.z * inv_h;
        float lx = 0.f, ly = 0.f, lz = 0.f;
        for (int c = 0; c < ncl; ++c) {
          uchar4 m = mi[c];
          float mono = powi(ux, m.x) * powi(uy, m.y) * powi(uz, m.z) / (factf(m.x) * factf(m.y) * factf(m.z));
          lx += Lk[midx(m.x + 1, m.y, m.z)] * mono;
          ly += Lk[midx(m.x, m.y + 1, m.z)] * mono;
          lz += Lk[midx(m.x, m.y, m.z + 1)] * mono;
        }
        float ih2 = inv_h * inv_h;
        uint32_t o = perm[i];
        acc_out[o] = G * (ax + lx * ih2);
        acc_out[n + o] = G * (ay + ly * ih2);
        acc_out[2 * n + o] = G * (az + lz * ih2);
      }
    }
  }
  if (kCount) {
    unsigned long long v = n_in;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(useful, v);
  }
}

}  // namespace

cudaError_t p2p_l2p(Ctx &c, float *acc, cudaStream_t st) {
  if (c.nleaves == 0) return cudaSuccess;
  const int T = 256;
  unsigned g = blocks_for(c.nleaves, 8);
  if (g > 152 * 16) g = 152 * 16;
  auto kern = c.prm.profile ? k_p2p_l2p<true> : k_p2p_l2p<false>;
  // zeroed by hfmm_short_range_forces before the first phase
  unsigned long long *useful = reinterpret_cast<unsigned long long *>(P<uint64_t>(c.d_small) + 2);
  kern<<<g, T, 0, st>>>(P<uint32_t>(c.leaves), c.nleaves, P<uint4>(c.cell), P<uint2>(c.range), P<uint32_t>(c.p2p_beg),
                        P<uint32_t>(c.p2p_end), P<uint64_t>(c.p2p), P<float4>(c.pm4), P<float>(c.L),
                        P<uint32_t>(c.idx), c.n, c.p, c.nc, (float)c.prm.box, (float)(1.0 / c.rs), (float)(c.rc * c.rc),
                        (float)c.prm.G, acc, useful);
  note_launch();
  return cudaGetLastError();
}

}  // namespace hfmm
