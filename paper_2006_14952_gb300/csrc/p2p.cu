// Cut-off P2P over each sink leaf's P2P list (Sec. 2.1, the pair force
// f_(1)(r) r of Sec. 2.2, kept for 0 < r < R_c), added to the L2P accelerations
// already in the caller's particle order (the un-permute).
//
// One warp per sink leaf (taken from a global work counter).  The source
// particles of all leaves on the sink's list are streamed through a per-warp
// shared-memory buffer, already translated into the sink leaf's frame (the
// leaf-centre difference is an exact integer in half units).  Lanes are split
// as (sink i, stream s): with cs sinks in the chunk, S = 32 / cs streams walk
// the buffer, so small leaves still keep the warp busy; the streams are added
// in a fixed order at the end (deterministic).
//
// Pair force: a = -m S(x) r / r^3, S(x) = erfc(x/2) + x e^(-x^2/4) / sqrt(pi),
// x = r / r_s, evaluated as S = exp2(-x^2 log2(e) / 4) * Q(r / R_c) with Q a
// degree-9 polynomial interpolating e^(x^2/4) erfc(x/2) + x / sqrt(pi) at
// Chebyshev nodes on [0, R_c] (coefficients from the host, fit_pair_factor()).
#include "common.cuh"

namespace hfmm {
namespace {

constexpr int kCap = 256;  // staged source particles per warp

template <bool kCount>
__global__ void __launch_bounds__(256) k_p2p(const uint32_t *__restrict__ leaves, int64_t nl,
                                             const uint4 *__restrict__ cell, const uint2 *__restrict__ range,
                                             const uint32_t *__restrict__ beg, const uint32_t *__restrict__ end,
                                             const uint64_t *__restrict__ lst, const float4 *__restrict__ pm4,
                                             const uint32_t *__restrict__ perm, int64_t n, float box, PairFit fit,
                                             float G, float *__restrict__ acc_out,
                                             unsigned long long *__restrict__ ctr) {
  __shared__ float4 sbuf[8][kCap];
  const int lane = threadIdx.x & 31;
  float4 *buf = sbuf[threadIdx.x >> 5];
  const float half_unit = box / (float)kHalfBox;
  uint32_t n_in = 0;  // pairs inside the cut-off (profile mode only)
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(ctr, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if ((int64_t)t >= nl) break;
    const uint32_t k = leaves[t];
    const uint4 ca = cell[k];
    const uint2 r = range[k];
    const uint32_t tb = beg[k], te = end[k];
    for (uint32_t cbase = r.x; cbase < r.x + r.y; cbase += 32) {
      const uint32_t rem = r.x + r.y - cbase;
      const int cs = rem < 32 ? (int)rem : 32;
      const int S = 32 / cs, stream = lane / cs, il = lane % cs;
      const bool active = stream < S;
      const float4 xi = pm4[cbase + il];
      float ax = 0.f, ay = 0.f, az = 0.f;
      uint32_t q = tb, jq = 0;
      while (q < te) {
        int fill = 0;
        while (fill < kCap && q < te) {
          const uint32_t qi = q + lane;
          const bool valid = qi < te;
          uint32_t cnt = 0, first = 0;
          float dx = 0.f, dy = 0.f, dz = 0.f;
          if (valid) {
            const uint64_t e = lst[qi];
            const uint32_t b = pair_src(e);
            const uint2 rb = range[b];
            int64_t dd[3];
            half_delta(ca, cell[b], pair_shift(e), dd);
            dx = (float)dd[0] * half_unit;
            dy = (float)dd[1] * half_unit;
            dz = (float)dd[2] * half_unit;
            first = rb.x;
            cnt = rb.y;
          }
          const uint32_t start = lane == 0 ? jq : 0u;
          const uint32_t avail = valid ? cnt - start : 0u;
          uint32_t incl = avail;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          const uint32_t excl = incl - avail;
          const uint32_t room = (uint32_t)(kCap - fill);
          const uint32_t take = excl >= room ? 0u : min(avail, room - excl);
          for (uint32_t j = 0; j < take; ++j) {
            const float4 s4 = pm4[first + start + j];
            buf[fill + excl + j] = make_float4(s4.x + dx, s4.y + dy, s4.z + dz, s4.w);
          }
          const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
          const unsigned full = __ballot_sync(0xffffffffu, valid && incl <= room);
          const int nfull = __popc(full);
          const uint32_t pex = __shfl_sync(0xffffffffu, excl, nfull & 31);
          const uint32_t pstart = nfull == 0 ? jq : 0u;
          const bool partial = nfull < 32 && q + nfull < te;
          jq = partial ? pstart + (pex < room ? room - pex : 0u) : 0u;
          q += nfull;
          fill += (int)(total < room ? total : room);
        }
        __syncwarp();
        if (active) {
          for (int kk = stream; kk < fill; kk += S) {
            const float4 s4 = buf[kk];
            const float dx = xi.x - s4.x, dy = xi.y - s4.y, dz = xi.z - s4.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const bool in = (r2 < fit.rc2) && (r2 > 0.f);
            if (kCount) n_in += in;
            // outside (0, R_c) the value below may be inf/NaN; the select discards it
            const float rinv = rsqrtf(r2);
            const float tt = r2 * rinv * fit.inv_rc;
            float qv = fit.c[9];
#pragma unroll
            for (int j = 8; j >= 0; --j) qv = fmaf(qv, tt, fit.c[j]);
            const float sfac = exp2f(r2 * fit.kexp) * qv;
            const float f = in ? -(sfac * rinv * rinv * rinv) * s4.w : 0.f;
            ax = fmaf(f, dx, ax);
            ay = fmaf(f, dy, ay);
            az = fmaf(f, dz, az);
          }
        }
        __syncwarp();
      }
      // add the streams of each sink in a fixed order
      buf[lane] = make_float4(ax, ay, az, 0.f);
      __syncwarp();
      if (lane < cs) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
        for (int s = 0; s < S; ++s) {
          const float4 v = buf[lane + s * cs];
          sx += v.x;
          sy += v.y;
          sz += v.z;
        }
        const uint32_t o = perm[cbase + lane];
        acc_out[o] += G * sx;
        acc_out[n + o] += G * sy;
        acc_out[2 * n + o] += G * sz;
      }
      __syncwarp();
    }
  }
  if (kCount) {
    unsigned long long v = n_in;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(ctr + 1, v);
  }
}

}  // namespace

cudaError_t p2p_pass(Ctx &c, float *acc, cudaStream_t st) {
  if (c.nleaves == 0) return cudaSuccess;
  const int T = 256;
  unsigned g = 152 * 8;
  if ((size_t)g * 8 > (size_t)c.nleaves) g = blocks_for(c.nleaves, 8);
  auto kern = (c.prm.profile & 2) ? k_p2p<true> : k_p2p<false>;
  // d_small[3] = work counter, d_small[4] = in-cut-off pair count (zeroed earlier when profiling)
  unsigned long long *ctr = reinterpret_cast<unsigned long long *>(P<uint64_t>(c.d_small) + 3);
  cudaError_t e = cudaMemsetAsync(ctr, 0, 8, st);
  if (e != cudaSuccess) return e;
  kern<<<g, T, 0, st>>>(P<uint32_t>(c.leaves), c.nleaves, P<uint4>(c.cell), P<uint2>(c.range), P<uint32_t>(c.p2p_beg),
                        P<uint32_t>(c.p2p_end), P<uint64_t>(c.p2p), P<float4>(c.pm4), P<uint32_t>(c.idx), c.n,
                        (float)c.prm.box, c.fit, (float)c.prm.G, acc, ctr);
  note_launch();
  return cudaGetLastError();
}

}  // namespace hfmm
