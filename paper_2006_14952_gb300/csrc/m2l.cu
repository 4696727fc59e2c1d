// M2L on CUDA cores (Eq. m2l with the truncated derivative tensors of Sec. 2.2):
//   L~_n(A) += sum_m M~_m(B) h_B^|m| h_A^(|n|+1) D_{n+m}(R),   R = z_A - z_B',
// evaluated per pair in units of r = |R|:  D_c(R) = r^-(|c|+1) D^_c(R / r), so
//   L~_n(A) += u^(|n|+1) sum_m (v^|m| M~_m(B)) D^_{n+m}(R^),  u = h_A / r, v = h_B / r,
// with |R^| = 1 and u, v <= theta: every factor is O(1) or smaller for any pair
// of levels.  The body forms D'_c = u^(|c|+1) D^_c once per c and takes the
// source coefficients as (v/u)^|m| M~_m, so each term u^(|n|+1) v^|m| D^ M~ is
// one FMA (u >= 2^-17 at the depth cap, so u^(p+1) and (v/u)^p stay in range).  D^ is the derivative tensor of erfc(x r^ / 2) / r^ at r^ = 1,
// x = r / r_s, from the radial prefactors f_(k) = ((1/r) d/dr)^k psi (or of the
// polynomial truncation 1/r - P(r) of Sec. 5 with split 1; radial_prefactors):
//   D^_c = sum_{k_d <= c_d/2} prod_d [c_d! / (2^k_d k_d! (c_d - 2k_d)!)] R^_d^(c_d-2k_d) f_(|c|-|k|).
//
// One lane per (sink, source) pair; a warp walks the pairs of one sink (lists
// are grouped by sink), keeps its partial local expansion in registers and
// reduces it across the warp at the end (through shared memory, in a fixed
// order), so no atomics are used and the result is deterministic.  Each launch adds into L (one launch per order).  The expansion order is a template parameter: all
// index arithmetic is literal in the generated straight-line bodies
// (gen_bodies.py -> gen_bodies.cuh).  For p >= 6 the output coefficients are split
// over G warps (slice g owns the outputs with index = g mod G); for p >= 7 the
// scaled source multipoles of each lane's pair are staged in shared memory.
#include "common.cuh"
#include "gen_bodies.cuh"

namespace hfmm {
namespace {

// Normalised prefactors f^_k = r^(2k+1) f_(k)(r), k = 0..P, of the kernel of
// split S: S = 0 the Gaussian erfc(x/2)/r with x = r / r_s (the recurrence
// f^_(k+1) = -(2k+1) f^_k + (-1)^(k+1) x^(2k+1) e^(-x^2/4) / (2^k sqrt(pi)));
// S = 1 the polynomial truncation 1/r - P(r) with w = r / R_c:
// f^_0 = 1 - w (15 - 10 w^2 + 3 w^4) / 8, f^_1 = -1 + w^3 (5 - 3 w^2) / 2,
// f^_2 = 3 - 3 w^5 and the Newtonian (-1)^k (2k-1)!! beyond.
template <int P, int S>
__device__ __forceinline__ void radial_prefactors(float x, float (&f)[P + 1]) {
  if constexpr (S == 1) {
    const float w = x, w2 = w * w;
    f[0] = 1.f - w * (15.f - 10.f * w2 + 3.f * w2 * w2) * 0.125f;
    if constexpr (P >= 1) f[1] = -1.f + w2 * w * (5.f - 3.f * w2) * 0.5f;
    if constexpr (P >= 2) f[2] = 3.f - 3.f * w2 * w2 * w;
    float dk = 3.f;  // |f^_k| = (2k - 1)!!
#pragma unroll
    for (int q = 3; q <= P; ++q) {
      dk *= (float)(2 * q - 1);
      f[q] = (q & 1) ? -dk : dk;
    }
  } else {
    const float kInvSqrtPi = 0.56418958354775628f;
    f[0] = erfcf(0.5f * x);
    float tk = -x * kInvSqrtPi * __expf(-0.25f * x * x);
    const float hx2 = 0.5f * x * x;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      f[q + 1] = -(float)(2 * q + 1) * f[q] + tk;
      tk = -tk * hx2;
    }
  }
}

template <int P, int G, int g, int S>
__device__ __forceinline__ void m2l_sink(uint32_t k, uint32_t tb, uint32_t te, const uint4 *__restrict__ cell,
                                         const uint64_t *__restrict__ lst, const float *__restrict__ M,
                                         float *__restrict__ L, int ldm, float inv_rs, float *__restrict__ wsm) {
  constexpr int NC = ncoef(P);
  constexpr int NS = (NC + G - 1) / G;
  constexpr bool kSmem = M2LSlices<P>::kSmem;
  const int lane = threadIdx.x & 31;
  const uint4 ca = cell[k];
  float acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.f;
  for (uint32_t t = tb + lane; t < te; t += 32) {
    const uint64_t e = lst[t];
    const uint32_t b = pair_src(e), sh = pair_shift(e);
    const uint4 cb = cell[b];
    int64_t dd[3];
    half_delta(ca, cb, sh, dd);
    // R = z_A - z_B' in half units (exact integers below 2^24)
    const float Rx = -(float)dd[0], Ry = -(float)dd[1], Rz = -(float)dd[2];
    const float r2 = Rx * Rx + Ry * Ry + Rz * Rz;
    const float rinv = rsqrtf(r2);
    const float x = r2 * rinv * inv_rs;  // r / r_s (S = 0) or r / R_c (S = 1)
    const float u = (float)(2 * half_width(ca.w)) * rinv;
    const float v = (float)half_width(cb.w) / (float)half_width(ca.w);  // v/u = h_B / h_A (exact)
    float f[P + 1];
    radial_prefactors<P, S>(x, f);
    float U[P + 1];
    U[0] = u;
#pragma unroll
    for (int q = 1; q <= P; ++q) U[q] = U[q - 1] * u;
    const float *Mb = M + (size_t)b * ldm;
    if constexpr (kSmem) {
      float *col = wsm + lane;
      M2LLoad<P>::template run<32>(Mb, v, col);
      M2LBody<P, G, g>::run(Rx * rinv, Ry * rinv, Rz * rinv, f, U, col, acc);
    } else {
      float Mp[NC];
      M2LLoad<P>::template run<1>(Mb, v, Mp);
      M2LBody<P, G, g>::run(Rx * rinv, Ry * rinv, Rz * rinv, f, U, Mp, acc);
    }
  }
  if constexpr (!kSmem) {
    // sum over the lanes by a transpose in shared memory: each lane writes its
    // partial row (stride NC + 1: no bank conflicts), then lane c adds column c
    // over the 32 rows in lane order (deterministic) and stores it
    static_assert(G == 1, "the transpose path sums whole rows");
#pragma unroll
    for (int s = 0; s < NC; ++s) wsm[lane * (NC + 1) + s] = acc[s];
    __syncwarp();
    for (int cix = lane; cix < NC; cix += 32) {
      float a = 0.f;
#pragma unroll 8
      for (int m = 0; m < 32; ++m) a += wsm[m * (NC + 1) + cix];
      L[(size_t)k * ldm + cix] += a;
    }
    __syncwarp();
  } else {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      float a = acc[s];
#pragma unroll
      for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      const int n = s * G + g;
      if (lane == 0 && n < NC) L[(size_t)k * ldm + n] += a;
    }
  }
}

// resident blocks of 128 threads per SM the register budget allows without
// spilling, by order (measured with -Xptxas -v: p <= 4 at 128, p = 5 at 168 registers)
template <int P>
constexpr int m2l_min_blocks() { return P <= 4 ? 4 : P == 5 ? 3 : 2; }

template <int P, int G, int S>
__global__ void __launch_bounds__(128, m2l_min_blocks<P>()) k_m2l(int64_t nn, const uint4 *__restrict__ cell,
                                             const uint32_t *__restrict__ beg, const uint32_t *__restrict__ end,
                                             const uint64_t *__restrict__ lst, const float *__restrict__ M,
                                             float *__restrict__ L, int ldm, float inv_rs,
                                             const TreeState *tz) {
  extern __shared__ float sm[];
  nn = tree_nodes(tz, nn);  // graph mode: the node count from the device tree state
  // per warp: p >= 7 the staged multipoles (32 x NC), else the reduction transpose (32 x (NC + 1))
  float *wsm = sm + (threadIdx.x >> 5) * (M2LSlices<P>::kSmem ? ncoef(P) * 32 : 32 * (ncoef(P) + 1));
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nn * G; w += nw) {
    const uint32_t k = (uint32_t)(w / G);
    const int g = (int)(w % G);
    const uint32_t tb = beg[k], te = end[k];
    if (tb == te) continue;
    if constexpr (G == 1) {
      m2l_sink<P, 1, 0, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm);
    } else if constexpr (G == 2) {
      if (g == 0) m2l_sink<P, 2, 0, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm);
      else m2l_sink<P, 2, 1, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm);
    } else if constexpr (G == 4) {
      if (g == 0) m2l_sink<P, 4, 0, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm);
      else if (g == 1) m2l_sink<P, 4, 1, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm);
      else if (g == 2) m2l_sink<P, 4, 2, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm);
      else m2l_sink<P, 4, 3, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm);
    } else {
      static_assert(G == 8, "slices");
      switch (g) {
        case 0: m2l_sink<P, 8, 0, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm); break;
        case 1: m2l_sink<P, 8, 1, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm); break;
        case 2: m2l_sink<P, 8, 2, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm); break;
        case 3: m2l_sink<P, 8, 3, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm); break;
        case 4: m2l_sink<P, 8, 4, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm); break;
        case 5: m2l_sink<P, 8, 5, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm); break;
        case 6: m2l_sink<P, 8, 6, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm); break;
        default: m2l_sink<P, 8, 7, S>(k, tb, te, cell, lst, M, L, ldm, inv_rs, wsm); break;
      }
    }
  }
}

template <int P, int S>
cudaError_t launch(Ctx &c, cudaStream_t st) {
  constexpr int G = M2LSlices<P>::G;
  unsigned g = blocks_for((size_t)c.nnodes * G, 4);
  const unsigned cap = 152u * (unsigned)(c.prm.tile_m2l_blocks > 0 ? c.prm.tile_m2l_blocks : 64);
  if (g > cap) g = cap;
  // r / r_s (Gaussian) or r / R_c (polynomial) with r in half units: x = r_half * (L / 2^22) / scale
  const float inv_rs = (float)(c.prm.box / (double)kHalfBox / (S == 1 ? c.rc : c.rs));
  size_t smem = M2LSlices<P>::kSmem ? (size_t)4 * ncoef(P) * 32 * sizeof(float)
                                    : (size_t)4 * 32 * (ncoef(P) + 1) * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_m2l<P, G, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // the entries [mid, end) of each sink: pairs outside the operator table
  k_m2l<P, G, S><<<g, 128, smem, st>>>(c.nnodes, hfmm::P<uint4>(c.cell), hfmm::P<uint32_t>(c.m2l_mid),
                                    hfmm::P<uint32_t>(c.m2l_end), hfmm::P<uint64_t>(c.m2l), hfmm::P<float>(c.M),
                                    hfmm::P<float>(c.L), c.ldm, inv_rs,
                                    c.graph_tree ? hfmm::P<TreeState>(c.tstate) : nullptr);
  note_launch();
  return cudaGetLastError();
}

// M2L on the k-d tree (tree = 1; orders 1..6; split S as in k_m2l): one warp per sink node as in
// k_m2l, with R = c_A - (c_B + s L) formed in FP64 from the box centres and the
// scales h_A, h_B of the two nodes (powers of two: v / u = h_B / h_A is exact).
template <int P, int S>
__global__ void __launch_bounds__(128, m2l_min_blocks<P>()) k_kd_m2l(int64_t nn, const double *__restrict__ geo,
                                                                 int64_t cap, const float *__restrict__ hs,
                                                                 const uint32_t *__restrict__ beg,
                                                                 const uint32_t *__restrict__ end,
                                                                 const uint64_t *__restrict__ lst,
                                                                 const float *__restrict__ M, float *__restrict__ L,
                                                                 int ldm, double box, float inv_rs) {
  constexpr int NC = ncoef(P);
  static_assert(M2LSlices<P>::G == 1 && !M2LSlices<P>::kSmem, "orders 1..6");
  extern __shared__ float sm[];
  float *wsm = sm + (threadIdx.x >> 5) * 32 * (NC + 1);
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < nn; k += nw) {
    const uint32_t tb = beg[k], te = end[k];
    if (tb == te) continue;
    const double ca[3] = {geo[k], geo[cap + k], geo[2 * cap + k]};
    const float hA = hs[k];
    float acc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) acc[q] = 0.f;
    for (uint32_t t = tb + lane; t < te; t += 32) {
      const uint64_t e = lst[t];
      const uint32_t b = pair_src(e), sh = pair_shift(e);
      float R[3];
#pragma unroll
      for (int d = 0; d < 3; ++d)
        R[d] = (float)__dsub_rn(ca[d], __dadd_rn(geo[d * cap + b], (double)shift_component(sh, d) * box));
      const float r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
      const float rinv = rsqrtf(r2);
      float f[P + 1];
      radial_prefactors<P, S>(r2 * rinv * inv_rs, f);
      const float u = hA * rinv;
      float U[P + 1];
      U[0] = u;
#pragma unroll
      for (int q = 1; q <= P; ++q) U[q] = U[q - 1] * u;
      float Mp[NC];
      M2LLoad<P>::template run<1>(M + (size_t)b * ldm, hs[b] / hA, Mp);
      M2LBody<P, 1, 0>::run(R[0] * rinv, R[1] * rinv, R[2] * rinv, f, U, Mp, acc);
    }
    // sum over the lanes in a fixed order (shared-memory transpose, as in k_m2l)
#pragma unroll
    for (int q = 0; q < NC; ++q) wsm[lane * (NC + 1) + q] = acc[q];
    __syncwarp();
    for (int cix = lane; cix < NC; cix += 32) {
      float a = 0.f;
#pragma unroll 8
      for (int m = 0; m < 32; ++m) a += wsm[m * (NC + 1) + cix];
      L[(size_t)k * ldm + cix] += a;
    }
    __syncwarp();
  }
}

template <int P, int S>
cudaError_t launch_kd(Ctx &c, cudaStream_t st) {
  unsigned g = blocks_for((size_t)c.nnodes, 4);
  const unsigned cap = 152u * (unsigned)(c.prm.tile_m2l_blocks > 0 ? c.prm.tile_m2l_blocks : 64);
  if (g > cap) g = cap;
  const size_t smem = (size_t)4 * 32 * (ncoef(P) + 1) * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_kd_m2l<P, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_kd_m2l<P, S><<<g, 128, smem, st>>>(c.nnodes, hfmm::P<double>(c.kd.geo), c.kd.cap, hfmm::P<float>(c.kd.hs),
                                   hfmm::P<uint32_t>(c.m2l_beg), hfmm::P<uint32_t>(c.m2l_end),
                                   hfmm::P<uint64_t>(c.m2l), hfmm::P<float>(c.M), hfmm::P<float>(c.L), c.ldm,
                                   c.prm.box, (float)(1.0 / (S == 1 ? c.rc : c.rs)));
  note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t kd_m2l(Ctx &c, cudaStream_t st) {
  if (c.nm2l == 0 || c.nnodes == 0) return cudaSuccess;
  const bool poly = c.prm.split == 1;
  switch (c.p) {
    case 1: return poly ? launch_kd<1, 1>(c, st) : launch_kd<1, 0>(c, st);
    case 2: return poly ? launch_kd<2, 1>(c, st) : launch_kd<2, 0>(c, st);
    case 3: return poly ? launch_kd<3, 1>(c, st) : launch_kd<3, 0>(c, st);
    case 4: return poly ? launch_kd<4, 1>(c, st) : launch_kd<4, 0>(c, st);
    case 5: return poly ? launch_kd<5, 1>(c, st) : launch_kd<5, 0>(c, st);
    case 6: return poly ? launch_kd<6, 1>(c, st) : launch_kd<6, 0>(c, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t m2l_pass(Ctx &c, int q, cudaStream_t st) {
  if (c.nm2l == 0 || c.nnodes == 0) return cudaSuccess;
  const bool poly = c.prm.split == 1;
  switch (q) {
    case 1: return poly ? launch<1, 1>(c, st) : launch<1, 0>(c, st);
    case 2: return poly ? launch<2, 1>(c, st) : launch<2, 0>(c, st);
    case 3: return poly ? launch<3, 1>(c, st) : launch<3, 0>(c, st);
    case 4: return poly ? launch<4, 1>(c, st) : launch<4, 0>(c, st);
    case 5: return poly ? launch<5, 1>(c, st) : launch<5, 0>(c, st);
    case 6: return poly ? launch<6, 1>(c, st) : launch<6, 0>(c, st);
    case 7: return poly ? launch<7, 1>(c, st) : launch<7, 0>(c, st);
    case 8: return poly ? launch<8, 1>(c, st) : launch<8, 0>(c, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hfmm
