// M2L through per-(level, offset) operator tables (Eq. m2l with the truncated
// derivative tensors of Sec. 2.2).
//
// Two cells of the same level l (side h) whose centres differ by an integer
// offset o (in cells: z_B' - z_A = o h) interact through an operator that
// depends on (l, o) alone, because the expansion centres are the geometric
// centres.  With the scaled expansions M~ = M / h^|m| and L~ = L h^(|n|+1):
//   L~_n(A) += sum_m T_{n+m} M~_m(B),   T_c = D_c(R) h^(|c|+1),   R = -o h,
// and in units of r = |o| h (the form the per-pair kernel also uses):
//   T_c = |o|^-(|c|+1) D^_c(-o / |o|),   D^ the derivative tensor of
//   erfc(x r^ / 2) / r^ at r^ = 1, x = r / r_s.
// The table holds T_c for |c| <= p at every level 0..21 and every offset with
// |o_d| <= K, K = 2 floor(1/theta) + 1: a pair accepted at level l descends from
// a parent pair that failed the opening-angle test, whose offset is below 1/theta
// in parent cells, and each child centre moves by at most one cell per axis.
// It is computed once per context in FP64 and rounded to FP32.
//
// The table M2L kernel has the layout of the per-pair kernel (one warp per sink,
// one lane per pair, partial expansions reduced across the warp, no atomics)
// but reads T instead of evaluating the prefactors and D^ for every pair.
#include <cmath>

#include "common.cuh"
#include "gen_bodies.cuh"

namespace hfmm {
namespace {

constexpr int kTabLevels = kDepth + 1;  // levels 0..21

__device__ double hco_d(int n, int k) {  // n! / (2^k k! (n - 2k)!)
  double v = 1.0;
  for (int i = n - 2 * k + 1; i <= n; ++i) v *= (double)i;
  for (int i = 1; i <= k; ++i) v /= 2.0 * (double)i;
  return v;
}

// One thread per (level, offset) row: prefactors at unit distance, then every
// derivative component of order <= p by the radial formula of Sec. 2.2:
//   D^_c = sum_{k_d <= c_d/2} prod_d [c_d! / (2^k_d k_d! (c_d - 2 k_d)!)] R^_d^(c_d - 2k_d) f_(|c| - |k|).
__global__ void k_table_build(float *__restrict__ tab, int K, int ld, int p, double box, double rs) {
  const int W = 2 * K + 1;
  const int64_t rows = (int64_t)kTabLevels * W * W * W;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows) return;
  const int oz = (int)(t % W) - K, oy = (int)((t / W) % W) - K, ox = (int)((t / ((int64_t)W * W)) % W) - K;
  const int l = (int)(t / ((int64_t)W * W * W));
  float *row = tab + t * ld;
  const int nc = ncoef(p);
  const double o2 = (double)ox * ox + (double)oy * oy + (double)oz * oz;
  if (o2 == 0.0) {  // coincident centres never reach M2L
    for (int c = 0; c < ld; ++c) row[c] = 0.f;
    return;
  }
  const double on = sqrt(o2);
  const double x = on * ldexp(box, -l) / rs;  // r / r_s
  const double kInvSqrtPi = 0.56418958354775628695;
  double f[kPMax + 1];
  f[0] = erfc(0.5 * x);
  double tk = -x * kInvSqrtPi * exp(-0.25 * x * x);
  const double hx2 = 0.5 * x * x;
  for (int q = 0; q < p; ++q) {
    f[q + 1] = -(double)(2 * q + 1) * f[q] + tk;
    tk = -tk * hx2;
  }
  const double R[3] = {-ox / on, -oy / on, -oz / on};
  double pw[3][kPMax + 1];
  for (int d = 0; d < 3; ++d) {
    pw[d][0] = 1.0;
    for (int j = 1; j <= p; ++j) pw[d][j] = pw[d][j - 1] * R[d];
  }
  const double inv_on = 1.0 / on;
  for (int c = 0; c < ld; ++c) {
    if (c >= nc) {
      row[c] = 0.f;
      continue;
    }
    int cx, cy, cz;
    mdecode(c, cx, cy, cz);
    const int cn = cx + cy + cz;
    double d = 0.0;
    for (int kx = 0; 2 * kx <= cx; ++kx)
      for (int ky = 0; 2 * ky <= cy; ++ky)
        for (int kz = 0; 2 * kz <= cz; ++kz)
          d += hco_d(cx, kx) * hco_d(cy, ky) * hco_d(cz, kz) * pw[0][cx - 2 * kx] * pw[1][cy - 2 * ky] *
               pw[2][cz - 2 * kz] * f[cn - kx - ky - kz];
    double s = inv_on;
    for (int j = 0; j < cn; ++j) s *= inv_on;  // |o|^-(|c|+1)
    row[c] = (float)(d * s);
  }
}

__device__ __forceinline__ int clamp_k(int64_t v, int K) { return v > K ? K : v < -K ? -K : (int)v; }

template <int P, int G, int g>
__device__ __forceinline__ void m2l_tab_sink(uint32_t k, uint32_t tb, uint32_t te, const uint4 *__restrict__ cell,
                                             const uint64_t *__restrict__ lst, const float *__restrict__ M,
                                             float *__restrict__ L, int ldm, const float *__restrict__ tab, int K,
                                             int ld, float *__restrict__ wsm) {
  constexpr int NC = ncoef(P);
  constexpr int NS = (NC + G - 1) / G;
  constexpr bool kSmem = M2LSlices<P>::kSmem;
  const int lane = threadIdx.x & 31;
  const int W = 2 * K + 1;
  const uint4 ca = cell[k];
  const int sh = kDepth + 1 - (int)ca.w;  // log2 of the cell side in half units
  const int64_t lrow = (int64_t)ca.w * W * W * W;
  float acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.f;
  for (uint32_t t = tb + lane; t < te; t += 32) {
    const uint64_t e = lst[t];
    const uint32_t b = pair_src(e);
    int64_t dd[3];
    half_delta(ca, cell[b], pair_shift(e), dd);
    // offset in cells (exact: same level), kept inside the table
    const int ox = clamp_k(dd[0] >> sh, K), oy = clamp_k(dd[1] >> sh, K), oz = clamp_k(dd[2] >> sh, K);
    const float4 *T4 =
        reinterpret_cast<const float4 *>(tab + (lrow + ((int64_t)(ox + K) * W + (oy + K)) * W + (oz + K)) * ld);
    const float *Mb = M + (size_t)b * ldm;
    if constexpr (kSmem) {
      float *col = wsm + lane;
      M2LLoad<P>::template run<32>(Mb, 1.f, col);
      M2LTabBody<P, G, g>::run(T4, col, acc);
    } else {
      float Mp[NC];
      M2LLoad<P>::template run<1>(Mb, 1.f, Mp);
      M2LTabBody<P, G, g>::run(T4, Mp, acc);
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    float a = acc[s];
#pragma unroll
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    const int n = s * G + g;
    if (lane == 0 && n < NC) L[(size_t)k * ldm + n] += a;
  }
}

template <int P, int G>
__global__ void __launch_bounds__(128) k_m2l_tab(int64_t nn, const uint4 *__restrict__ cell,
                                                 const uint32_t *__restrict__ beg, const uint32_t *__restrict__ mid,
                                                 const uint64_t *__restrict__ lst, const float *__restrict__ M,
                                                 float *__restrict__ L, int ldm, const float *__restrict__ tab, int K,
                                                 int ld) {
  extern __shared__ float sm[];
  float *wsm = sm + (threadIdx.x >> 5) * (M2LSlices<P>::kSmem ? ncoef(P) * 32 : 0);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nn * G; w += nw) {
    const uint32_t k = (uint32_t)(w / G);
    const int g = (int)(w % G);
    const uint32_t tb = beg[k], te = mid[k];
    if (tb >= te) continue;
    if constexpr (G == 1) {
      m2l_tab_sink<P, 1, 0>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm);
    } else if constexpr (G == 2) {
      if (g == 0) m2l_tab_sink<P, 2, 0>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm);
      else m2l_tab_sink<P, 2, 1>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm);
    } else if constexpr (G == 4) {
      if (g == 0) m2l_tab_sink<P, 4, 0>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm);
      else if (g == 1) m2l_tab_sink<P, 4, 1>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm);
      else if (g == 2) m2l_tab_sink<P, 4, 2>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm);
      else m2l_tab_sink<P, 4, 3>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm);
    } else {
      static_assert(G == 8, "slices");
      switch (g) {
        case 0: m2l_tab_sink<P, 8, 0>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm); break;
        case 1: m2l_tab_sink<P, 8, 1>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm); break;
        case 2: m2l_tab_sink<P, 8, 2>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm); break;
        case 3: m2l_tab_sink<P, 8, 3>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm); break;
        case 4: m2l_tab_sink<P, 8, 4>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm); break;
        case 5: m2l_tab_sink<P, 8, 5>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm); break;
        case 6: m2l_tab_sink<P, 8, 6>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm); break;
        default: m2l_tab_sink<P, 8, 7>(k, tb, te, cell, lst, M, L, ldm, tab, K, ld, wsm); break;
      }
    }
  }
}

template <int P>
cudaError_t launch(Ctx &c, cudaStream_t st) {
  constexpr int G = M2LTabSlices<P>::G;
  unsigned g = blocks_for((size_t)c.nnodes * G, 4);
  const unsigned cap = 152u * (unsigned)(c.prm.tile_m2l_blocks > 0 ? c.prm.tile_m2l_blocks : 64);
  if (g > cap) g = cap;
  size_t smem = M2LSlices<P>::kSmem ? (size_t)4 * ncoef(P) * 32 * sizeof(float) : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_m2l_tab<P, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_m2l_tab<P, G><<<g, 128, smem, st>>>(c.nnodes, hfmm::P<uint4>(c.cell), hfmm::P<uint32_t>(c.m2l_beg),
                                        hfmm::P<uint32_t>(c.m2l_mid), hfmm::P<uint64_t>(c.m2l), hfmm::P<float>(c.M),
                                        hfmm::P<float>(c.L), c.ldm, hfmm::P<float>(c.tab), c.tab_k, c.tab_ld);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

int m2l_table_extent(const hfmm_params &p) {
  if (!(p.theta > 0)) return 0;
  int k = 2 * (int)std::floor(1.0 / p.theta) + 1;
  if (k > 15) k = 15;
  // keep the table within 256 MB
  const int ld = (ncoef(p.order) + 3) & ~3;
  while (k > 1 && (double)kTabLevels * (2 * k + 1) * (2 * k + 1) * (2 * k + 1) * ld * 4 > 256.0 * (1 << 20)) --k;
  return k;
}

cudaError_t m2l_table_build(Ctx &c, cudaStream_t st) {
  c.tab_ready = false;
  if (c.tab_k <= 0) return cudaSuccess;
  const int W = 2 * c.tab_k + 1;
  c.tab_ld = (ncoef(c.p) + 3) & ~3;
  const int64_t rows = (int64_t)kTabLevels * W * W * W;
  cudaError_t e = ensure(c.tab, (size_t)rows * c.tab_ld * sizeof(float));
  if (e != cudaSuccess) return e;
  k_table_build<<<blocks_for(rows, 128), 128, 0, st>>>(P<float>(c.tab), c.tab_k, c.tab_ld, c.p, c.prm.box, c.rs);
  note_launch();
  e = cudaGetLastError();
  if (e == cudaSuccess) c.tab_ready = true;
  return e;
}

cudaError_t m2l_pass_table(Ctx &c, int q, cudaStream_t st) {
  if (c.nm2l == 0 || c.nnodes == 0 || !c.tab_ready) return cudaSuccess;
  switch (q) {
    case 1: return launch<1>(c, st);
    case 2: return launch<2>(c, st);
    case 3: return launch<3>(c, st);
    case 4: return launch<4>(c, st);
    case 5: return launch<5>(c, st);
    case 6: return launch<6>(c, st);
    case 7: return launch<7>(c, st);
    case 8: return launch<8>(c, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hfmm
