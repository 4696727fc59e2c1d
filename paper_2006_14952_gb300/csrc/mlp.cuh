// Learned acceptance network: 12 features -> 64 -> ReLU -> 64 -> ReLU -> 8 logits
// (class 0 = open the pair, class q-1 = accept M2L at expansion order q = 2..8).
// Weights and biases are BF16; inputs and hidden activations are rounded to
// BF16; products are exact in FP32 and sums accumulate in FP32.
//
// Weight blob (BF16, this order): W1[64][12], b1[64], W2[64][64], b2[64],
// W3[8][64], b3[8]  (5512 values).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace hfmm {

constexpr int kMlpIn = 12, kMlpH = 64, kMlpOut = 8;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpH * kMlpIn, kOffW2 = kOffB1 + kMlpH, kOffB2 = kOffW2 + kMlpH * kMlpH,
              kOffW3 = kOffB2 + kMlpH, kOffB3 = kOffW3 + kMlpOut * kMlpH, kMlpW = kOffB3 + kMlpOut;  // 5512

// Shared-memory image of the weights in mma.sync m16n8k16 B-fragment order:
//  layer 1: [8 n-tiles][1 k-tile][2 regs][32 lanes], layer 2: [8][4][2][32], layer 3: [1][4][2][32]
//  (each word = two BF16), then biases as FP32: b1[64], b2[64], b3[8].
constexpr int kFragL1 = 8 * 1 * 2 * 32, kFragL2 = 8 * 4 * 2 * 32, kFragL3 = 1 * 4 * 2 * 32;
constexpr int kMlpSmemWords = kFragL1 + kFragL2 + kFragL3 + kMlpH + kMlpH + kMlpOut;

// Fill the shared image from the BF16 blob (all threads of the block take part).
__device__ __forceinline__ void mlp_stage(const __nv_bfloat16 *__restrict__ w, uint32_t *__restrict__ s) {
  auto pk = [](const __nv_bfloat16 *p, int r, int c0, int ncol, int ld) -> uint32_t {
    const unsigned short lo = c0 < ncol ? __bfloat16_as_ushort(p[r * ld + c0]) : 0;
    const unsigned short hi = c0 + 1 < ncol ? __bfloat16_as_ushort(p[r * ld + c0 + 1]) : 0;
    return (uint32_t)lo | ((uint32_t)hi << 16);
  };
  for (int i = threadIdx.x; i < kFragL1 + kFragL2 + kFragL3; i += blockDim.x) {
    int lane = i & 31, rr = (i >> 5) & 1, rest = i >> 6;
    const int g = lane >> 2, t = lane & 3;
    uint32_t v;
    if (i < kFragL1) {  // rest = n-tile (k-tile 0)
      const int n = rest * 8 + g, k0 = 2 * t + 8 * rr;
      v = pk(w + kOffW1, n, k0, kMlpIn, kMlpIn);
    } else if (i < kFragL1 + kFragL2) {
      const int j = i - kFragL1;
      lane = j & 31;
      rr = (j >> 5) & 1;
      const int kt = (j >> 6) & 3, nt = j >> 8;
      const int n = nt * 8 + ((j & 31) >> 2), k0 = kt * 16 + 2 * (j & 3) + 8 * rr;
      v = pk(w + kOffW2, n, k0, kMlpH, kMlpH);
    } else {
      const int j = i - kFragL1 - kFragL2;
      rr = (j >> 5) & 1;
      const int kt = (j >> 6) & 3;
      const int n = (j & 31) >> 2, k0 = kt * 16 + 2 * (j & 3) + 8 * rr;
      v = pk(w + kOffW3, n, k0, kMlpH, kMlpH);
    }
    s[i] = v;
  }
  float *bias = reinterpret_cast<float *>(s + kFragL1 + kFragL2 + kFragL3);
  for (int i = threadIdx.x; i < kMlpH + kMlpH + kMlpOut; i += blockDim.x) {
    const int o = i < kMlpH ? kOffB1 + i : (i < 2 * kMlpH ? kOffB2 + i - kMlpH : kOffB3 + i - 2 * kMlpH);
    bias[i] = __bfloat162float(w[o]);
  }
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

// One warp evaluates 16 rows.  x: 16 rows x 16 BF16 (features 12..15 zero),
// row stride 16.  On return logits[4] hold (row g, cols 2t, 2t+1) and
// (row g+8, cols 2t, 2t+1), g = lane / 4, t = lane % 4.
__device__ __forceinline__ void mlp_logits16(const uint32_t *__restrict__ s, const __nv_bfloat16 *__restrict__ x,
                                             float (&logits)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const float *bias = reinterpret_cast<const float *>(s + kFragL1 + kFragL2 + kFragL3);
  const uint32_t *xw = reinterpret_cast<const uint32_t *>(x);  // 8 words per row
  uint32_t a[4] = {xw[g * 8 + t], xw[(g + 8) * 8 + t], xw[g * 8 + 4 + t], xw[(g + 8) * 8 + 4 + t]};
  // layer 1
  uint32_t h1[4][4];  // A fragments of layer 2 (4 k-tiles)
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = bias[nt * 8 + 2 * t], b1v = bias[nt * 8 + 2 * t + 1];
    float c[4] = {b0, b1v, b0, b1v};
    mma_bf16_16816(c, a, s[(nt * 2 + 0) * 32 + lane], s[(nt * 2 + 1) * 32 + lane]);
    const uint32_t lo = pack_bf16(fmaxf(c[0], 0.f), fmaxf(c[1], 0.f));
    const uint32_t hi = pack_bf16(fmaxf(c[2], 0.f), fmaxf(c[3], 0.f));
    h1[nt >> 1][(nt & 1) * 2 + 0] = lo;
    h1[nt >> 1][(nt & 1) * 2 + 1] = hi;
  }
  // layer 2
  const uint32_t *s2 = s + kFragL1;
  uint32_t h2[4][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = bias[kMlpH + nt * 8 + 2 * t], b1v = bias[kMlpH + nt * 8 + 2 * t + 1];
    float c[4] = {b0, b1v, b0, b1v};
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      const uint32_t af[4] = {h1[kt][0], h1[kt][1], h1[kt][2], h1[kt][3]};
      mma_bf16_16816(c, af, s2[((nt * 4 + kt) * 2 + 0) * 32 + lane], s2[((nt * 4 + kt) * 2 + 1) * 32 + lane]);
    }
    h2[nt >> 1][(nt & 1) * 2 + 0] = pack_bf16(fmaxf(c[0], 0.f), fmaxf(c[1], 0.f));
    h2[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16(fmaxf(c[2], 0.f), fmaxf(c[3], 0.f));
  }
  // layer 3
  const uint32_t *s3 = s + kFragL1 + kFragL2;
  const float b0 = bias[2 * kMlpH + 2 * t], b1v = bias[2 * kMlpH + 2 * t + 1];
  float c[4] = {b0, b1v, b0, b1v};
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) {
    const uint32_t af[4] = {h2[kt][0], h2[kt][1], h2[kt][2], h2[kt][3]};
    mma_bf16_16816(c, af, s3[(kt * 2 + 0) * 32 + lane], s3[(kt * 2 + 1) * 32 + lane]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) logits[i] = c[i];
}

// Argmax over the 8 logits of rows g and g+8 (ties: lowest class); every lane
// of the quad receives both results.
__device__ __forceinline__ void mlp_argmax16(const float (&l)[4], int &cls_g, int &cls_g8) {
  const int t = threadIdx.x & 3;
  float v0 = l[0], v8 = l[2];
  int i0 = 2 * t, i8 = 2 * t;
  if (l[1] > v0) { v0 = l[1]; i0 = 2 * t + 1; }
  if (l[3] > v8) { v8 = l[3]; i8 = 2 * t + 1; }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    const float w0 = __shfl_xor_sync(0xffffffffu, v0, o), w8 = __shfl_xor_sync(0xffffffffu, v8, o);
    const int j0 = __shfl_xor_sync(0xffffffffu, i0, o), j8 = __shfl_xor_sync(0xffffffffu, i8, o);
    if (w0 > v0 || (w0 == v0 && j0 < i0)) { v0 = w0; i0 = j0; }
    if (w8 > v8 || (w8 == v8 && j8 < i8)) { v8 = w8; i8 = j8; }
  }
  cls_g = i0;
  cls_g8 = i8;
}

// ---------------------------------------------------------------- features
// Pair features (all dimensionless, half units for lengths): 0 S_c/r_s,
// 1 S_m/r_s, 2 S_max/R_c, 3 h_A/S_c, 4 h_B/S_c, 5 max(h_A,h_B)/S_c,
// 6 (level_A - level_B)/8, 7 log2(1+n_A)/16, 8 log2(1+n_B)/16,
// 9 |dipole of B| / |monopole|, 10 |quadrupole of B| / |monopole| (scaled
// multipoles M~ = M / h^|m|), 11 S_c/R_c.
__device__ __forceinline__ void pair_features(uint4 ca, uint4 cb, uint32_t s, uint32_t na, uint32_t nb,
                                              const float *__restrict__ Mb, float inv_rs_h, float inv_rc_h,
                                              float *f) {
  int64_t dd[3];
  half_delta(ca, cb, s, dd);
  const int64_t wa = half_width(ca.w), wb = half_width(cb.w), ext = wa + wb;
  float sc2 = 0.f, sm2 = 0.f, sx2 = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int64_t a = dd[d] < 0 ? -dd[d] : dd[d];
    const int64_t gp = a - ext > 0 ? a - ext : 0;
    const float fa = (float)a, fg = (float)gp, fx = (float)(a + ext);
    sc2 += fa * fa;
    sm2 += fg * fg;
    sx2 += fx * fx;
  }
  const float sc = sqrtf(sc2), sm = sqrtf(sm2), sx = sqrtf(sx2);
  const float ha = (float)(2 * wa), hb = (float)(2 * wb);
  const float isc = 1.f / sc;
  f[0] = sc * inv_rs_h;
  f[1] = sm * inv_rs_h;
  f[2] = sx * inv_rc_h;
  f[3] = ha * isc;
  f[4] = hb * isc;
  f[5] = fmaxf(ha, hb) * isc;
  f[6] = ((float)ca.w - (float)cb.w) * 0.125f;
  f[7] = __log2f(1.f + (float)na) * 0.0625f;
  f[8] = __log2f(1.f + (float)nb) * 0.0625f;
  const float m0 = fabsf(Mb[0]) + 1e-30f;
  f[9] = sqrtf(Mb[1] * Mb[1] + Mb[2] * Mb[2] + Mb[3] * Mb[3]) / m0;
  float q2 = 0.f;
#pragma unroll
  for (int c = 4; c < 10; ++c) q2 += Mb[c] * Mb[c];
  f[10] = sqrtf(q2) / m0;
  f[11] = sc * inv_rc_h;
}

}  // namespace hfmm
