// Helpers shared by the P2P kernels (one-sided p2p.cu, mutual p2p_mutual.cu):
// packed FP32x2 operand pairs, the one-instruction MUFU rsqrt and exp2, and the
// pair-law constants passed as kernel parameters.
#pragma once

#include "common.cuh"

namespace hfmm {
namespace {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// One MUFU instruction each (relative error about 2^-22); the arguments here are
// never denormal: r^2 > 0 in the cut-off range, and the exponent is -r^2 log2(e) / 4r_s^2 >= -7.3.
__device__ __forceinline__ float rsqrt_mufu(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float exp2_mufu(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The pair-factor constants duplicated into (x, x) pairs, the operand form of the
// packed FP32x2 instructions, passed as kernel parameters (no register pairs to fill).
struct PairFit2 {
  float2 c[10];
  float2 nrmid, kexp;  // -R_c / 2, -log2(e) / (4 r_s^2)
  float2 pc0, pc1;     // polynomial split: -5 / (2 R_c^3), 3 / (2 R_c^5)
  float rc2;
};

// The host side of PairFit2 for a context.
inline PairFit2 pair_fit2(const Ctx &c) {
  PairFit2 f;
  for (int j = 0; j < 10; ++j) f.c[j] = make_float2(c.fit.c[j], c.fit.c[j]);
  f.nrmid = make_float2(-c.fit.rmid, -c.fit.rmid);
  f.kexp = make_float2(c.fit.kexp, c.fit.kexp);
  const float pc0 = (float)(-2.5 / (c.rc * c.rc * c.rc)), pc1 = (float)(1.5 / (c.rc * c.rc * c.rc * c.rc * c.rc));
  f.pc0 = make_float2(pc0, pc0);
  f.pc1 = make_float2(pc1, pc1);
  f.rc2 = c.fit.rc2;
  return f;
}

}  // namespace
}  // namespace hfmm
