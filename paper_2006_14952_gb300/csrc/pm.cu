// Long-range (PM) accelerations of the force split of Sec. 2.2, and the
// kick-drift-kick step (the synchronised global step of Sec. 4).
//
// The long-range pair potential erf(r / 2r_s) / r has the Fourier transform
// 4 pi exp(-k^2 r_s^2) / k^2.  With the mass m_g assigned to the mesh points
// x_g = g L / N_g by cloud-in-cell (CIC) weights:
//   a(k) = i k G 4 pi exp(-k^2 r_s^2) / (k^2 W(k)^2) m(k) / L^3,
//   W(k) = prod_d sinc^2(k_d L / 2N_g)   (the CIC window of the assignment and
//                                         of the interpolation, divided out),
// zero at k = 0 and on the Nyquist plane of each gradient component; the mesh
// acceleration is the inverse transform (the Fourier series sums the modes, so
// the unnormalised inverse FFT is the right scaling) and is interpolated back to
// the particles with the same CIC weights.  Sign convention: a = G grad Phi,
// Phi = sum_j m_j psi(x - x_j), as for the short-range pair force.
//
// The mass assignment accumulates 64-bit fixed-point integers (mass * weight *
// 2^s, s chosen from N * max|m| so no sum can overflow; the weights in FP32
// from FP64 cell offsets), so the mesh, and with it every acceleration, is the
// same on every run whatever order the atomics land in.  Mesh transforms use cuFFT (FP32, one R2C and a batch of three C2R).
#include <cufft.h>

#include <cmath>
#include <vector>

#include "common.cuh"

namespace hfmm {
namespace {

__global__ void k_mass_absmax(const float4 *__restrict__ pm4, int64_t n, unsigned *__restrict__ out) {
  unsigned v = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v = max(v, __float_as_uint(fabsf(pm4[i].w)));  // non-negative floats order like their bit patterns
  for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v) atomicMax(out, v);
}

// Fixed-point scale 2^s with N * max|m| * 2^s <= 2^61 (its exponent s).
__device__ __forceinline__ int fixed_exponent(const unsigned *mmax_bits, int64_t n) {
  const double bound = (double)__uint_as_float(*mmax_bits) * (double)n;
  if (!(bound > 0)) return 0;
  int e;
  frexp(bound, &e);  // bound < 2^e
  return 61 - e;
}

// Mesh cell and offset of one coordinate when N_g / L = 2^tm_exp exactly: u =
// x 2^tm_exp = 1.f 2^s, floor(u) is the 53-bit significand shifted right by
// 52 - s and u - floor(u) the bits shifted out, converted to FP32 (one correct
// rounding, as of the exact FP64 difference) -- no FP64 arithmetic (this GPU's
// FP64 rate is low).  False, with nothing computed, outside [0, L) (x = L after
// a wrap that rounded up), for x below 2^-120 or u below 2^-100 (but not zero),
// or u above 2^51.
__device__ __forceinline__ bool cic_bits(double x, double box, int tm_exp, int &c, float &d) {
  const long long b = __double_as_longlong(x);
  if (b < 0 || b >= __double_as_longlong(box)) return false;
  if (b == 0) {
    c = 0;
    d = 0.f;
    return true;
  }
  const int ex = (int)((b >> 52) & 0x7ff) - 1023, s = ex + tm_exp;
  if (ex < -120 || s < -100 || s > 51) return false;
  if (s < 0) {  // u < 1: the offset is u itself, (float)x scaled exactly (both normal in FP32)
    c = 0;
    d = ldexpf((float)x, tm_exp);
    return true;
  }
  const unsigned long long m = ((unsigned long long)b & 0xfffffffffffffull) | (1ull << 52);
  c = (int)(m >> (52 - s));
  d = ldexpf((float)(m & ((1ull << (52 - s)) - 1ull)), s - 52);
  return true;
}

// Base mesh point and fractional offsets of particle i: u = x N_g / L in FP64
// (wrapped positions: u in [0, N_g]), the offset u - floor(u) exact in FP64 and
// then rounded once to FP32 (the CIC weights are formed in FP32).  tm_exp: N_g / L
// = 2^tm_exp, read from the bits (or kNoExp: the FP64 route).
constexpr int kNoExp = 1 << 20;
__device__ __forceinline__ void cic_setup(const double *__restrict__ xs, int64_t n, int64_t i, double to_mesh,
                                          int tm_exp, double box, int ng, int (&i0)[3], float (&d)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double x = xs[k * n + i];
    int c;
    if (tm_exp == kNoExp || !cic_bits(x, box, tm_exp, c, d[k])) {
      const double u = x * to_mesh;
      const double f = floor(u);
      d[k] = (float)(u - f);
      c = (int)f;
    }
    if (c >= ng) c -= ng;
    if (c < 0) c += ng;
    i0[k] = c;
  }
}

// CIC mass assignment in 64-bit fixed point: corner value round(m 2^s w_x w_y w_z)
// (FP32 product, one rounding to an integer).  Consecutive particles (Morton
// order) mostly share their base mesh point: the lanes of a warp with the same
// base point form groups (match on the point's index); when every group is a run
// of adjacent lanes, each run adds its eight corner values with a segmented
// shuffle sum (integers: exact, so the mesh is the same as with one atomic per
// particle) and the run's first lane issues the eight atomics; otherwise every
// lane issues its own.
__global__ void k_deposit(const double *__restrict__ xs, const float4 *__restrict__ pm4, int64_t n, double to_mesh,
                          int tm_exp, double box, int ng, const unsigned *__restrict__ mmax, unsigned long long *__restrict__ q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool valid = i < n;  // whole warps stay for the warp-wide steps
  int i0[3] = {0, 0, 0};
  float d[3] = {0.f, 0.f, 0.f};
  float ms = 0.f;
  uint32_t key = 0xffffffffu - (uint32_t)lane;  // distinct keys (above any mesh index) for lanes past n
  if (valid) {
    cic_setup(xs, n, i, to_mesh, tm_exp, box, ng, i0, d);
    ms = ldexpf(pm4[i].w, fixed_exponent(mmax, n));
    key = ((uint32_t)i0[0] * (uint32_t)ng + (uint32_t)i0[1]) * (uint32_t)ng + (uint32_t)i0[2];
  }
  const unsigned grp = __match_any_sync(0xffffffffu, key);
  const int first = __ffs(grp) - 1, last = 31 - __clz(grp);
  const unsigned run = (unsigned)((1ull << (last - first + 1)) - 1ull);
  const bool agg = __all_sync(0xffffffffu, (grp >> first) == run);
#pragma unroll
  for (int ox = 0; ox < 2; ++ox) {
    const float wx = ox ? d[0] : 1.f - d[0];
    const int gx = i0[0] + ox == ng ? 0 : i0[0] + ox;
#pragma unroll
    for (int oy = 0; oy < 2; ++oy) {
      const float wy = oy ? d[1] : 1.f - d[1];
      const int gy = i0[1] + oy == ng ? 0 : i0[1] + oy;
#pragma unroll
      for (int oz = 0; oz < 2; ++oz) {
        const float wz = oz ? d[2] : 1.f - d[2];
        const int gz = i0[2] + oz == ng ? 0 : i0[2] + oz;
        long long v = valid ? __float2ll_rn(ms * (wx * wy * wz)) : 0ll;
        unsigned long long *dst = q + ((int64_t)gx * ng + gy) * ng + gz;
        if (agg) {
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_down_sync(0xffffffffu, v, o);
            if (lane + o <= last) v += t;
          }
          if (valid && lane == first) atomicAdd(dst, (unsigned long long)v);
        } else if (valid) {
          atomicAdd(dst, (unsigned long long)v);
        }
      }
    }
  }
}

// Mesh density: the fixed-point sums times 2^-s (exact scaling), rounded to FP32.
__global__ void k_fixed_to_real(const unsigned long long *__restrict__ q, int64_t cells, const unsigned *mmax,
                                int64_t n, float *__restrict__ rho) {
  const double inv = ldexp(1.0, -fixed_exponent(mmax, n));
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < cells; g += stride)
    rho[g] = (float)((double)(long long)q[g] * inv);
}

__device__ __forceinline__ float sincf_(float x) { return fabsf(x) < 1e-4f ? 1.f - x * x / 6.f : sinf(x) / x; }

// m(k) -> the three gradient components i k_d G(k) m(k) / L^3 (R2C layout [ng][ng][ng/2+1]).
// gtab == nullptr: the Gaussian Green function; otherwise gtab[i^2 + j^2 + l^2]
// holds the long-range Green function at that integer |k|^2 (units (2 pi / L)^2).
__global__ void k_green(const cufftComplex *__restrict__ mk, int ng, float box, float rs, float G,
                        const float *__restrict__ gtab, cufftComplex *__restrict__ ak) {
  const int nz = ng / 2 + 1;
  const int64_t total = (int64_t)ng * ng * nz;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int iz = (int)(t % nz), iy = (int)((t / nz) % ng), ix = (int)(t / ((int64_t)nz * ng));
  const float kf = 2.f * 3.14159265358979f / box;
  const int jx = ix <= ng / 2 ? ix : ix - ng, jy = iy <= ng / 2 ? iy : iy - ng;
  const float kx = kf * (float)jx;
  const float ky = kf * (float)jy;
  const float kz = kf * (float)iz;
  const float k2 = kx * kx + ky * ky + kz * kz;
  float g = 0.f;
  if (k2 > 0.f) {
    const float hh = 0.5f * box / (float)ng;
    const float w = sincf_(kx * hh) * sincf_(ky * hh) * sincf_(kz * hh);
    const float w2 = w * w;  // W(k) = (product of sincs)^2, divided out twice
    if (gtab)
      g = G * gtab[jx * jx + jy * jy + iz * iz] / (w2 * w2) / (box * box * box);
    else
      g = 4.f * 3.14159265358979f * G * expf(-k2 * rs * rs) / (k2 * w2 * w2) / (box * box * box);
  }
  const bool even = (ng & 1) == 0;
  const float kd[3] = {(even && ix == ng / 2) ? 0.f : kx, (even && iy == ng / 2) ? 0.f : ky,
                       (even && iz == ng / 2) ? 0.f : kz};
  const cufftComplex m = mk[t];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float s = kd[d] * g;  // i s (re + i im) = -s im + i s re
    ak[d * total + t] = make_float2(-s * m.y, s * m.x);
  }
}

__global__ void k_interpolate(const double *__restrict__ xs, const uint32_t *__restrict__ perm, int64_t n,
                              double to_mesh, int tm_exp, double box, int ng, const float *__restrict__ a,
                              float *__restrict__ acc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int i0[3];
  float d[3];
  cic_setup(xs, n, i, to_mesh, tm_exp, box, ng, i0, d);
  const int64_t cells = (int64_t)ng * ng * ng;
  float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int ox = 0; ox < 2; ++ox) {
    const float wx = ox ? d[0] : 1.f - d[0];
    const int gx = i0[0] + ox == ng ? 0 : i0[0] + ox;
#pragma unroll
    for (int oy = 0; oy < 2; ++oy) {
      const float wy = oy ? d[1] : 1.f - d[1];
      const int gy = i0[1] + oy == ng ? 0 : i0[1] + oy;
#pragma unroll
      for (int oz = 0; oz < 2; ++oz) {
        const float wz = oz ? d[2] : 1.f - d[2];
        const int gz = i0[2] + oz == ng ? 0 : i0[2] + oz;
        const int64_t g = ((int64_t)gx * ng + gy) * ng + gz;
        const float w = wx * wy * wz;
#pragma unroll
        for (int k = 0; k < 3; ++k) s[k] = fmaf(w, a[k * cells + g], s[k]);
      }
    }
  }
  const uint32_t o = perm[i];
#pragma unroll
  for (int k = 0; k < 3; ++k) acc[k * n + o] += s[k];
}

__global__ void k_kick(float *__restrict__ vel, const float *__restrict__ acc, int64_t n3, float h, StepGuard g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g.tree_overflow && (*g.tree_overflow || *g.walk_overflow || *g.walk_left)) return;
  if (i < n3) vel[i] = fmaf(h, acc[i], vel[i]);
}

// inv_pow2 = 1 / box when box is a power of two (the quotient is then an exact
// product: no FP64 division, which is slow on this GPU), else 0.
__global__ void k_drift(double *__restrict__ pos, const float *__restrict__ vel, int64_t n3, double dt, double box,
                        double inv_pow2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  double x = pos[i] + dt * (double)vel[i];
  const long long b = __double_as_longlong(x);
  if (b < 0 || b >= __double_as_longlong(box)) {  // outside [0, L) (or NaN): wrap (in [0, L) nothing to do)
    x -= box * floor(div_box(x, box, inv_pow2));
    if (x >= box) x -= box;  // rounding of a value just below 0
  }
  pos[i] = x;
}

cudaError_t fft_error(cufftResult r) { return r == CUFFT_SUCCESS ? cudaSuccess : cudaErrorUnknown; }

}  // namespace

void pm_release(Ctx &c) {
  if (c.pm_plan_r2c >= 0) cufftDestroy(c.pm_plan_r2c);
  if (c.pm_plan_c2r >= 0) cufftDestroy(c.pm_plan_c2r);
  c.pm_plan_r2c = c.pm_plan_c2r = -1;
  release(c.pm_q);
  release(c.pm_rho);
  release(c.pm_mk);
  release(c.pm_ak);
  release(c.pm_a);
  release(c.pm_gtab);
  c.pm_gtab_n = 0;
}

namespace {

// Gauss-Legendre rule of n points on [0, 1]: Newton's method on the Legendre
// polynomial P_n (three-term recurrence), started from the Chebyshev-like
// estimates cos(pi (i + 3/4) / (n + 1/2)) of its roots.
void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // (2 / ((1 - t^2) P'^2)) / 2 for [0, 1]
  }
}

// Long-range Green function of the polynomial split at |k|^2 = (2 pi / L)^2 n,
// n = 0..3 (ng/2)^2: 4 pi / k^2 minus the transform of the short-range kernel
// 1/r - P(r) (r < R_c),
//   psi^(k) = (4 pi R_c / k) int_0^1 [1 - (15 x - 10 x^3 + 3 x^5) / 8] sin(k R_c x) dx,
// by a 96-point Gauss-Legendre rule in FP64 (k R_c stays below 10 pi for the
// meshes allowed, a few oscillations of a smooth integrand).
cudaError_t green_table_poly(Ctx &c) {
  const int ng = c.prm.pm_grid, h = ng / 2;
  const size_t nt = (size_t)3 * h * h + 1;
  if (c.pm_gtab_n == nt) return cudaSuccess;
  std::vector<double> gx, gw;
  gauss_legendre01(96, gx, gw);
  std::vector<float> tab(nt, 0.f);
  const double kf = 2.0 * M_PI / c.prm.box, rc = c.rc;
  for (size_t n = 1; n < nt; ++n) {
    const double k = kf * std::sqrt((double)n);
    double integ = 0.0;
    for (int i = 0; i < 96; ++i) {
      const double x = gx[i];
      integ += gw[i] * (1.0 - (15.0 * x - 10.0 * x * x * x + 3.0 * x * x * x * x * x) / 8.0) * std::sin(k * rc * x);
    }
    tab[n] = (float)(4.0 * M_PI / (k * k) - 4.0 * M_PI * rc / k * integ);
  }
  cudaError_t e = ensure(c.pm_gtab, nt * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(c.pm_gtab.p, tab.data(), nt * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) c.pm_gtab_n = nt;
  return e;
}

}  // namespace

cudaError_t pm_prepare(Ctx &c) {
  const int ng = c.prm.pm_grid;
  const int64_t cells = (int64_t)ng * ng * ng, kcells = (int64_t)ng * ng * (ng / 2 + 1);
  cudaError_t e;
  if ((e = ensure(c.pm_q, cells * 8)) != cudaSuccess) return e;
  if ((e = ensure(c.pm_rho, cells * 4)) != cudaSuccess) return e;
  if ((e = ensure(c.pm_mk, kcells * sizeof(cufftComplex))) != cudaSuccess) return e;
  if ((e = ensure(c.pm_ak, 3 * kcells * sizeof(cufftComplex))) != cudaSuccess) return e;
  if ((e = ensure(c.pm_a, 3 * cells * 4)) != cudaSuccess) return e;
  if (c.pm_plan_r2c < 0) {
    cufftHandle p;
    if ((e = fft_error(cufftPlan3d(&p, ng, ng, ng, CUFFT_R2C))) != cudaSuccess) return e;
    c.pm_plan_r2c = p;
    int dims[3] = {ng, ng, ng};
    if ((e = fft_error(cufftPlanMany(&p, 3, dims, nullptr, 1, (int)kcells, nullptr, 1, (int)cells, CUFFT_C2R, 3))) !=
        cudaSuccess)
      return e;
    c.pm_plan_c2r = p;
  }
  if (c.prm.split == 1 && (e = green_table_poly(c)) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t pm_long_range(Ctx &c, float *acc, cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  const int ng = c.prm.pm_grid;
  const int64_t cells = (int64_t)ng * ng * ng, kcells = (int64_t)ng * ng * (ng / 2 + 1);
  cudaError_t e;
  if ((e = pm_prepare(c)) != cudaSuccess) return e;
  if ((e = fft_error(cufftSetStream(c.pm_plan_r2c, st))) != cudaSuccess) return e;
  if ((e = fft_error(cufftSetStream(c.pm_plan_c2r, st))) != cudaSuccess) return e;

  unsigned *mmax = reinterpret_cast<unsigned *>(P<uint64_t>(c.d_small) + 2);
  if ((e = cudaMemsetAsync(mmax, 0, 8, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c.pm_q.p, 0, cells * 8, st)) != cudaSuccess) return e;
  const int T = 256;
  const double to_mesh = (double)ng / c.prm.box;
  int tm_exp = 0;  // N_g / L = 2^tm_exp exactly (both powers of two), else the FP64 route
  const bool pow2 = std::frexp(to_mesh, &tm_exp) == 0.5 && box_inverse_if_pow2(c.prm.box) != 0.0;
  tm_exp = pow2 ? tm_exp - 1 : kNoExp;
  unsigned gm = blocks_for(c.n, T);
  if (gm > 152 * 16) gm = 152 * 16;
  k_mass_absmax<<<gm, T, 0, st>>>(P<float4>(c.pm4), c.n, mmax);
  k_deposit<<<blocks_for(c.n, T), T, 0, st>>>(P<double>(c.xs), P<float4>(c.pm4), c.n, to_mesh, tm_exp, c.prm.box,
                                              ng, mmax,
                                              P<unsigned long long>(c.pm_q));
  unsigned gc = blocks_for(cells, T);
  if (gc > 152 * 16) gc = 152 * 16;
  k_fixed_to_real<<<gc, T, 0, st>>>(P<unsigned long long>(c.pm_q), cells, mmax, c.n,
                                                      P<float>(c.pm_rho));
  note_launch(3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = fft_error(cufftExecR2C(c.pm_plan_r2c, P<cufftReal>(c.pm_rho), P<cufftComplex>(c.pm_mk)))) != cudaSuccess)
    return e;
  k_green<<<blocks_for(kcells, T), T, 0, st>>>(P<cufftComplex>(c.pm_mk), ng, (float)c.prm.box, (float)c.rs,
                                               (float)c.prm.G, c.prm.split == 1 ? P<float>(c.pm_gtab) : nullptr,
                                               P<cufftComplex>(c.pm_ak));
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = fft_error(cufftExecC2R(c.pm_plan_c2r, P<cufftComplex>(c.pm_ak), P<cufftReal>(c.pm_a)))) != cudaSuccess)
    return e;
  k_interpolate<<<blocks_for(c.n, T), T, 0, st>>>(P<double>(c.xs), P<uint32_t>(c.idx), c.n, to_mesh, tm_exp,
                                                  c.prm.box, ng,
                                                  P<float>(c.pm_a), acc);
  note_launch();
  return cudaGetLastError();
}

cudaError_t kick(float *vel, const float *acc, int64_t n, double h, cudaStream_t st) {
  return kick_guarded(vel, acc, n, h, StepGuard{}, st);
}

cudaError_t kick_guarded(float *vel, const float *acc, int64_t n, double h, StepGuard g, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_kick<<<blocks_for(3 * n, 256), 256, 0, st>>>(vel, acc, 3 * n, (float)h, g);
  note_launch();
  return cudaGetLastError();
}

cudaError_t drift(double *pos, const float *vel, int64_t n, double dt, double box, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_drift<<<blocks_for(3 * n, 256), 256, 0, st>>>(pos, vel, 3 * n, dt, box, box_inverse_if_pow2(box));
  note_launch();
  return cudaGetLastError();
}

}  // namespace hfmm
