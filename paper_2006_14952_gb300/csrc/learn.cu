// Training data for the learned acceptance: for candidate cell pairs (rules 1
// and 3 passed, L / S_c within the safety bound), the network's features and
// the error of accepting the pair with M2L at each order q = 2..8, measured
// against the pair's own direct sum.
//
// Error of a pair (A, B) at order q: the contribution of B's particles to the
// accelerations of up to 32 particles of A (evenly strided), once by direct
// summation of the pair force (FP64 separations, FP32 force law with erfcf /
// expf) and once by P2M (the order-8 multipole, truncated to order q), M2L at
// order q (Eq. m2l with the truncated derivative tensors, evaluated in units
// of the centre distance as in m2l.cu) and L2P (Eq. l2p);
//   err_q = sqrt(sum_i |a_q,i - a_i|^2) / sqrt(sum_i |a_i|^2).
#include "mlp.cuh"

namespace hfmm {
namespace {

constexpr int kLT = 128;
constexpr int kMaxSink = 32;

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

__global__ void __launch_bounds__(kLT) k_pair_errors(const uint64_t *__restrict__ cand, int64_t ncand,
                                                    const uint4 *__restrict__ cell, const uint2 *__restrict__ range,
                                                    const double *__restrict__ xs, const float4 *__restrict__ pm4,
                                                    int64_t n, const float *__restrict__ M, int ldm, double box,
                                                    float rs, float inv_rs_h, float inv_rc_h, float G,
                                                    float *__restrict__ feat, float *__restrict__ err) {
  __shared__ uchar4 mi[kNCMax];
  __shared__ float Dh[kNCMax], Lq[kNCMax], fk[kPMax + 1];
  __shared__ float ex[kMaxSink][3], red[kLT][3];
  __shared__ float num[kMaxSink], den[kMaxSink];
  const int tid = threadIdx.x;
  for (int c = tid; c < kNCMax; c += kLT) {
    int x, y, z;
    mdecode(c, x, y, z);
    mi[c] = make_uchar4((unsigned char)x, (unsigned char)y, (unsigned char)z, (unsigned char)(x + y + z));
  }
  __syncthreads();
  const float kInvSqrtPi = 0.56418958354775628f;
  for (int64_t pi = blockIdx.x; pi < ncand; pi += gridDim.x) {
    const uint64_t e = cand[pi];
    const uint32_t a = pair_sink(e), b = pair_src(e), s = pair_shift(e);
    const uint4 ca = cell[a], cb = cell[b];
    const uint2 ra = range[a], rb = range[b];
    const float *Mb = M + (size_t)b * ldm;
    if (tid == 0) pair_features(ca, cb, s, ra.y, rb.y, Mb, inv_rs_h, inv_rc_h, feat + pi * kMlpIn);
    const int ns = ra.y < (uint32_t)kMaxSink ? (int)ra.y : kMaxSink;
    const int streams = kLT / ns;
    const double ha = box / (double)(1u << ca.w), hbx = box / (double)(1u << cb.w);
    const double za[3] = {((double)ca.x + 0.5) * ha, ((double)ca.y + 0.5) * ha, ((double)ca.z + 0.5) * ha};
    const double shx = (double)shift_component(s, 0) * box, shy = (double)shift_component(s, 1) * box,
                 shz = (double)shift_component(s, 2) * box;
    // direct contribution of B to the sampled sinks of A
    {
      const int k = tid % ns, st = tid / ns;
      float ax = 0.f, ay = 0.f, az = 0.f;
      if (st < streams) {
        const uint32_t i = ra.x + (uint32_t)(((uint64_t)k * ra.y) / ns);
        const double xi = xs[i], yi = xs[n + i], zi = xs[2 * n + i];
        for (uint32_t j = rb.x + st; j < rb.x + rb.y; j += streams) {
          const float dx = (float)(xi - (xs[j] + shx)), dy = (float)(yi - (xs[n + j] + shy)),
                      dz = (float)(zi - (xs[2 * n + j] + shz));
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (!(r2 > 0.f)) continue;
          const float r = sqrtf(r2), x = r / rs;
          const float S = erfcf(0.5f * x) + x * kInvSqrtPi * expf(-0.25f * x * x);
          const float f = -S / (r2 * r) * pm4[j].w;
          ax += f * dx;
          ay += f * dy;
          az += f * dz;
        }
      }
      red[tid][0] = ax;
      red[tid][1] = ay;
      red[tid][2] = az;
    }
    __syncthreads();
    if (tid < ns) {
      float sx = 0.f, sy = 0.f, sz = 0.f;
      for (int q = 0; q < streams; ++q) {
        sx += red[tid + q * ns][0];
        sy += red[tid + q * ns][1];
        sz += red[tid + q * ns][2];
      }
      ex[tid][0] = G * sx;
      ex[tid][1] = G * sy;
      ex[tid][2] = G * sz;
    }
    // unit separation, prefactors at r^ = 1, derivative tensor to order 8
    int64_t dd[3];
    half_delta(ca, cb, s, dd);
    const float Rx = -(float)dd[0], Ry = -(float)dd[1], Rz = -(float)dd[2];
    const float r2h = Rx * Rx + Ry * Ry + Rz * Rz, rinv = rsqrtf(r2h);
    const float xr = r2h * rinv * inv_rs_h;
    const float R[3] = {Rx * rinv, Ry * rinv, Rz * rinv};
    const float u = (float)(2 * half_width(ca.w)) * rinv, v = (float)(2 * half_width(cb.w)) * rinv;
    if (tid == 0) {
      fk[0] = erfcf(0.5f * xr);
      float tk = -xr * kInvSqrtPi * expf(-0.25f * xr * xr);
      for (int q = 0; q < kPMax; ++q) {
        fk[q + 1] = -(float)(2 * q + 1) * fk[q] + tk;
        tk = -tk * 0.5f * xr * xr;
      }
    }
    __syncthreads();
    for (int c = tid; c < kNCMax; c += kLT) {
      const uchar4 nn = mi[c];
      float sum = 0.f;
      for (int kx = 0; 2 * kx <= nn.x; ++kx)
        for (int ky = 0; 2 * ky <= nn.y; ++ky)
          for (int kz = 0; 2 * kz <= nn.z; ++kz) {
            const float co = factf(nn.x) / (ldexpf(1.f, kx) * factf(kx) * factf(nn.x - 2 * kx)) * factf(nn.y) /
                             (ldexpf(1.f, ky) * factf(ky) * factf(nn.y - 2 * ky)) * factf(nn.z) /
                             (ldexpf(1.f, kz) * factf(kz) * factf(nn.z - 2 * kz));
            sum += co * powi(R[0], nn.x - 2 * kx) * powi(R[1], nn.y - 2 * ky) * powi(R[2], nn.z - 2 * kz) *
                   fk[nn.w - kx - ky - kz];
          }
      Dh[c] = sum;
    }
    __syncthreads();
    const float inv_ha2 = (float)(1.0 / (ha * ha));
    for (int q = 2; q <= 8; ++q) {
      const int ncq = ncoef(q);
      for (int c = tid; c < ncq; c += kLT) {
        const uchar4 nn = mi[c];
        float sum = 0.f;
        const int rem = ncoef(q - nn.w);
        for (int m = 0; m < rem; ++m) {
          const uchar4 mm = mi[m];
          sum += Mb[m] * powi(v, mm.w) * Dh[midx(nn.x + mm.x, nn.y + mm.y, nn.z + mm.z)];
        }
        Lq[c] = sum * powi(u, nn.w + 1);
      }
      __syncthreads();
      if (tid < ns) {
        const uint32_t i = ra.x + (uint32_t)(((uint64_t)tid * ra.y) / ns);
        const float ux = (float)((xs[i] - za[0]) / ha), uy = (float)((xs[n + i] - za[1]) / ha),
                    uz = (float)((xs[2 * n + i] - za[2]) / ha);
        float lx = 0.f, ly = 0.f, lz = 0.f;
        for (int c = 0; c < ncoef(q - 1); ++c) {
          const uchar4 mm = mi[c];
          const float mono = powi(ux, mm.x) * powi(uy, mm.y) * powi(uz, mm.z) / (factf(mm.x) * factf(mm.y) * factf(mm.z));
          lx += Lq[midx(mm.x + 1, mm.y, mm.z)] * mono;
          ly += Lq[midx(mm.x, mm.y + 1, mm.z)] * mono;
          lz += Lq[midx(mm.x, mm.y, mm.z + 1)] * mono;
        }
        const float gx = G * inv_ha2 * lx - ex[tid][0], gy = G * inv_ha2 * ly - ex[tid][1],
                    gz = G * inv_ha2 * lz - ex[tid][2];
        num[tid] = gx * gx + gy * gy + gz * gz;
        den[tid] = ex[tid][0] * ex[tid][0] + ex[tid][1] * ex[tid][1] + ex[tid][2] * ex[tid][2];
      }
      __syncthreads();
      if (tid == 0) {
        float sn = 0.f, sd = 0.f;
        for (int k = 0; k < ns; ++k) {
          sn += num[k];
          sd += den[k];
        }
        err[pi * 7 + (q - 2)] = sd > 0.f ? sqrtf(sn / sd) : 0.f;
      }
      __syncthreads();
    }
  }
}

}  // namespace

cudaError_t collect_pairs(Ctx &c, int64_t max_pairs, uint32_t sample_mod, float *feat, float *err, int64_t *count,
                          cudaStream_t st) {
  cudaError_t e;
  *count = 0;
  if (c.n == 0) return cudaSuccess;
  if ((e = ensure(c.cand, (size_t)(max_pairs > 0 ? max_pairs : 1) * 8)) != cudaSuccess) return e;
  c.cand_cap = (uint64_t)max_pairs;
  c.sample_mod = sample_mod ? sample_mod : 1u;
  if ((e = cudaMemsetAsync(P<uint64_t>(c.d_small) + 7, 0, 8, st)) != cudaSuccess) return e;
  size_t eb = (size_t)c.nnodes * c.ldm * sizeof(float);
  if ((e = ensure(c.M, eb)) != cudaSuccess) return e;
  if ((e = upward(c, st)) != cudaSuccess) return e;
  c.collect = true;
  e = traverse(c, st);
  c.collect = false;
  if (e != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(c.h_pinned, P<uint64_t>(c.d_small) + 7, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  int64_t nc = (int64_t)c.h_pinned[0];
  if (nc > max_pairs) nc = max_pairs;
  *count = nc;
  c.ncand_last = nc;
  if (nc == 0) return cudaSuccess;
  const double hu = c.prm.box / (double)kHalfBox;
  k_pair_errors<<<152 * 8, kLT, 0, st>>>(P<uint64_t>(c.cand), nc, P<uint4>(c.cell), P<uint2>(c.range),
                                         P<double>(c.xs), P<float4>(c.pm4), c.n, P<float>(c.M), c.ldm, c.prm.box,
                                         (float)c.rs, (float)(hu / c.rs), (float)(hu / c.rc), (float)c.prm.G, feat,
                                         err);
  note_launch();
  return cudaGetLastError();
}

}  // namespace hfmm
