// Inference and training kernels of the learned-acceptance network (mlp.cuh).
//  k_mlp_infer: tensor-core inference (mma.sync m16n8k16 BF16 -> FP32), one
//               warp per 16 rows; the same routine the traversal calls.
//  k_mlp_grad:  softmax cross-entropy forward + backward, one warp per sample,
//               BF16-rounded weights / inputs / activations with FP32 sums and
//               the rounding treated as identity in the backward pass;
//               per-block gradient partials (shared-memory accumulation).
//  k_mlp_reduce, k_mlp_adam: fixed-order reduction of the partials and an
//               Adam step on the FP32 master weights, writing the BF16 copy.
#include "mlp.cuh"

namespace hfmm {
namespace {

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void __launch_bounds__(256) k_mlp_infer(const __nv_bfloat16 *__restrict__ w, const float *__restrict__ x,
                                                   int64_t n, float *__restrict__ logits, int *__restrict__ cls) {
  __shared__ uint32_t sw[kMlpSmemWords];
  __shared__ __align__(16) __nv_bfloat16 xs[8][16 * 16];
  mlp_stage(w, sw);
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  __nv_bfloat16 *xr = xs[wp];
  const int64_t nwarp = (int64_t)gridDim.x * 8;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + wp) * 16; base < n; base += nwarp * 16) {
    for (int i = lane; i < 256; i += 32) {
      const int r = i >> 4, c = i & 15;
      const int64_t row = base + r;
      xr[i] = __float2bfloat16_rn((c < kMlpIn && row < n) ? x[row * kMlpIn + c] : 0.f);
    }
    __syncwarp();
    float l[4];
    mlp_logits16(sw, xr, l);
    int c0, c8;
    mlp_argmax16(l, c0, c8);
    const int64_t r0 = base + g, r8 = base + g + 8;
    if (logits) {
      if (r0 < n) { logits[r0 * 8 + 2 * t] = l[0]; logits[r0 * 8 + 2 * t + 1] = l[1]; }
      if (r8 < n) { logits[r8 * 8 + 2 * t] = l[2]; logits[r8 * 8 + 2 * t + 1] = l[3]; }
    }
    if (cls && t == 0) {
      if (r0 < n) cls[r0] = c0;
      if (r8 < n) cls[r8] = c8;
    }
    __syncwarp();
  }
}

constexpr int kGradThreads = 256;

__global__ void __launch_bounds__(kGradThreads) k_mlp_grad(const float *__restrict__ wm, const float *__restrict__ x,
                                                           const int *__restrict__ labels,
                                                           const float *__restrict__ cw, int64_t n,
                                                           float *__restrict__ part, float *__restrict__ loss_part) {
  __shared__ float gs[kMlpW];
  __shared__ float act[8][4][kMlpH];  // per warp: z1, h1, z2, h2
  __shared__ float dz2s[8][kMlpH];
  __shared__ float lsum[8];
  for (int i = threadIdx.x; i < kMlpW; i += blockDim.x) gs[i] = 0.f;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (lane == 0) lsum[wp] = 0.f;
  __syncthreads();
  // BF16-rounded weights read on the fly from the FP32 master copy
  auto W1 = [&](int i) { return bf(__ldg(wm + kOffW1 + i)); };
  auto B1 = [&](int i) { return bf(__ldg(wm + kOffB1 + i)); };
  auto W2 = [&](int i) { return bf(__ldg(wm + kOffW2 + i)); };
  auto B2 = [&](int i) { return bf(__ldg(wm + kOffB2 + i)); };
  auto W3 = [&](int i) { return bf(__ldg(wm + kOffW3 + i)); };
  auto B3 = [&](int i) { return bf(__ldg(wm + kOffB3 + i)); };
  float *z1 = act[wp][0], *h1 = act[wp][1], *z2 = act[wp][2], *h2 = act[wp][3];
  for (int64_t sidx = (int64_t)blockIdx.x * 8 + wp; sidx < n; sidx += (int64_t)gridDim.x * 8) {
    float xr[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) xr[k] = bf(x[sidx * kMlpIn + k]);
    const int lab = labels[sidx];
    const float wgt = cw ? cw[lab] : 1.f;
    // forward
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int u = lane + 32 * r;
      float z = B1(u);
      for (int k = 0; k < kMlpIn; ++k) z += W1(u * kMlpIn + k) * xr[k];
      z1[u] = z;
      h1[u] = bf(fmaxf(z, 0.f));
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int u = lane + 32 * r;
      float z = B2(u);
      for (int k = 0; k < kMlpH; ++k) z += W2(u * kMlpH + k) * h1[k];
      z2[u] = z;
      h2[u] = bf(fmaxf(z, 0.f));
    }
    __syncwarp();
    float zo = -1e30f;
    if (lane < kMlpOut) {
      float z = B3(lane);
      for (int k = 0; k < kMlpH; ++k) z += W3(lane * kMlpH + k) * h2[k];
      zo = z;
    }
    float mx = zo;
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float ex = lane < kMlpOut ? __expf(zo - mx) : 0.f, se = ex;
    for (int o = 16; o; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    const float pr = ex / se;
    const float dz3 = lane < kMlpOut ? wgt * (pr - (lane == lab ? 1.f : 0.f)) : 0.f;
    const float plab = __shfl_sync(0xffffffffu, pr, lab);
    if (lane == 0) lsum[wp] += -wgt * __logf(fmaxf(plab, 1e-30f));
    // backward
    if (lane < kMlpOut) atomicAdd(&gs[kOffB3 + lane], dz3);
    float d3[kMlpOut];
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) d3[o] = __shfl_sync(0xffffffffu, dz3, o);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int k = lane + 32 * r;
      float dh = 0.f;
#pragma unroll
      for (int o = 0; o < kMlpOut; ++o) {
        atomicAdd(&gs[kOffW3 + o * kMlpH + k], d3[o] * h2[k]);
        dh += W3(o * kMlpH + k) * d3[o];
      }
      dz2s[wp][k] = z2[k] > 0.f ? dh : 0.f;
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int u = lane + 32 * r;
      const float d = dz2s[wp][u];
      atomicAdd(&gs[kOffB2 + u], d);
      if (d != 0.f)
        for (int k = 0; k < kMlpH; ++k) atomicAdd(&gs[kOffW2 + u * kMlpH + k], d * h1[k]);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int k = lane + 32 * r;
      float dh = 0.f;
      for (int u = 0; u < kMlpH; ++u) dh += W2(u * kMlpH + k) * dz2s[wp][u];
      const float d = z1[k] > 0.f ? dh : 0.f;
      atomicAdd(&gs[kOffB1 + k], d);
      if (d != 0.f)
        for (int j = 0; j < kMlpIn; ++j) atomicAdd(&gs[kOffW1 + k * kMlpIn + j], d * xr[j]);
    }
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kMlpW; i += blockDim.x) part[(size_t)blockIdx.x * kMlpW + i] = gs[i];
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int q = 0; q < 8; ++q) s += lsum[q];
    loss_part[blockIdx.x] = s;
  }
}

__global__ void k_mlp_reduce(const float *__restrict__ part, const float *__restrict__ loss_part, int nb, float scale,
                             float *__restrict__ grad, float *__restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kMlpW) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * kMlpW + i];
    grad[i] = s * scale;
  }
  if (i == 0 && loss) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += loss_part[b];
    *loss = s * scale;
  }
}

__global__ void k_mlp_adam(float *__restrict__ wm, float *__restrict__ m1, float *__restrict__ m2,
                           const float *__restrict__ grad, float lr, float b1, float b2, float eps, float c1, float c2,
                           __nv_bfloat16 *__restrict__ wout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpW) return;
  const float gr = grad[i];
  const float a = b1 * m1[i] + (1.f - b1) * gr, b = b2 * m2[i] + (1.f - b2) * gr * gr;
  m1[i] = a;
  m2[i] = b;
  const float w = wm[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
  wm[i] = w;
  if (wout) wout[i] = __float2bfloat16_rn(w);
}

}  // namespace

cudaError_t mlp_infer(const void *w_bf16, const float *x, int64_t n, float *logits, int *cls, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  unsigned g = (unsigned)((n + 127) / 128);
  if (g > 152 * 8) g = 152 * 8;
  k_mlp_infer<<<g, 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(w_bf16), x, n, logits, cls);
  note_launch();
  return cudaGetLastError();
}

size_t mlp_train_scratch_bytes() { return (size_t)(152 * 2) * (kMlpW + 1) * sizeof(float); }

cudaError_t mlp_grad(const float *wm, const float *x, const int *labels, const float *cw, int64_t n, float *grad,
                     float *loss, void *scratch, cudaStream_t st) {
  if (n <= 0) return cudaErrorInvalidValue;
  int nb = (int)((n + 7) / 8);
  if (nb > 152 * 2) nb = 152 * 2;
  float *part = static_cast<float *>(scratch);
  float *lp = part + (size_t)nb * kMlpW;
  k_mlp_grad<<<nb, kGradThreads, 0, st>>>(wm, x, labels, cw, n, part, lp);
  k_mlp_reduce<<<(kMlpW + 255) / 256, 256, 0, st>>>(part, lp, nb, 1.f / (float)n, grad, loss);
  note_launch(2);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float *wm, float *m1, float *m2, const float *grad, float lr, int step, void *w_bf16,
                     cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_mlp_adam<<<(kMlpW + 255) / 256, 256, 0, st>>>(wm, m1, m2, grad, lr, b1, b2, eps, c1, c2,
                                                   static_cast<__nv_bfloat16 *>(w_bf16));
  note_launch();
  return cudaGetLastError();
}

}  // namespace hfmm
