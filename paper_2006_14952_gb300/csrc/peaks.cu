// Throughput probes for the roofline of the ALU-bound kernels (the P2P pair
// sum and the CUDA-core M2L): FP32 fused multiply-add, packed FP32x2
// fused multiply-add, and the two special-function instructions the pair
// law uses (ex2, rsqrt).  Each thread runs independent dependency chains long
// enough to hide the pipeline latency; the grid fills every SM with 2048
// threads.  The rate is work per second over one launch timed with CUDA
// events on the caller's stream, after one untimed warm-up launch.
#include "common.cuh"

namespace hfmm {
namespace {

constexpr int kChains = 16;  // independent chains per thread
constexpr int kUnroll = 8;   // loop body: kChains * kUnroll operations per thread

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// kind 0: fma.rn.f32; 1: packed fma.rn.f32x2; 2: ex2.approx; 3: rsqrt.approx.
template <int kKind>
__global__ void __launch_bounds__(256) k_alu_peak(int iters, float seed, float *__restrict__ out) {
  const float b = 0.99999994f, c = 1e-7f;
  float x[kChains];
  float2 y[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    x[j] = seed + 1e-3f * (float)(threadIdx.x + j);
    y[j] = make_float2(x[j], x[j] + 0.5f);
  }
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) {
        if (kKind == 0) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[j]) : "f"(b), "f"(c));
        if (kKind == 1) y[j] = __ffma2_rn(y[j], b2, c2);
        if (kKind == 2) x[j] = ex2_approx(x[j]);
        if (kKind == 3) x[j] = rsqrt_approx(x[j]);
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += kKind == 1 ? y[j].x + y[j].y : x[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace hfmm

using namespace hfmm;

extern "C" int hfmm_alu_peak(int kind, int iters, float *scratch, double *rate, double *ms, void *stream) {
  if (kind < 0 || kind > 3 || iters < 1 || !scratch || !rate) return HFMM_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HFMM_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned blocks = (unsigned)sms * 8u;  // 8 blocks of 256 threads: 2048 threads per SM
  auto launch = [&]() {
    switch (kind) {
      case 0: k_alu_peak<0><<<blocks, 256, 0, st>>>(iters, 1.0f, scratch); break;
      case 1: k_alu_peak<1><<<blocks, 256, 0, st>>>(iters, 1.0f, scratch); break;
      case 2: k_alu_peak<2><<<blocks, 256, 0, st>>>(iters, -3.0f, scratch); break;
      default: k_alu_peak<3><<<blocks, 256, 0, st>>>(iters, 2.0f, scratch); break;
    }
    note_launch();
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HFMM_ERR_CUDA;
  launch();  // warm-up
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  float t = 0.f;
  cudaError_t err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || !(t > 0.f)) return HFMM_ERR_CUDA;
  // operations per thread; an FMA counts 2 flop, a packed FMA 4
  const double ops = (double)iters * kChains * kUnroll * (kind == 0 ? 2.0 : kind == 1 ? 4.0 : 1.0);
  *rate = ops * (double)blocks * 256.0 / (t * 1e-3);
  if (ms) *ms = t;
  return HFMM_OK;
}
