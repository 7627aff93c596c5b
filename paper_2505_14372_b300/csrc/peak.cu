// FP32 CUDA-core throughput microbenchmark: the denominator of the FFT tile
// kernels' roofline (their arithmetic is FP32 FMA/ADD/MUL on the CUDA cores).
//
// Every thread runs kChains independent multiply-add recurrences
// x <- x * a + b (no dependency between chains, so the FMA pipe is never
// waiting on a result), kUnroll rounds per loop trip; the grid holds
// kBlocksPerSM 256-thread blocks per SM (64 warps per SM, full occupancy at
// the ~40 registers a thread needs).  Scalar FFMA and packed FFMA2 (two
// FP32 FMAs per instruction, sm_100+) are both measured: the caller takes
// the faster as the measured peak.  The result of the chains is written only
// when it equals an impossible value, which keeps them live without memory
// traffic.
#include <cuda_runtime.h>

#include <string>

#include "engine.h"
#include "errors.h"
#include "ptycho.h"

namespace {

constexpr int kChains = 16;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

__global__ void __launch_bounds__(kThreads) k_ffma(float* sink, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == -1.2345e30f) sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_ffma2(float* sink, int iters, float a, float b) {
  float2 x[kChains / 2];
#pragma unroll
  for (int i = 0; i < kChains / 2; ++i)
    x[i] = make_float2((float)(threadIdx.x + 2 * i) * 1e-3f, (float)(threadIdx.x + 2 * i + 1) * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
      for (int i = 0; i < kChains / 2; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains / 2; ++i) s += x[i].x + x[i].y;
  if (s == -1.2345e30f) sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" int ptycho_fp32_peak_launch(int32_t packed, int32_t iters, float* sink, double* flops_out,
                                       ptycho_stream stream) {
  if (iters < 1) return perr(PTYCHO_EINVAL, "iters < 1");
  if (!sink || !flops_out) return perr(PTYCHO_EINVAL, "NULL argument");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return perr(PTYCHO_ECUDA, "no CUDA device");
  }
  const int blocks = sms * kBlocksPerSM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a = 1 - 2^-20, b = 2^-20: every chain stays near [0, 1], far from
  // overflow or denormals, for any number of rounds
  const float a = 1.0f - 9.5367431640625e-7f, b = 9.5367431640625e-7f;
  if (packed) k_ffma2<<<blocks, kThreads, 0, s>>>(sink, iters, a, b);
  else k_ffma<<<blocks, kThreads, 0, s>>>(sink, iters, a, b);
  ptycho::count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return perr(PTYCHO_ECUDA, std::string("FFMA launch failed: ") + cudaGetErrorString(e));
  *flops_out = 2.0 * (double)blocks * kThreads * (double)iters * kUnroll * kChains;
  return PTYCHO_OK;
}

extern "C" int32_t ptycho_fp32_peak_sink_elems(void) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms * kBlocksPerSM * kThreads;
}
