// Pointwise kernels around the FFT tile: incoherent mode sum, noise-model
// loss and detector seed (arXiv 2505.14372 §3, §3.1), FP64 reductions and
// the complex Adam update (§3.2).
#pragma once
#include <stdint.h>

#include "noise.cuh"
#include "radix.cuh"

namespace ptycho {

constexpr int kRedThreads = 256;

// Block-wide FP64 sum; every thread gets the total.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) t += sh[i];
  return t;
}

// Complex Adam on element e: m <- b1 m + (1-b1) g; v <- b2 v + (1-b2)|g|^2;
// z <- z - lr (m bc1) / (sqrt(v bc2) + eps), bc = 1/(1 - beta^t) (§3.2).
// The update on values held in registers (z, m, v in and out).
__device__ __forceinline__ void adam_math(float2& z, float2& m, float& v, float2 g, float lr, float b1, float b2,
                                          float eps, float bc1, float bc2) {
  m.x = fmaf(b1, m.x, (1.0f - b1) * g.x);
  m.y = fmaf(b1, m.y, (1.0f - b1) * g.y);
  v = fmaf(b2, v, (1.0f - b2) * cabs2(g));
  const float den = sqrtf(v * bc2) + eps;
  const float s = lr * bc1 / den;
  z.x -= s * m.x;
  z.y -= s * m.y;
}
__device__ __forceinline__ void adam_elem(float2* __restrict__ z, float2* __restrict__ m, float* __restrict__ v,
                                          long long e, float2 g, float lr, float b1, float b2, float eps, float bc1,
                                          float bc2) {
  float2 zz = z[e], mm = m[e];
  float vv = v[e];
  adam_math(zz, mm, vv, g, lr, b1, b2, eps, bc1, bc2);
  z[e] = zz;
  m[e] = mm;
  v[e] = vv;
}

// I[j][u][v] = sum_k |A[j][k][perm(u)][perm(v)]|^2 / NP (natural order out).
template <class TL>
__global__ void k_modesum(const float2* __restrict__ A, float* __restrict__ I, int B, int K) {
  constexpr int N = TL::N;
  const long long total = (long long)B * TL::NP;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / TL::NP);
    const int q = (int)(e - (long long)j * TL::NP);
    const int u = q / N, v = q - u * N;
    const int p = TL::perm(u) * N + TL::perm(v);
    const float2* a = A + (size_t)j * K * TL::NP + p;
    float s = 0.f;
    for (int k = 0; k < K; ++k) s += cabs2(__ldg(a + (size_t)k * TL::NP));
    I[e] = s * (1.0f / (float)TL::NP);
  }
}

// Noise-model loss per pixel (noise.cuh) and the adjoint seed weight
// w = 2 l'(I) / NP, in spectral slot order.  Block partial sums of l go to
// partials[blockIdx.x] in FP64.
template <class TL>
__global__ void __launch_bounds__(kRedThreads) k_loss(const float2* __restrict__ A, const float* __restrict__ Iexp,
                                                      const int* __restrict__ idx, int npos, int B, int K,
                                                      int model, float eps, float c, float* __restrict__ w,
                                                      double* __restrict__ partials) {
  __shared__ double sh[32];
  constexpr int N = TL::N;
  const long long total = (long long)B * TL::NP;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / TL::NP);
    const int p = (int)(e - (long long)j * TL::NP);
    const int pu = p / N, pv = p - pu * N;
    const int jj = idx ? idx[j] : j;
    if (jj < 0 || jj >= npos) {  // flagged by the tile kernels; contributes nothing
      w[e] = 0.0f;
      continue;
    }
    const float E = __ldg(Iexp + (size_t)jj * TL::NP + TL::nat(pu) * N + TL::nat(pv));
    const float2* a = A + (size_t)j * K * TL::NP + p;
    float I = 0.f;
    for (int k = 0; k < K; ++k) I += cabs2(__ldg(a + (size_t)k * TL::NP));
    I *= 1.0f / (float)TL::NP;
    float l, dl;
    noise_model(model, eps, c, I, E, l, dl);
    w[e] = 2.0f * dl * (1.0f / (float)TL::NP);
    acc += (double)l;
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// Adjoint seed weight for an external cotangent dL/dI: w = 2 gI / NP
// (spectral slot order).
template <class TL>
__global__ void k_seed(const float* __restrict__ gI, int B, float* __restrict__ w) {
  constexpr int N = TL::N;
  const long long total = (long long)B * TL::NP;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / TL::NP);
    const int p = (int)(e - (long long)j * TL::NP);
    const int pu = p / N, pv = p - pu * N;
    w[e] = 2.0f * __ldg(gI + (size_t)j * TL::NP + TL::nat(pu) * N + TL::nat(pv)) * (1.0f / (float)TL::NP);
  }
}

}  // namespace ptycho
