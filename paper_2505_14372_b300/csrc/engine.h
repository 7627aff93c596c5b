// Host-side table of launchers for one window size (one tile shape).
#pragma once
#include <cuda_runtime.h>

#include "launch.h"

namespace ptycho {

struct EngineOps {
  int N, G, T, R1, R2;
  size_t smem;
  cudaError_t (*probe_spectrum)(const float2* P, float2* Phat, int K, cudaStream_t s);
  // variant: Variant (launch.h); engines without all variants return
  // cudaErrorNotSupported for the others (see has_variants)
  cudaError_t (*forward)(const LaunchArgs& L, int clusters, bool store, int variant, cudaStream_t s);
  cudaError_t (*adjoint)(const LaunchArgs& L, int clusters, bool store, int variant, cudaStream_t s);
  cudaError_t (*probe_grad)(const float2* gPhat, float2* gP, int K, int acc, cudaStream_t s);
  cudaError_t (*fft_debug)(const float2* in, float2* out, int count, int dir, cudaStream_t s);
  cudaError_t (*modesum)(const float2* A, float* I, int B, int K, cudaStream_t s);
  cudaError_t (*loss)(const float2* A, const float* Iexp, const int* idx, int npos, int B, int K, int model,
                      float eps, float c, float* w, double* partials, int nblocks, cudaStream_t s);
  cudaError_t (*seed)(const float* gI, int B, float* w, cudaStream_t s);
  // resident clusters of the forward / adjoint kernels on the current device
  int (*resident_clusters)(bool adjoint, bool store, int variant);
  // position-major loss + adjoint (entry waves recomputed; `clusters` clusters)
  cudaError_t (*adjoint_pos)(const LaunchArgs& L, const PosArgs& F, int clusters, int variant, cudaStream_t s);
  int (*resident_pos)(int variant);
  // bounded exchange waits of this tile's kernels that gave up since the
  // last call (read and cleared)
  unsigned (*take_exchange_timeouts)();
  // launches the bounded-wait self-test (one cluster whose waits run out)
  cudaError_t (*exchange_probe)(cudaStream_t s);
  bool has_variants;  // reduced-precision waves and ePIE are instantiated
  // fused end of a gradient step (single-CTA tiles; cudaErrorNotSupported
  // otherwise) and its grid for an object of nO elements and K modes (0:
  // not available for this tile)
  cudaError_t (*step_tail)(const TailArgs& A, int blocks, cudaStream_t s);
  int (*tail_blocks)(long long nO, int K);
  // checked build (check.cuh): index-check bits of this tile's kernels since
  // the last call, read and cleared (always 0 in the normal build)
  unsigned (*take_check_bits)();
};

const EngineOps* engine_64();
const EngineOps* engine_128();
const EngineOps* engine_192();
const EngineOps* engine_256();

// tensor-core DFT variants (mode 1 TF32x3, 2 BF16x3, 3 TF32x1, 4 BF16x6), 192x192 only
const EngineOps* engine_192_tc(int mode);

inline const EngineOps* engine_for(int N, int dft = 0) {
  if (dft != 0) return N == 192 ? engine_192_tc(dft) : nullptr;
  switch (N) {
    case 64: return engine_64();
    case 128: return engine_128();
    case 192: return engine_192();
    case 256: return engine_256();
    default: return nullptr;
  }
}

// elementwise launchers (elementwise.cu)
cudaError_t launch_sumsq(const float2* g, long long n, double* partials, int nblocks, cudaStream_t s);
cudaError_t launch_finalize(const double* partials, int n0, int n1, double* out, int sqrt_second,
                            cudaStream_t s);
cudaError_t launch_regularize(const float2* O, float2* gO, int S, int H, int W, const float2* P, float2* gP,
                              long long nP, float l2, float tik, float lay, float l2p, float tv, float tvl,
                              float eta, double* partials, int nblocks, cudaStream_t s);
// bcd (device, optional): bias corrections written by launch_adam_count, used instead of bc1, bc2;
// norm_partials (optional): kNormBlocks FP64 partials of |g|^2 (the update then runs on that grid)
cudaError_t launch_adam(float2* z, float2* m, float* v, const float2* g, long long n, float lr, float b1,
                        float b2, float eps, float bc1, float bc2, cudaStream_t s, const float* bcd = nullptr,
                        double* norm_partials = nullptr);
cudaError_t launch_adam_count(long long* t, float b1, float b2, float* bc, cudaStream_t s);
// order[0, L.total): the launch's positions sorted by (problem, Hilbert index
// of the window origin), the processing order of the position-major kernel
cudaError_t launch_locality_order(const LaunchArgs& L, int* order, cudaStream_t s);
cudaError_t launch_slice_absmax(const float2* O, int S, long long per_slice, unsigned* omax, cudaStream_t s);
cudaError_t launch_axpy(float2* z, const float2* g, long long n, float a, cudaStream_t s);
cudaError_t launch_transmission(const float2* O, int S, int H, int W, int N, const float* pos, const int* idx, int npos,
                                int B, const double* num, const double* den, float gamma, float* T, cudaStream_t s);
cudaError_t launch_divide(const float2* num, const float* den, const float* den_prev, float reg, long long n,
                          long long period, float2* out, cudaStream_t s);
cudaError_t launch_weighted_update(float2* z, const float2* dz, const float* aw, const float* w, float beta, long long n,
                                   long long period, cudaStream_t s);
cudaError_t launch_add(float* y, const float* x, long long n, cudaStream_t s);
// fixed-order sums of the per-position gradients of the deterministic
// variant: gO [S][H][W] += object patches [B][S][N][N] of the group's
// positions pos[idx[j]] (index order), gPhat [K][N][N] += pgrad [B][K][N][N]
cudaError_t launch_det_reduce(const float2* patches, const float2* pgrad, const float* pos, const int* idx, int npos,
                              int B, int S, int K, int H, int W, int N, float2* gO, float2* gPhat, cudaStream_t s);

// process-wide count of kernels this library has launched (engine_impl /
// elementwise launchers bump it once per launch)
void count_launch();

constexpr int kLossBlocks = 1184;  // 148 SMs x 8 resident reduction blocks
constexpr int kNormBlocks = 592;

}  // namespace ptycho
