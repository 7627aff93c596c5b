// Allocation-free forward model: ptycho_forward_static.
//
// Some callers cannot allocate device memory.  A live-reconstruction loop
// fed by the detector must not stall in cudaMalloc, which takes driver locks
// and can synchronise the whole device.  An application may hand all device
// memory to its own pool at start-up and forbid any other allocation.  A
// plug-in may run under a host framework whose contract forbids allocating.
// Such callers cannot create a ptycho_ctx, because its scratch arena and
// tables are cudaMalloc'd.  This entry point needs no context.  Its scratch
// (probe spectra, far fields, the propagator chirp and a status word) lives
// in one file-scope __device__ array of fixed size, and the caller passes
// only inputs and outputs.
//
// The array is a property of the loaded library: every GPU that loads it
// holds kStaticScratchBytes until the process exits.  All calls on a device
// share it, so calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it; callers must order them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "engine.h"
#include "errors.h"
#include "launch.h"
#include "ptycho.h"

namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device, resolved once per device
// (cudaGetSymbolAddress with that device current): in host code the array's
// name is only a stand-in, not a device address.
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return perr(PTYCHO_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return perr(PTYCHO_ECUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                    cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PTYCHO_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Separable Fresnel chirp per gap in spectral slot order (the same table
// ptycho_create builds on the host): phase in turns formed and reduced in
// FP64 before the sincos.
__global__ void k_static_chirp_table(float2* Hc, const double* dz_dev, int gaps, int N, int R1, int R2, double lam,
                                     double dx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= gaps * N) return;
  const int s = i / N, p = i % N;
  const int n = p / R2 + R1 * (p % R2);
  const double f = n < (N + 1) / 2 ? n : n - N;
  double t = lam * dz_dev[s] * f * f / (2.0 * (double)N * N * dx * dx);
  t -= rint(t);
  double sn, cs;
  sincospi(-2.0 * t, &sn, &cs);
  Hc[i] = make_float2((float)cs, (float)sn);
}

}  // namespace

extern "C" int ptycho_forward_static(const ptycho_geom* g, const ptycho_c64* O, const ptycho_c64* P, const float* pos,
                                     int32_t B, float* I_out, ptycho_stream stream) {
  if (!g) return perr(PTYCHO_EINVAL, "geometry is NULL");
  const ptycho::EngineOps* ops = ptycho::engine_for(g->h, g->dft);
  if (!ops || g->h != g->w) return perr(PTYCHO_EINVAL, "window must be square with N in {64, 128, 192, 256}");
  if (g->S < 1 || g->K < 1 || g->H < g->h || g->W < g->w || !(g->dx > 0) || !(g->lambda > 0) ||
      (g->S > 1 && !g->dz))
    return perr(PTYCHO_EINVAL, "bad geometry");
  if (B < 0) return perr(PTYCHO_EINVAL, "B < 0");
  if (B == 0) return PTYCHO_OK;
  if (!O || !P || !pos || !I_out) return perr(PTYCHO_EINVAL, "NULL array argument");
  const int N = g->h, K = g->K, S = g->S;
  const size_t NP = (size_t)N * N;
  // scratch layout: status | dz (FP64) | chirp | probe spectra | far fields
  const size_t off_dz = 256;
  const size_t off_hc = off_dz + align256((size_t)std::max(S - 1, 1) * 8);
  const size_t off_ph = off_hc + align256((size_t)std::max(S - 1, 1) * N * 8);
  const size_t off_a = off_ph + align256((size_t)K * NP * 8);
  const size_t need = off_a + align256((size_t)B * K * NP * 8);
  if (need > kStaticScratchBytes)
    return perr(PTYCHO_EINVAL, "problem needs " + std::to_string(need) + " bytes of scratch; the static scratch of "
                                   "ptycho_forward_static holds " + std::to_string(kStaticScratchBytes) +
                                   " (use ptycho_forward with a context instead)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return perr(PTYCHO_ECUDA, "no CUDA device");
  }
  void* base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc) return rc;
  unsigned char* sc = static_cast<unsigned char*>(base);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* status = reinterpret_cast<unsigned*>(sc);
  float2* Hc = reinterpret_cast<float2*>(sc + off_hc);
  float2* Phat = reinterpret_cast<float2*>(sc + off_ph);
  float2* A = reinterpret_cast<float2*>(sc + off_a);
  // the status word starts at zero; far fields of skipped (out-of-bounds)
  // items read as zero rather than as a previous call's values
  if (cudaMemsetAsync(status, 0, sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(A, 0, (size_t)B * K * NP * 8, s) != cudaSuccess) {
    cudaGetLastError();
    return perr(PTYCHO_ECUDA, "cudaMemsetAsync failed");
  }
  if (S > 1) {
    if (cudaMemcpyAsync(sc + off_dz, g->dz, (size_t)(S - 1) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      return perr(PTYCHO_ECUDA, "copy of the slice gaps failed");
    }
    const int n = (S - 1) * N;
    k_static_chirp_table<<<(n + 255) / 256, 256, 0, s>>>(Hc, reinterpret_cast<const double*>(sc + off_dz), S - 1, N,
                                                          ops->R1, ops->R2, g->lambda, g->dx);
    ptycho::count_launch();
  }
  int blT = -1;
  if (g->bandlimit > 0) {
    const double x = g->bandlimit * (double)g->h * (double)g->w * 0.5;
    blT = (int)std::min(std::floor(std::floor(x * x) / ((double)N * N)), 2.0e9);
  }
  cudaError_t e = ops->probe_spectrum(reinterpret_cast<const float2*>(P), Phat, K, s);
  if (e == cudaSuccess) {
    ptycho::LaunchArgs la{};
    ptycho::ProblemDesc& d = la.d[0];
    d.O = reinterpret_cast<const float2*>(O);
    d.Phat = Phat;
    d.pos = pos;
    d.idx = nullptr;
    d.Hc = Hc;
    d.A = A;
    d.S = S;
    d.K = K;
    d.H = g->H;
    d.W = g->W;
    d.B = B;
    d.npos = B;
    d.blT = blT;
    d.item0 = 0;
    la.nd = 1;
    la.total = B * K;
    la.status = status;
    e = ops->forward(la, std::min(B * K, ops->resident_clusters(false, false, ptycho::kVarF32)), false,
                     ptycho::kVarF32, s);
  }
  if (e == cudaSuccess) e = ops->modesum(A, I_out, B, K, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return perr(PTYCHO_ECUDA, std::string("forward launch failed: ") + cudaGetErrorString(e));
  }
  return PTYCHO_OK;
}
