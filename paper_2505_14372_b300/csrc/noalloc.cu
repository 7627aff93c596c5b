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
// only inputs and outputs (and, optionally, a device word for the status).
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

#include "ctxid.h"
#include "engine.h"
#include "errors.h"
#include "internal.h"
#include "launch.h"
#include "ptycho.h"

namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;  // 32 MiB
constexpr int kMaxStaticGaps = 64;                 // S <= 65 slices
constexpr int kAddrCache = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per CUDA context.  In host code the
// array's name is only a stand-in, not a device address; a __device__ array
// exists once per context (a non-primary context on the same device, or the
// primary context re-created after cudaDeviceReset, holds its own copy), so
// the address is resolved with cudaGetSymbolAddress once per context, with
// that context current, and cached under the context's unique id
// (current_context_id, never reused within a process).
struct AddrEntry {
  unsigned long long ctx_id;
  void* addr;
};
AddrEntry g_addr[kAddrCache] = {};
int g_addr_next = 0;
std::mutex g_addr_mu;

int resolve_symbol(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return perr(PTYCHO_ECUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                  cudaGetErrorString(e));
  }
  *out = p;
  return PTYCHO_OK;
}

// Address of the scratch in the current context (resolving it, and making
// the runtime bind its primary context, on the context's first call).
int scratch_address(void** out) {
  std::lock_guard<std::mutex> lk(g_addr_mu);
  unsigned long long id = 0;
  int rc = ptycho::current_context_id(&id);
  if (rc) return rc;
  void* fresh = nullptr;
  if (id == 0) {
    // no context bound yet: the runtime binds the device's primary context
    // while resolving the symbol
    if ((rc = resolve_symbol(&fresh))) return rc;
    if ((rc = ptycho::current_context_id(&id))) return rc;
    if (id == 0) return perr(PTYCHO_ECUDA, "no current CUDA context");
  }
  for (const AddrEntry& a : g_addr)
    if (a.addr && a.ctx_id == id) {
      *out = a.addr;
      return PTYCHO_OK;
    }
  if (!fresh && (rc = resolve_symbol(&fresh))) return rc;
  g_addr[g_addr_next] = {id, fresh};
  g_addr_next = (g_addr_next + 1) % kAddrCache;
  *out = fresh;
  return PTYCHO_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// The slice gaps travel by value in the kernel's parameters, so a call copies
// nothing from host memory.
struct Gaps {
  double dz[kMaxStaticGaps];
};

// Separable Fresnel chirp per gap in spectral slot order (the same table
// ptycho_create builds on the host): phase in turns formed and reduced in
// FP64 before the sincos.
__global__ void k_static_chirp_table(float2* Hc, const __grid_constant__ Gaps gaps, int ngaps, int N, int R1, int R2,
                                     double lam, double dx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ngaps * N) return;
  const int s = i / N, p = i % N;
  const int n = p / R2 + R1 * (p % R2);
  const double f = n < (N + 1) / 2 ? n : n - N;
  double t = lam * gaps.dz[s] * f * f / (2.0 * (double)N * N * dx * dx);
  t -= rint(t);
  double sn, cs;
  sincospi(-2.0 * t, &sn, &cs);
  Hc[i] = make_float2((float)cs, (float)sn);
}

}  // namespace

extern "C" int ptycho_forward_static(const ptycho_geom* g, const ptycho_c64* O, const ptycho_c64* P, const float* pos,
                                     int32_t B, float* I_out, uint32_t* status_out, ptycho_stream stream) {
  ptycho::Range range("ptycho_forward_static");
  int rc = ptycho::validate_geom(g);
  if (rc) return rc;
  if (g->S - 1 > kMaxStaticGaps)
    return perr(PTYCHO_EINVAL, "ptycho_forward_static takes at most " + std::to_string(kMaxStaticGaps + 1) +
                                   " slices (use ptycho_forward with a context instead)");
  const ptycho::EngineOps* ops = ptycho::engine_for(g->h, g->dft);
  if (B < 0) return perr(PTYCHO_EINVAL, "B < 0");
  if (B == 0) return PTYCHO_OK;
  if (!O || !P || !pos || !I_out) return perr(PTYCHO_EINVAL, "NULL array argument");
  const int N = g->h, K = g->K, S = g->S;
  const size_t NP = (size_t)N * N;
  // scratch layout: status | chirp | probe spectra | far fields
  const size_t off_hc = 256;
  const size_t off_ph = off_hc + align256((size_t)std::max(S - 1, 1) * N * 8);
  const size_t off_a = off_ph + align256((size_t)K * NP * 8);
  const size_t need = off_a + align256((size_t)B * K * NP * 8);
  if (need > kStaticScratchBytes)
    return perr(PTYCHO_EINVAL, "problem needs " + std::to_string(need) + " bytes of scratch; the static scratch of "
                                   "ptycho_forward_static holds " + std::to_string(kStaticScratchBytes) +
                                   " (use ptycho_forward with a context instead)");
  void* base = nullptr;
  if ((rc = scratch_address(&base))) return rc;
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
    Gaps gaps{};
    for (int i = 0; i + 1 < S; ++i) gaps.dz[i] = g->dz[i];
    const int n = (S - 1) * N;
    k_static_chirp_table<<<(n + 255) / 256, 256, 0, s>>>(Hc, gaps, S - 1, N, ops->R1, ops->R2, g->lambda, g->dx);
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
  if (e == cudaSuccess && status_out) e = cudaMemcpyAsync(status_out, status, sizeof(unsigned), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return perr(PTYCHO_ECUDA, std::string("forward launch failed: ") + cudaGetErrorString(e));
  }
  return PTYCHO_OK;
}
