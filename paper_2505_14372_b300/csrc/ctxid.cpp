// current_context_id: the driver's cuCtxGetCurrent / cuCtxGetId, reached
// through the runtime's driver entry points (no link against libcuda).
#include "ctxid.h"

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "errors.h"
#include "ptycho.h"

namespace ptycho {

namespace {
std::once_flag g_once;
PFN_cuCtxGetCurrent_v4000 g_get_current = nullptr;
PFN_cuCtxGetId_v12000 g_get_id = nullptr;

void resolve() {
  cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
  void* f1 = nullptr;
  void* f2 = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) == cudaSuccess &&
      cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
      q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess && f1 && f2) {
    g_get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
    g_get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
  } else {
    cudaGetLastError();
  }
}
}  // namespace

int current_context_id(unsigned long long* id) {
  std::call_once(g_once, resolve);
  if (!g_get_current || !g_get_id) return perr(PTYCHO_ECUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not available");
  CUcontext ctx = nullptr;
  if (g_get_current(&ctx) != CUDA_SUCCESS) return perr(PTYCHO_ECUDA, "cuCtxGetCurrent failed");
  *id = 0;
  if (ctx && g_get_id(ctx, id) != CUDA_SUCCESS) return perr(PTYCHO_ECUDA, "cuCtxGetId failed");
  return PTYCHO_OK;
}

}  // namespace ptycho
