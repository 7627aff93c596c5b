// Internal interface between the context runtime (api.cu) and the serving
// runtime (server.cpp).  Not part of the C-ABI.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

#include "ptycho.h"

// 1 in the checked build (check.cuh)
#ifndef PTYCHO_CHECKED
#define PTYCHO_CHECKED 0
#endif

namespace ptycho {

// Named NVTX range over the lifetime of the object: the library's entry
// points and kernel launches show by name on the timelines of profilers
// that collect NVTX (a pointer check when none is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Host checks of a geometry (dimensions, window size, DFT mode, physics
// parameters, noise model, waves mode, storage format, object size);
// PTYCHO_OK or PTYCHO_EINVAL with the thread-local message set.
int validate_geom(const ptycho_geom* g);

// One problem's gradient step inside a batched launch (device pointers).
struct StepJob {
  ptycho_ctx* c;
  float2* O;
  float2* P;
  float2* mO;
  float* vO;
  float2* mP;
  float* vP;
  int64_t t;            // Adam step count after this step (>= 1)
  ptycho_opt opt;
  const float* pos;     // [n_pos][2]
  const float* Iexp;    // [n_pos][N][N]
  int n_pos;
  const int* idx;       // [B] group
  int B;
  double* stats;        // device double[2]: loss, gradient norm
};

// Scratch of the position-major loss + adjoint kernel shared by the
// problems of one window size: per cluster, the entry waves of up to kmodes
// modes and smax + 1 waves each, the far fields of up to kmodes modes and
// the mode-summed intensity.
struct PosScratch {
  char* slots = nullptr;     // [clusters][slot_bytes]
  long long slot_bytes = 0;
  float2* A = nullptr;       // [clusters][kmodes NP]
  float* I = nullptr;        // [clusters][NP]
  int* order = nullptr;      // [order_cap] processing order of a launch's positions
  unsigned* queue = nullptr; // [2] work queue of a launch (zeroed once by the owner)
  int clusters = 0, kmodes = 0, smax = 0, order_cap = 0;
};
// Bytes of a PosScratch for window N (clusters = resident_slots(N)).
size_t pos_scratch_bytes(int N, int kmodes, int smax);
// Carves a PosScratch out of one device allocation of pos_scratch_bytes.
PosScratch pos_scratch_at(char* base, int N, int kmodes, int smax);

int ctx_create_shared_slots(const ptycho_geom* geom, int max_batch, ptycho_ctx** out);
size_t ctx_device_bytes(const ptycho_ctx* c);
int resident_slots(int N);
// One gradient step for each job (all of one window size).  With `ps` (and
// every job's modes and slices within it) one position-major launch covers
// all jobs; otherwise one forward and one recomputing adjoint launch over
// their (position, mode) items, with `slots` as the adjoint's scratch.
// *tile_launches: the tile-kernel launches the step made (1 or 2).
int step_batch(const StepJob* jobs, int n, float2* slots, int nslots, long long slot_stride, const PosScratch* ps,
               unsigned* status, cudaStream_t s, int* tile_launches);

}  // namespace ptycho
