// Internal interface between the context runtime (api.cu) and the serving
// runtime (server.cpp).  Not part of the C-ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ptycho.h"

namespace ptycho {

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

int ctx_create_shared_slots(const ptycho_geom* geom, int max_batch, ptycho_ctx** out);
size_t ctx_device_bytes(const ptycho_ctx* c);
int resident_slots(int N);
int step_batch(const StepJob* jobs, int n, float2* slots, int nslots, long long slot_stride, unsigned* status,
               cudaStream_t s);

}  // namespace ptycho
