// Identity of the current CUDA context, for state the library keeps per
// context (device-symbol addresses, constant tables): a __device__ variable
// exists once per context, so a non-primary context on the same device, or
// the primary context re-created after cudaDeviceReset, needs its own.
#pragma once

namespace ptycho {

// *id = the unique id (cuCtxGetId, never reused within a process) of the
// context current on the calling thread, or 0 when none is current.
// PTYCHO_OK, or PTYCHO_ECUDA (message set) when the driver cannot tell.
int current_context_id(unsigned long long* id);

}  // namespace ptycho
