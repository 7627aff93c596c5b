// Continuous-batching server (placeholder until the serving runtime lands).
#include "errors.h"
#include "ptycho.h"

extern "C" {
int ptycho_server_create(size_t, int32_t, ptycho_server** out) {
  if (out) *out = nullptr;
  return perr(PTYCHO_EINVAL, "serving runtime not built yet");
}
int ptycho_server_destroy(ptycho_server*) { return PTYCHO_OK; }
int ptycho_submit(ptycho_server*, const ptycho_request*, uint64_t*) { return perr(PTYCHO_EINVAL, "no server"); }
int ptycho_poll(ptycho_server*, uint64_t, ptycho_status*, ptycho_result*) { return perr(PTYCHO_EINVAL, "no server"); }
int ptycho_wait(ptycho_server*, uint64_t, double) { return perr(PTYCHO_EINVAL, "no server"); }
int ptycho_release(ptycho_server*, uint64_t) { return perr(PTYCHO_EINVAL, "no server"); }
int ptycho_server_stats_get(ptycho_server*, ptycho_server_stats*) { return perr(PTYCHO_EINVAL, "no server"); }
}
