// Error reporting, version and statistics switches of the ugp C ABI.
#include <stdarg.h>
#include <stdio.h>

#include "ugp_internal.cuh"

namespace ugp {

static thread_local char g_err[512] = "";
static unsigned long long* g_counters = nullptr;

ugp_status fail(ugp_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

ugp_status cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_err, sizeof(g_err), "%s: %s (%d)", what, cudaGetErrorString(e), int(e));
  return UGP_ERR_CUDA;
}

void clear_error() { g_err[0] = 0; }

unsigned long long* trace_counters() { return g_counters; }

bool valid_bvh(const ugp_bvh* b) { return b != nullptr && b->magic == kBvhMagic; }

}  // namespace ugp

extern "C" {

const char* ugp_status_string(ugp_status s) {
  switch (s) {
    case UGP_OK: return "ok";
    case UGP_ERR_INVALID_ARG: return "invalid argument";
    case UGP_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case UGP_ERR_CUDA: return "CUDA error";
    case UGP_ERR_ITER_LIMIT: return "iteration limit reached";
    case UGP_ERR_TIMEOUT: return "timeout";
    case UGP_ERR_NOT_BUILT: return "BVH not built or released";
    case UGP_ERR_OVERFLOW: return "stack or buffer overflow";
  }
  return "unknown status";
}

const char* ugp_last_error(void) { return ugp::g_err; }

const char* ugp_version(void) { return "ugp 0.1 (sm_103a)"; }

ugp_status ugp_set_trace_counters(unsigned long long* counters) {
  ugp::g_counters = counters;
  return UGP_OK;
}

}  // extern "C"
