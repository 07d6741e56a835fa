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

// ---- launch accounting and event timing
static unsigned long long g_launches = 0;
struct Prof {
  bool on = false;
  int max_records = 0, used = 0;
  bool overflow = false;
  cudaEvent_t* ev = nullptr;  // 2 * capacity events, created lazily
  int capacity = 0;
  int* stage = nullptr;
  long long launches[UGP_PROFILE_STAGES] = {0};
  int open_slot = -1;
};
static Prof g_prof;

static bool g_prof_suspended = false;

void prof_suspend(bool on) { g_prof_suspended = on; }

void add_launches(int stage, int64_t n) {
  g_launches += (unsigned long long)n;
  if (g_prof.on && stage >= 0 && stage < UGP_PROFILE_STAGES) g_prof.launches[stage] += n;
}

void prof_begin(int stage, cudaStream_t s) {
  (void)stage;
  if (g_prof_suspended || !g_prof.on) return;
  if (g_prof.used >= g_prof.max_records) {
    g_prof.overflow = true;
    g_prof.open_slot = -1;
    return;
  }
  const int i = g_prof.used;
  if (i >= g_prof.capacity) {
    g_prof.open_slot = -1;
    g_prof.overflow = true;
    return;
  }
  cudaEventRecord(g_prof.ev[2 * i], s);
  g_prof.open_slot = i;
}

void prof_end(int stage, cudaStream_t s, int n_kernels) {
  if (g_prof_suspended) return;
  g_launches += (unsigned long long)n_kernels;
  if (!g_prof.on) return;
  g_prof.launches[stage] += n_kernels;
  const int i = g_prof.open_slot;
  if (i < 0) return;
  cudaEventRecord(g_prof.ev[2 * i + 1], s);
  g_prof.stage[i] = stage;
  g_prof.used = i + 1;
  g_prof.open_slot = -1;
}

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

int64_t ugp_launch_count(void) { return int64_t(ugp::g_launches); }

ugp_status ugp_profile_begin(int32_t max_records) {
  using ugp::g_prof;
  ugp::clear_error();
  if (max_records <= 0 || max_records > (1 << 22))
    return ugp::fail(UGP_ERR_INVALID_ARG, "ugp_profile_begin: max_records out of range");
  if (max_records > g_prof.capacity) {
    cudaEvent_t* ev = new cudaEvent_t[2 * size_t(max_records)];
    int* st = new int[size_t(max_records)];
    for (int i = 0; i < 2 * g_prof.capacity; ++i) ev[i] = g_prof.ev[i];
    for (int i = 2 * g_prof.capacity; i < 2 * max_records; ++i) {
      const cudaError_t e = cudaEventCreate(&ev[i]);
      if (e != cudaSuccess) {
        for (int j = 2 * g_prof.capacity; j < i; ++j) cudaEventDestroy(ev[j]);
        delete[] ev;
        delete[] st;
        return ugp::cuda_fail(e, "cudaEventCreate");
      }
    }
    delete[] g_prof.ev;
    delete[] g_prof.stage;
    g_prof.ev = ev;
    g_prof.stage = st;
    g_prof.capacity = max_records;
  }
  g_prof.on = true;
  g_prof.max_records = max_records;
  g_prof.used = 0;
  g_prof.overflow = false;
  g_prof.open_slot = -1;
  for (long long& l : g_prof.launches) l = 0;
  return UGP_OK;
}

ugp_status ugp_profile_end(double* ms_out, int64_t* launches_out) {
  using ugp::g_prof;
  ugp::clear_error();
  if (!g_prof.on) return ugp::fail(UGP_ERR_INVALID_ARG, "ugp_profile_end: profiling is not on");
  g_prof.on = false;
  double ms[UGP_PROFILE_STAGES] = {0};
  for (int i = 0; i < g_prof.used; ++i) {
    const cudaError_t e = cudaEventSynchronize(g_prof.ev[2 * i + 1]);
    if (e != cudaSuccess) return ugp::cuda_fail(e, "cudaEventSynchronize");
    float t = 0.f;
    const cudaError_t e2 = cudaEventElapsedTime(&t, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]);
    if (e2 != cudaSuccess) return ugp::cuda_fail(e2, "cudaEventElapsedTime");
    ms[g_prof.stage[i]] += t;
  }
  for (int k = 0; k < UGP_PROFILE_STAGES; ++k) {
    if (ms_out) ms_out[k] = ms[k];
    if (launches_out) launches_out[k] = g_prof.launches[k];
  }
  if (g_prof.overflow) return ugp::fail(UGP_ERR_OVERFLOW, "ugp_profile_end: more launches than max_records");
  return UGP_OK;
}

ugp_status ugp_set_trace_counters(unsigned long long* counters) {
  ugp::g_counters = counters;
  return UGP_OK;
}

}  // extern "C"
