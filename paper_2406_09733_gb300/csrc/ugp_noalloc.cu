// Free-flight sampling for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: plug-ins whose host application owns every device
// allocation, or real-time loops that must not hit the allocator.  ugp_sample_free_flight_noalloc is
// ugp_sample_free_flight with its scratch queue in a fixed device array that lives in the
// library image, so the caller passes only inputs and outputs.
#include <mutex>

#include "ugp_dense.cuh"
#include "ugp_trace.cuh"

namespace ugp {
namespace {

// Room for the queue of UGP_NOALLOC_MAX_RAYS rays: a 256-byte header, kDenseCols columns of
// 4-byte entries, each padded to 256 bytes, and 64 interval slots of the second finish pass (the
// layout of dense_queue_at; fewer slots than a workspace of that size gets, to keep the array
// small: the second pass then runs 64 warps).
constexpr int64_t kNoallocMaxRays = UGP_NOALLOC_MAX_RAYS;
constexpr int64_t kNoallocSlots = 64;
constexpr size_t kNoallocBytes = dense_queue_bytes(kNoallocMaxRays, kNoallocSlots);

static __device__ __align__(256) unsigned char g_ff_scratch[kNoallocBytes];

// Device address of g_ff_scratch per device, looked up once with that device current. The cache
// lives as long as the process: after cudaDeviceReset the library image is loaded again and the
// cached address is stale, so a process that resets a device must not call this entry point on
// that device afterwards.
struct ScratchSlot {
  int device;
  void* ptr;
};
static ScratchSlot g_slots[64];
static int g_nslots = 0;
static std::mutex g_mu;

ugp_status scratch_for_current_device(void** out) {
  int dev = 0;
  UGP_CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  for (int i = 0; i < g_nslots; ++i)
    if (g_slots[i].device == dev) {
      *out = g_slots[i].ptr;
      return UGP_OK;
    }
  if (g_nslots == 64) return fail(UGP_ERR_INVALID_ARG, "ugp_sample_free_flight_noalloc: too many devices");
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_ff_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
  g_slots[g_nslots++] = {dev, p};
  *out = p;
  return UGP_OK;
}

}  // namespace
}  // namespace ugp

using namespace ugp;

extern "C" ugp_status ugp_sample_free_flight_noalloc(const ugp_bvh* bvh, int64_t n_rays, const float* o3,
                                                     const float* d3, const float* t0, const float* t1,
                                                     const float* u, const float* u2,
                                                     const int32_t* exclude_prim, int32_t* prim_out,
                                                     float* t_u_out, float* t_spawn_out, uint8_t* status_out,
                                                     void* stream) {
  clear_error();
  ugp_status s = check_rays("ugp_sample_free_flight_noalloc", bvh, n_rays, o3, d3, t0, t1);
  if (s != UGP_OK) return s;
  if (n_rays > kNoallocMaxRays)
    return fail(UGP_ERR_INVALID_ARG, "ugp_sample_free_flight_noalloc: %lld rays exceed the fixed scratch of %lld rays",
                (long long)n_rays, (long long)kNoallocMaxRays);
  if (n_rays > 0 && (!u || !u2 || !prim_out || !t_u_out || !t_spawn_out))
    return fail(UGP_ERR_INVALID_ARG, "ugp_sample_free_flight_noalloc: NULL uniform or output array");
  if (n_rays == 0) return UGP_OK;
  if (dense_queue_bytes(n_rays, kNoallocSlots) > kNoallocBytes)
    return fail(UGP_ERR_INVALID_ARG, "ugp_sample_free_flight_noalloc: scratch layout mismatch");
  void* scratch = nullptr;
  s = scratch_for_current_device(&scratch);
  if (s != UGP_OK) return s;
  // The queue is laid out for n_rays entries inside the fixed array (without the per-ray slot
  // lists, so the dense pass collects its intervals by traversal); launch_free_flight clears
  // its counter on `stream` before use.
  return launch_free_flight(trace_scene(bvh), n_rays, o3, d3, t0, t1, u, u2, exclude_prim, prim_out, t_u_out,
                            t_spawn_out, status_out, scratch, false, static_cast<cudaStream_t>(stream),
                            kNoallocSlots);
}
