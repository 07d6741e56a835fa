// Standalone free-flight query (ugp_sample_free_flight); the algorithm is in ugp_freeflight.cuh.
#include "ugp_dense.cuh"
#include "ugp_freeflight.cuh"

namespace ugp {
namespace {

// Rays of a standalone query: caller arrays.
template <bool STATS>
struct ArrayScanSrc {
  TraceScene sc;
  int64_t n;
  const float *o3, *d3, *t0a, *t1a, *ua, *u2a;
  const int32_t* excl;
  int32_t* prim_out;
  float *tu_out, *tsp_out;
  uint8_t* st_out;
  unsigned long long* ctr;
  DenseQueue dq;
  int cur;
  float u, u2;
  __device__ int count() const { return int(n); }
  __device__ TraceScene scene() const { return sc; }
  __device__ bool begin(int i, ScanState& s, float& uo) {
    cur = i;
    s.ray = make_ray(ld3(o3, i), ld3(d3, i));
    s.t0 = __ldg(t0a + i);
    s.t1 = __ldg(t1a + i);
    s.ex = excl ? __ldg(excl + i) : -1;
    s.list = dq.list ? const_cast<int*>(dq.list) + size_t(i) * kListCap : nullptr;
    u = __ldg(ua + i);
    u2 = __ldg(u2a + i);
    uo = u;
    return true;
  }
  __device__ void finish(const ScanState& s, const FFResult& r) {
    if (r.pending) dense_push(dq, cur, cur, r.lo, r.hi, r.Flo, u, u2, s.ray.o, s.ray.d, s.t0, s.t1, s.ex, r.nlist);
    else dense_none(dq, cur);
    prim_out[cur] = r.prim;
    tu_out[cur] = r.t_u;
    tsp_out[cur] = r.t_spawn;
    if (st_out) st_out[cur] = s.st;
    if (STATS) add_counters(ctr, s.n_nodes, s.n_prims, 1u, 1u, r.pending ? 1u : 0u);
  }
};

template <bool STATS>
__global__ void __launch_bounds__(kFFBlock, kFFBlocksPerSM)
k_free_flight(TraceScene sc, int64_t n_rays, const float* __restrict__ o3, const float* __restrict__ d3,
              const float* __restrict__ t0a, const float* __restrict__ t1a, const float* __restrict__ ua,
              const float* __restrict__ u2a, const int32_t* __restrict__ excl,
              int32_t* __restrict__ prim_out, float* __restrict__ tu_out, float* __restrict__ tsp_out,
              uint8_t* __restrict__ st_out, unsigned long long* __restrict__ ctr, DenseQueue dq, int* next) {
  __shared__ FFSmem sm;
  ArrayScanSrc<STATS> src{sc, n_rays, o3, d3, t0a, t1a, ua, u2a, excl, prim_out, tu_out, tsp_out, st_out, ctr, dq,
                          0, 0.f, 0.f};
  scan_persistent(sm, src, next);
}

}  // namespace

int scan_grid(const void* kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kFFBlock, 0) != cudaSuccess || per_sm <= 0)
    per_sm = 1;
  return (sms > 0 ? sms : 1) * per_sm;
}

ugp_status launch_free_flight(const TraceScene& sc, int64_t n, const float* o3, const float* d3,
                              const float* t0, const float* t1, const float* u, const float* u2,
                              const int32_t* excl, int32_t* prim, float* tu, float* tsp, uint8_t* st,
                              void* workspace, bool with_lists, cudaStream_t stream, int64_t slots) {
  unsigned long long* ctr = trace_counters();
  if (slots < 0) slots = big_slots(n);
  DenseQueue dq = dense_queue_at(workspace, n, slots);
  if (with_lists)
    dq.list = reinterpret_cast<const int*>(static_cast<char*>(workspace) + dense_queue_bytes(n, slots));
  int* next = dq.count + 1;  // the scan's ray counter, in the queue header next to the queue length
  UGP_CUDA_CHECK(cudaMemsetAsync(dq.count, 0, 2 * sizeof(int), stream));
  const void* kern = ctr ? (const void*)k_free_flight<true> : (const void*)k_free_flight<false>;
  const int64_t need = (n + kFFBlock - 1) / kFFBlock;
  const int cap = scan_grid(kern);
  const unsigned grid = unsigned(need < cap ? need : cap);
  prof_begin(kStQuery, stream);
  if (ctr)
    k_free_flight<true><<<grid, kFFBlock, 0, stream>>>(sc, n, o3, d3, t0, t1, u, u2, excl, prim, tu, tsp, st, ctr, dq,
                                                      next);
  else
    k_free_flight<false><<<grid, kFFBlock, 0, stream>>>(sc, n, o3, d3, t0, t1, u, u2, excl, prim, tu, tsp, st, ctr, dq,
                                                       next);
  prof_end(kStQuery, stream);
  UGP_CUDA_CHECK(cudaGetLastError());
  return launch_dense(sc, dq, n, nullptr, n, prim, tu, tsp, st, 0, ctr, nullptr, stream);
}

}  // namespace ugp

using namespace ugp;

extern "C" ugp_status ugp_sample_free_flight(const ugp_bvh* bvh, int64_t n_rays, const float* o3,
                                             const float* d3, const float* t0, const float* t1,
                                             const float* u, const float* u2, const int32_t* exclude_prim,
                                             int32_t* prim_out, float* t_u_out, float* t_spawn_out,
                                             uint8_t* status_out, void* workspace, size_t workspace_bytes,
                                             void* stream) {
  clear_error();
  ugp_status s = check_rays("ugp_sample_free_flight", bvh, n_rays, o3, d3, t0, t1);
  if (s != UGP_OK) return s;
  if (n_rays > 0 && (!u || !u2 || !prim_out || !t_u_out || !t_spawn_out))
    return fail(UGP_ERR_INVALID_ARG, "ugp_sample_free_flight: NULL uniform or output array");
  if (n_rays == 0) return UGP_OK;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(UGP_ERR_INVALID_ARG, "ugp_sample_free_flight: workspace must be non-NULL and 256-byte aligned");
  if (n_rays > (int64_t(1) << 31) - 1)
    return fail(UGP_ERR_INVALID_ARG, "ugp_sample_free_flight: at most 2^31 - 1 rays per call");
  const size_t need = dense_queue_bytes(n_rays) + slot_list_bytes(n_rays);
  if (workspace_bytes < need)
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_sample_free_flight: need %zu bytes, got %zu", need, workspace_bytes);
  return launch_free_flight(trace_scene(bvh), n_rays, o3, d3, t0, t1, u, u2, exclude_prim, prim_out, t_u_out,
                            t_spawn_out, status_out, workspace, true, static_cast<cudaStream_t>(stream));
}

extern "C" size_t ugp_sample_free_flight_workspace_size(int64_t n_rays) {
  if (n_rays < 0 || n_rays > (int64_t(1) << 31) - 1) return 0;
  return dense_queue_bytes(n_rays) + slot_list_bytes(n_rays);
}
