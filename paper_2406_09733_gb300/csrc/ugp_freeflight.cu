// Standalone free-flight query (ugp_sample_free_flight); the algorithm is in ugp_freeflight.cuh.
#include "ugp_dense.cuh"
#include "ugp_freeflight.cuh"

namespace ugp {
namespace {

template <bool STATS>
__global__ void __launch_bounds__(kFFBlock)
k_free_flight(TraceScene sc, int64_t n_rays, const float* __restrict__ o3, const float* __restrict__ d3,
              const float* __restrict__ t0a, const float* __restrict__ t1a, const float* __restrict__ ua,
              const float* __restrict__ u2a, const int32_t* __restrict__ excl,
              int32_t* __restrict__ prim_out, float* __restrict__ tu_out, float* __restrict__ tsp_out,
              uint8_t* __restrict__ st_out, unsigned long long* __restrict__ ctr, DenseQueue dq) {
  __shared__ FFSmem sm;
  const int64_t r = int64_t(blockIdx.x) * kFFBlock + threadIdx.x;
  if (r >= n_rays) return;
  Ctx c{sm, int(threadIdx.x), sc, make_ray(ld3(o3, r), ld3(d3, r)), __ldg(t0a + r), __ldg(t1a + r),
        excl ? __ldg(excl + r) : -1, 0u, 0u, UGP_RAY_OK,
        dq.list ? const_cast<int*>(dq.list) + r * kListCap : nullptr, 0};
  const float u = __ldg(ua + r), u2 = __ldg(u2a + r);
  const FFResult res = ff_sample(c, u, u2);
  if (res.pending) dense_push(dq, int(r), res.lo, res.hi, res.Flo, u, u2, c.ray.o, c.ray.d, c.t0, c.t1, c.ex, res.nlist);
  prim_out[r] = res.prim;
  tu_out[r] = res.t_u;
  tsp_out[r] = res.t_spawn;
  if (st_out) st_out[r] = c.st;
  if (STATS) add_counters(ctr, c.n_nodes, c.n_prims, 1u, 1u, res.pending ? 1u : 0u);
}

}  // namespace
ugp_status launch_free_flight(const TraceScene& sc, int64_t n, const float* o3, const float* d3,
                              const float* t0, const float* t1, const float* u, const float* u2,
                              const int32_t* excl, int32_t* prim, float* tu, float* tsp, uint8_t* st,
                              void* workspace, bool with_lists, cudaStream_t stream) {
  const unsigned grid = unsigned((n + kFFBlock - 1) / kFFBlock);
  unsigned long long* ctr = trace_counters();
  DenseQueue dq = dense_queue_at(workspace, n);
  if (with_lists) dq.list = reinterpret_cast<const int*>(static_cast<char*>(workspace) + dense_queue_bytes(n));
  UGP_CUDA_CHECK(cudaMemsetAsync(dq.count, 0, sizeof(int), stream));
  prof_begin(kStQuery, stream);
  if (ctr)
    k_free_flight<true><<<grid, kFFBlock, 0, stream>>>(sc, n, o3, d3, t0, t1, u, u2, excl, prim, tu, tsp, st, ctr, dq);
  else
    k_free_flight<false><<<grid, kFFBlock, 0, stream>>>(sc, n, o3, d3, t0, t1, u, u2, excl, prim, tu, tsp, st, ctr, dq);
  prof_end(kStQuery, stream);
  UGP_CUDA_CHECK(cudaGetLastError());
  return launch_dense(sc, dq, prim, tu, tsp, st, 0, ctr, nullptr, stream);
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
