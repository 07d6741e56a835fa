// Launch interface of the tracing kernels (shared by the C entry points and the renderer).
#pragma once

#include "ugp_internal.cuh"

namespace ugp {

constexpr int kTrBlock = 128;      // transmittance: threads per block
constexpr int kTrStack = 48;       // transmittance: traversal stack depth
constexpr int kTrBlocksPerSM = 8;  // transmittance: resident blocks per SM (24 KB shared, <= 64 registers)
constexpr int kFFBlock = 128;      // free flight: threads per block of the scan
constexpr int kFFStack = 36;       // free flight: traversal stack depth (4-wide nodes)
constexpr int kFFBlocksPerSM = 5;  // free flight: resident scan blocks per SM (41 KB shared, <= 102 registers)
constexpr int kB = 32;             // free flight: bins of the scan

struct TraceScene {
  const float4* nodes;   // binary nodes
  const uint4* nodes4;   // 4-wide quantised nodes (ugp_internal.cuh)
  const float4* prims;
  const float4* wlo;
  int64_t n_prims;
  int64_t n_nodes;
  float k2;
};

TraceScene trace_scene(const ugp_bvh* b);

ugp_status check_rays(const char* fn, const ugp_bvh* bvh, int64_t n, const void* o3, const void* d3,
                      const void* t0, const void* t1);

ugp_status launch_transmittance(const TraceScene& sc, int64_t n, const float* o3, const float* d3,
                                const float* t0, const float* t1, const int32_t* excl, float* T,
                                uint8_t* st, cudaStream_t stream);

// The workspace holds the finish's queue for n rays (dense_queue_bytes(n, slots)) and, with
// `with_lists`, the slot lists after it; slots < 0 takes the default number of interval slots.
ugp_status launch_free_flight(const TraceScene& sc, int64_t n, const float* o3, const float* d3,
                              const float* t0, const float* t1, const float* u, const float* u2,
                              const int32_t* excl, int32_t* prim, float* tu, float* tsp, uint8_t* st,
                              void* workspace, bool with_lists, cudaStream_t stream, int64_t slots = -1);

}  // namespace ugp
