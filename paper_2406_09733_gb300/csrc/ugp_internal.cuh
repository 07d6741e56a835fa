// Internal declarations shared by the CUDA translation units of the ugp library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ugp.h"

namespace ugp {

constexpr uint32_t kBvhMagic = 0x55475042u;  // "UGPB"

// Device layout of one primitive ("hot" record, 64 B, leaf order):
//   r0 = (W00 W01 W02 mu.x)
//   r1 = (W10 W11 W12 mu.y)
//   r2 = (W20 W21 W22 mu.z)
//   r3 = (g0, original index as int bits, 0, 0)
// W = S^-1 R^T is the whitening matrix of Eq. 2, g0 the normaliser of Eq. 1.
constexpr int kPrimF4 = 4;

// Device layout of one binary BVH node (64 B): the bounding boxes of both
// children and the child references.
//   n0 = (c0.lo.x c0.lo.y c0.lo.z c0.hi.x)
//   n1 = (c0.hi.y c0.hi.z c1.lo.x c1.lo.y)
//   n2 = (c1.lo.z c1.hi.x c1.hi.y c1.hi.z)
//   n3 = (child0, child1, 0, 0) as int bits; child >= 0 is an internal node,
//        child < 0 is the leaf holding primitive slot ~child.
constexpr int kNodeF4 = 4;
// Child reference of the unused second child of a one-primitive tree's root.
constexpr int kEmptyChild = INT32_MIN;

// Device layout of one 4-wide node (64 B) of the collapsed tree the hot traversals walk: the
// binary internal nodes at even depth, each with the (up to four) children and grandchildren
// below it, their boxes quantised to 8 bits per face against a per-node grid.
//   w0 = (o.x, o.y, o.z as float bits, exponents: byte a = e_a + 128 for axes a = 0, 1, 2)
//   w1 = (lo_x, lo_y, lo_z, hi_x)  byte c of each word: child c's quantised face
//   w2 = (hi_y, hi_z, 0, 0)
//   w3 = (child0, child1, child2, child3) as int: >= 0 the 4-wide node of that (binary)
//        index, < 0 and != kEmptyChild the leaf holding primitive slot ~child, kEmptyChild none.
// Child c's box along axis a is [o_a + lo_a(c) 2^e_a, o_a + hi_a(c) 2^e_a]; the faces are rounded
// outwards, so the quantised box contains the exact one. An empty slot's box is inverted
// (lo = 255, hi = 0 on every axis), so no ray enters it. A 4-wide node sits at the index of its
// binary node (the array has holes at odd depths, which are never read).
constexpr int kNode4U4 = 4;

}  // namespace ugp

struct ugp_bvh {
  uint32_t magic;
  int device;
  int64_t n_prims;
  int64_t n_nodes;
  float k;
  float k2;
  const float4* nodes;
  const uint4* nodes4;       // the 4-wide quantised tree (same indices as nodes, even depths only)
  const float4* prims;
  const float4* wlo;         // low float parts of W, 3 float4 per leaf slot
  const float* bounds_dev;   // in the workspace: ordered-int centroid bounds, root box, invalid count
  cudaStream_t stream;       // build stream, used only by synchronous info queries
  size_t persistent_bytes;
};

namespace ugp {

// Thread-local error message helpers (defined in ugp_api.cu).
ugp_status fail(ugp_status s, const char* fmt, ...);
ugp_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

// Trace statistics pointer (device), or nullptr.
unsigned long long* trace_counters();

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Launch accounting and optional event timing (defined in ugp_api.cu).  Wrap each launch:
//   prof_begin(stage, stream); kernel<<<...>>>(...); prof_end(stage, stream, n_kernels);
enum ProfStage { kStBuild = 0, kStCamera = 1, kStExtend = 2, kStShade = 3, kStShadow = 4, kStAccum = 5, kStQuery = 6,
                 kStDense = 7, kStGuide = 8, kStBatch = 9 };
void prof_begin(int stage, cudaStream_t s);
void prof_end(int stage, cudaStream_t s, int n_kernels = 1);

// Stable radix sort of (key, value) pairs by the low `bits` bits of the keys (ugp_sort.cu): 8
// bits per pass, three kernels per pass, the pairs alternating between buffers 0 and 1 (the
// result is in buffer radix_sort_passes(bits) & 1). `ws` holds radix_sort_workspace(n) bytes,
// 256-byte aligned.
size_t radix_sort_workspace(int64_t n);
int radix_sort_passes(int bits);
ugp_status radix_sort_pairs(uint32_t* k0, uint32_t* k1, int32_t* v0, int32_t* v1, int64_t n, int bits, void* ws,
                            cudaStream_t st);
// While suspended, prof_begin / prof_end neither record events nor count launches (used while
// launches are captured into a graph, whose bodies cannot hold event records).
void prof_suspend(bool on);
// Adds launches that ran inside a graph to the counts.
void add_launches(int stage, int64_t n);

bool valid_bvh(const ugp_bvh* b);

}  // namespace ugp

#define UGP_CUDA_CHECK(call)                                  \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ::ugp::cuda_fail(_e, #call); \
  } while (0)
