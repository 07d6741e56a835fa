// Rays whose t_u the scan has bracketed, for the finish passes (ugp_dense.cu). The table has one slot per
// scanned ray (its index in the scan's launch): the scan writes the ray's record there, or marks
// the slot empty (idx = -1), so no counter is shared between lanes; the finish pass walks the
// slots 32 at a time and takes the filled ones.
#pragma once

#include <cooperative_groups.h>

#include "ugp_trace.cuh"

namespace ugp {

// Structure of arrays in caller-provided scratch memory (a 256-byte header, then the columns).
struct DenseQueue {
  int* count;    // header ints: [0] unused, [1] ray counter of the persistent scan, [2] and [3]
                 // rays handed to the finish's second and third passes
  int* idx;      // output index of the ray (-1: empty slot)
  float *lo, *hi, *Flo, *u, *u2;
  float *ox, *oy, *oz, *dx, *dy, *dz, *t0, *t1;
  int* excl;
  int* nlist;    // primitive slots the scan recorded for the ray (> kListCap: list incomplete)
  int* scene;    // index of the ray's scene in `scenes` (batched rendering)
  int* wide;     // slots the finish's first pass handed to its second (count[2] of them)
  int* heavy;    // unused
  const int* list;  // per-ray slot lists, kListCap ints at list + idx * kListCap (NULL: none)
  const TraceScene* scenes;  // device table of scenes (NULL: every ray uses the launch's scene)
  float* big_iv;  // interval storage of the second pass: big_slots slots of kBigCap intervals
  int big_slots;
};

constexpr int kDenseCols = 19;
// Slots of the primitives the scan met before its window end, kept per ray so the dense pass
// can rebuild the window's intervals without another traversal.
constexpr int kListCap = 256;
inline size_t slot_list_bytes(int64_t n) { return align256(size_t(n) * kListCap * 4); }

// The finish's second pass keeps each ray's intervals (up to kBigCap, 9 words each) in a slot of
// global memory owned by one warp; a queue for `cap` rays has big_slots(cap) of them by default,
// one per 64 rays between 4 and 2432 (the warps a GB300 keeps resident in that pass), so that a
// launch of a few hundred thousand rays already fills the GPU.
constexpr int kBigCap = 2048;
constexpr int64_t big_slots(int64_t cap) { return cap / 64 < 4 ? 4 : (cap / 64 > 2432 ? 2432 : cap / 64); }
constexpr size_t big_slot_bytes() { return size_t(kBigCap) * 9 * 4; }

// Bytes of a queue for `cap` rays (256-byte aligned columns after a 256-byte header, then
// `slots` interval slots of the second pass); the slot lists, when used, take
// slot_list_bytes(cap) more.
constexpr size_t dense_queue_bytes(int64_t cap, int64_t slots) {
  return 256 + size_t(kDenseCols) * align256(size_t(cap) * 4) + size_t(slots) * big_slot_bytes();
}
constexpr size_t dense_queue_bytes(int64_t cap) { return dense_queue_bytes(cap, big_slots(cap)); }

inline DenseQueue dense_queue_at(void* base, int64_t cap, int64_t slots) {
  char* p = static_cast<char*>(base);
  const size_t col = align256(size_t(cap) * 4);
  auto F = [&](int k) { return reinterpret_cast<float*>(p + 256 + k * col); };
  DenseQueue q;
  q.count = reinterpret_cast<int*>(p);
  q.idx = reinterpret_cast<int*>(F(0));
  q.lo = F(1); q.hi = F(2); q.Flo = F(3); q.u = F(4); q.u2 = F(5);
  q.ox = F(6); q.oy = F(7); q.oz = F(8); q.dx = F(9); q.dy = F(10); q.dz = F(11);
  q.t0 = F(12); q.t1 = F(13);
  q.excl = reinterpret_cast<int*>(F(14));
  q.nlist = reinterpret_cast<int*>(F(15));
  q.scene = reinterpret_cast<int*>(F(16));
  q.wide = reinterpret_cast<int*>(F(17));
  q.heavy = reinterpret_cast<int*>(F(18));
  q.list = nullptr;
  q.scenes = nullptr;
  q.big_iv = reinterpret_cast<float*>(p + 256 + kDenseCols * col);
  q.big_slots = int(slots);
  return q;
}
inline DenseQueue dense_queue_at(void* base, int64_t cap) { return dense_queue_at(base, cap, big_slots(cap)); }

// Fills slot j with a bracketed ray whose results go to output index idx.
__device__ __forceinline__ void dense_push(const DenseQueue& q, int j, int idx, float lo, float hi, float Flo, float u,
                                           float u2, float3 o, float3 d, float t0, float t1, int excl, int nlist,
                                           int scene = 0) {
  q.idx[j] = idx;
  q.lo[j] = lo; q.hi[j] = hi; q.Flo[j] = Flo; q.u[j] = u; q.u2[j] = u2;
  q.ox[j] = o.x; q.oy[j] = o.y; q.oz[j] = o.z;
  q.dx[j] = d.x; q.dy[j] = d.y; q.dz[j] = d.z;
  q.t0[j] = t0; q.t1[j] = t1;
  q.excl[j] = excl;
  q.nlist[j] = nlist;
  if (q.scenes) q.scene[j] = scene;
}
// Marks slot j empty (the ray escaped or ended in the scan).
__device__ __forceinline__ void dense_none(const DenseQueue& q, int j) { q.idx[j] = -1; }

// Finishes every queued ray: prim_out[idx], t_spawn_out[idx] (the spawn distance, or t_u when
// spawn_mode == 1) and, when not NULL, t_u_out[idx] and status_out[idx].  `stats` as for the
// trace counters (nodes, primitives of the warp pass are added to [0], [1]), `rays_err` (may be
// NULL) counts rays that ended with a non-zero status.
// One-time setup of the finish kernel (shared-memory attribute, grid size); launch_dense calls it,
// and callers that capture launches into a graph call it before capturing.
ugp_status dense_prepare();
// Slots 0 .. n-1 are walked, n = *n_dev when n_dev is not NULL, else n_host; max_slots bounds n
// (grid size).
ugp_status launch_dense(const TraceScene& sc, const DenseQueue& q, int64_t n_host, const int* n_dev,
                        int64_t max_slots, int* prim_out, float* t_u_out, float* t_spawn_out, uint8_t* status_out,
                        int spawn_mode, unsigned long long* stats, unsigned long long* rays_err, cudaStream_t stream);

}  // namespace ugp
