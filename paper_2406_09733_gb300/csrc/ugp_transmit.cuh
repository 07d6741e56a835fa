// Transmittance (Sec. 5.3, Eq. 7) of one ray: device code shared by the query and the renderer.
#pragma once

#include "ugp_gauss.cuh"
#include "ugp_trace.cuh"

namespace ugp {

struct TrStats {
  unsigned n_nodes, n_prims;
  uint8_t st;
};

constexpr int kTrLeafQ = 4;       // primitives a lane may hold back (top of its stack column)
constexpr int kTrLeafBatch = 16;  // lanes with held-back primitives that start a joint leaf step

// Returns tau = 1/2 sum_k I_k(clip_k) over [t0, t1], stopping once it reaches 1 (then T = 0).
// Any traversal order gives the same sum; nearest-child-first makes the early exit come sooner.
// `stk` points at this thread's column of a shared-memory stack with `stride` between levels.
// The lanes that call together (the active mask) run in steps: a node step visits one node per
// lane and holds back the primitives it meets (up to kTrLeafQ, kept at the top of the stack
// column); a leaf step, taken once kTrLeafBatch lanes hold some (or a queue is nearly full or a
// traversal is over), tests one held-back primitive per lane, so the expensive test and erf run
// with most lanes together.
static __device__ float tr_optical_depth(const TraceScene& sc, const Ray& ray, float t0, float t1, int ex,
                                         int* stk, int stride, TrStats& ts) {
  const unsigned mask = __activemask();
  float acc = 0.f;
  int sp = 0, node = 0, nq = 0;
  bool tdone = !(sc.n_prims > 0 && t0 < t1), done = tdone;
  int* lq = stk + (kTrStack - kTrLeafQ) * stride;
  for (;;) {
    const unsigned pend = __ballot_sync(mask, !done && nq > 0);
    const bool urgent = __any_sync(mask, !done && (nq >= kTrLeafQ - 1 || (tdone && nq > 0)));
    if (pend && (__popc(pend) >= kTrLeafBatch || urgent)) {
      if (!done && nq > 0) {
        --nq;
        PrimHit h;
        if (prim_test(sc.prims, sc.wlo, lq[nq * stride], ray, t0, t1, sc.k2, ex, h)) acc += hit_half_integral(h);
        if (acc >= 1.f) done = true;  // saturated: T = 0 whatever follows
      }
    } else if (!done && !tdone) {
      if (unsigned(node) >= unsigned(sc.n_nodes)) {
        ts.st = UGP_RAY_BAD_NODE;
        tdone = true;
        nq = 0;
      } else {
        const float4* nd = sc.nodes + 4 * node;
        const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
        const int4 n3 = __ldg(reinterpret_cast<const int4*>(nd) + 3);
        ++ts.n_nodes;
        if ((n3.x < 0 && ~n3.x >= sc.n_prims) || (n3.y < 0 && n3.y != kEmptyChild && ~n3.y >= sc.n_prims)) {
          ts.st = UGP_RAY_BAD_NODE;
          tdone = true;
          nq = 0;
        } else {
          float e0, e1;
          bool h0 = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, ray, t0, t1, e0);
          bool h1 = n3.y != kEmptyChild && slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, ray, t0, t1, e1);
          if (h0 && n3.x < 0) {
            ++ts.n_prims;
            lq[nq * stride] = ~n3.x;
            ++nq;
            h0 = false;
          }
          if (h1 && n3.y < 0) {
            ++ts.n_prims;
            lq[nq * stride] = ~n3.y;
            ++nq;
            h1 = false;
          }
          if (h0 && h1) {
            const bool first0 = e0 <= e1;
            if (sp == kTrStack - kTrLeafQ) {
              ts.st = UGP_RAY_STACK_OVERFLOW;
              tdone = true;
              nq = 0;
            } else {
              stk[sp * stride] = first0 ? n3.y : n3.x;
              ++sp;
              node = first0 ? n3.x : n3.y;
            }
          } else if (h0) {
            node = n3.x;
          } else if (h1) {
            node = n3.y;
          } else if (sp == 0) {
            tdone = true;
          } else {
            --sp;
            node = stk[sp * stride];
          }
        }
      }
    }
    if (tdone && nq == 0) done = true;
    if (!__any_sync(mask, !done)) break;
  }
  return acc;
}

}  // namespace ugp
