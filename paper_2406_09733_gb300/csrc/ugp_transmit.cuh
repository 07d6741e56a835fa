// Transmittance (Sec. 5.3, Eq. 7) of one ray: device code shared by the query and the renderer.
#pragma once

#include "ugp_gauss.cuh"
#include "ugp_trace.cuh"

namespace ugp {

struct TrStats {
  unsigned n_nodes, n_prims;
  uint8_t st;
};

constexpr int kTrLeafQ = 6;       // primitives a lane may hold back (top of its stack column)
constexpr int kTrLeafBatch = 16;  // lanes with held-back primitives that start a joint leaf step

// Returns tau = 1/2 sum_k I_k(clip_k) over [t0, t1], stopping once it reaches 1 (then T = 0).
// The sum is kept in 64-bit fixed point (units of 2^-40), so it is the same in any traversal
// order, whatever rays share the warp (terms below 2^-41 are dropped: under 1e-10 in tau for a
// few hundred of them); nearest-child-first only makes the early exit come sooner.
// `stk` points at this thread's column of a shared-memory stack with `stride` between levels.
// The lanes that call together (the active mask) run in steps: a node step visits one node per
// lane and holds back the primitives it meets (up to kTrLeafQ, kept at the top of the stack
// column); a leaf step, taken once kTrLeafBatch lanes hold some (or a queue is nearly full or a
// traversal is over), tests one held-back primitive per lane, so the expensive test and erf run
// with most lanes together.
static __device__ float tr_optical_depth(const TraceScene& sc, const Ray& ray, float t0, float t1, int ex,
                                         int* stk, int stride, TrStats& ts) {
  const unsigned mask = __activemask();
  constexpr float kScale = 1099511627776.f;  // 2^40
  constexpr long long kOne = 1ll << 40;
  long long acc = 0;
  int sp = 0, node = 0, nq = 0;
  bool tdone = !(sc.n_prims > 0 && t0 < t1), done = tdone;
  int* lq = stk + (kTrStack - kTrLeafQ) * stride;
  for (;;) {
    const unsigned pend = __ballot_sync(mask, !done && nq > 0);
    // a node step may add four held-back primitives: it runs only while every lane has room
    const bool urgent = __any_sync(mask, !done && (nq > kTrLeafQ - 4 || (tdone && nq > 0)));
    if (pend && (__popc(pend) >= kTrLeafBatch || urgent)) {
      if (!done && nq > 0) {
        --nq;
        PrimHit h;
        if (prim_test(sc.prims, sc.wlo, lq[nq * stride], ray, t0, t1, sc.k2, ex, h))
          acc += __float2ll_rn(fminf(fmaxf(hit_half_integral(h), 0.f), 2.f) * kScale);
        if (acc >= kOne) done = true;  // saturated: T = 0 whatever follows
      }
    } else if (!done && !tdone) {
      if (unsigned(node) >= unsigned(sc.n_nodes)) {
        ts.st = UGP_RAY_BAD_NODE;
        tdone = true;
        nq = 0;
      } else {
        float en[4];
        int ch[4];
        const unsigned hm = node4_test(sc.nodes4, node, ray, t0, t1, en, ch);
        ++ts.n_nodes;
        float tk[4];
        int rk[4];
        bool bad = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          tk[k] = INFINITY;
          rk[k] = -1;
          if (!((hm >> k) & 1u)) continue;
          if ((ch[k] < 0 && ~ch[k] >= sc.n_prims) || (ch[k] >= 0 && ch[k] >= sc.n_nodes)) {
            bad = true;
            continue;
          }
          if (ch[k] < 0) {
            ++ts.n_prims;
            lq[nq * stride] = ~ch[k];  // nq <= kTrLeafQ - 4 here: a node adds at most four
            ++nq;
          } else {
            tk[k] = en[k];
            rk[k] = ch[k];
          }
        }
        sort4(tk, rk);
        const int nk = (rk[0] >= 0) + (rk[1] >= 0) + (rk[2] >= 0) + (rk[3] >= 0);
        if (bad) {
          ts.st = UGP_RAY_BAD_NODE;
          tdone = true;
          nq = 0;
        } else if (nk > 0) {
          if (sp + nk - 1 > kTrStack - kTrLeafQ) {
            ts.st = UGP_RAY_STACK_OVERFLOW;
            tdone = true;
            nq = 0;
          } else {
#pragma unroll
            for (int k = 3; k >= 1; --k)
              if (rk[k] >= 0) {
                stk[sp * stride] = rk[k];
                ++sp;
              }
            node = rk[0];
          }
        } else if (sp == 0) {
          tdone = true;
        } else {
          --sp;
          node = stk[sp * stride];
        }
      }
    }
    if (tdone && nq == 0) done = true;
    if (!__any_sync(mask, !done)) break;
  }
  return acc >= kOne ? 1.f : float(acc) * (1.f / kScale);
}

}  // namespace ugp
