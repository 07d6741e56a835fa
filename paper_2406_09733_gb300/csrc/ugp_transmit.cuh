// Transmittance (Sec. 5.3, Eq. 7) of one ray: device code shared by the query and the renderer.
#pragma once

#include "ugp_gauss.cuh"
#include "ugp_trace.cuh"

namespace ugp {

struct TrStats {
  unsigned n_nodes, n_prims;
  uint8_t st;
};

constexpr int kTrLeafQ = 10;  // primitives a lane may hold back (top of its stack column)

// Returns tau = 1/2 sum_k I_k(clip_k) over [t0, t1], stopping once it reaches 1 (then T = 0).
// The sum is kept in 64-bit fixed point (units of 2^-40), so it is the same in any traversal
// order and whichever lanes test a ray's primitives (terms below 2^-41 are dropped: under 1e-10
// in tau for a few hundred of them); nearest-child-first only makes the early exit come sooner.
// `stk` points at this thread's column of a shared-memory stack with `stride` between levels,
// `acc` at this thread's entry of a shared array of sums and `owner` at its entry of a shared
// int array (its neighbours in the warp are the other lanes' entries). The lanes that call together (the active mask) run in steps: a node
// step visits one node per lane and holds back the primitives it meets (up to kTrLeafQ, kept at
// the top of the stack column); a leaf step, taken once the lanes hold a primitive for each of
// them (or a queue is nearly full or a traversal is over), spreads the held-back primitives over
// the lanes, one per lane whichever ray it belongs to, and each lane adds its primitive's term to
// the owner's sum with a shared-memory atomic.
static_assert(kTrLeafQ < 16, "queue lengths are summed from four bit planes");
static __device__ float tr_optical_depth(const TraceScene& sc, const Ray& ray, float t0, float t1, int ex,
                                         int* stk, int stride, unsigned long long* acc, int* owner, TrStats& ts) {
  const unsigned mask = __activemask();
  const int lane = int(threadIdx.x) & 31;
  const unsigned below_me = (1u << lane) - 1u;
  const int nact = __popc(mask), rank = __popc(mask & below_me);
  constexpr float kScale = 1099511627776.f;  // 2^40
  constexpr unsigned long long kOne = 1ull << 40;
  *acc = 0ull;
  int sp = 0, node = 0, nq = 0;
  bool tdone = !(sc.n_prims > 0 && t0 < t1), done = tdone;
  int* lq = stk + (kTrStack - kTrLeafQ) * stride;
  __syncwarp(mask);
  for (;;) {
    // queue lengths (below 16) as four bit planes: their sum and each lane's exclusive prefix
    const int mine = done ? 0 : nq;
    const unsigned p0 = __ballot_sync(mask, (mine & 1) != 0), p1 = __ballot_sync(mask, (mine & 2) != 0),
                   p2 = __ballot_sync(mask, (mine & 4) != 0), p3 = __ballot_sync(mask, (mine & 8) != 0);
    const int total = __popc(p0) + 2 * __popc(p1) + 4 * __popc(p2) + 8 * __popc(p3);
    // a node step may add four held-back primitives: it runs only while every lane has room
    const bool urgent = __any_sync(mask, !done && (nq > kTrLeafQ - 4 || (tdone && nq > 0)));
    if (total > 0 && (total >= nact || urgent)) {
      // the lane of rank r takes item r of the queues laid end to end (lane order)
      const int off = __popc(p0 & below_me) + 2 * __popc(p1 & below_me) + 4 * __popc(p2 & below_me) +
                      8 * __popc(p3 & below_me);
      const unsigned starts = __reduce_or_sync(mask, (mine > 0 && off < 32) ? (1u << off) : 0u);
      const bool work = rank < total;
      // the k-th calling lane with queued primitives, by a table the owners fill
      int* owner_of = owner - lane;
      if (mine > 0) owner_of[__popc((p0 | p1 | p2 | p3) & below_me)] = lane;
      __syncwarp(mask);
      const int o = work ? owner_of[__popc(starts & (0xffffffffu >> (31 - rank))) - 1] : lane;
      const int off_o = __shfl_sync(mask, off, o);
      const int nq_o = __shfl_sync(mask, mine, o);
      Ray ro;
      ro.o = make_float3(__shfl_sync(mask, ray.o.x, o), __shfl_sync(mask, ray.o.y, o), __shfl_sync(mask, ray.o.z, o));
      ro.d = make_float3(__shfl_sync(mask, ray.d.x, o), __shfl_sync(mask, ray.d.y, o), __shfl_sync(mask, ray.d.z, o));
      ro.inv = make_float3(0.f, 0.f, 0.f);  // not used by the primitive test
      ro.inv_dd = __shfl_sync(mask, ray.inv_dd, o);
      const float t0o = __shfl_sync(mask, t0, o), t1o = __shfl_sync(mask, t1, o);
      const int exo = __shfl_sync(mask, ex, o);
      const float4* prims = reinterpret_cast<const float4*>(
          __shfl_sync(mask, reinterpret_cast<unsigned long long>(sc.prims), o));
      const float4* wlo = reinterpret_cast<const float4*>(
          __shfl_sync(mask, reinterpret_cast<unsigned long long>(sc.wlo), o));
      const float k2 = __shfl_sync(mask, sc.k2, o);
      if (work) {
        PrimHit h;
        const int slot = lq[(nq_o - 1 - (rank - off_o)) * stride + (o - lane)];
        if (prim_test(prims, wlo, slot, ro, t0o, t1o, k2, exo, h))
          atomicAdd(acc + (o - lane),
                    (unsigned long long)__float2ll_rn(fminf(fmaxf(hit_half_integral(h), 0.f), 2.f) * kScale));
      }
      __syncwarp(mask);
      if (mine > 0) {
        nq = mine - min(mine, max(0, nact - off));
        if (*acc >= kOne) {  // saturated: T = 0 whatever follows
          done = true;
          nq = 0;
        }
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
        int nk = 0;
        bool bad = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          tk[k] = INFINITY;
          rk[k] = -1;
          if (!((hm >> k) & 1u)) continue;
          if (ch[k] < 0) {
            // a primitive's slot is checked here (its record is loaded by slot); a child node's
            // index is checked when it is visited
            if (unsigned(~ch[k]) >= unsigned(sc.n_prims)) {
              bad = true;
              continue;
            }
            ++ts.n_prims;
            lq[nq * stride] = ~ch[k];  // nq <= kTrLeafQ - 4 here: a node adds at most four
            ++nq;
          } else {
            tk[k] = en[k];
            rk[k] = ch[k];
            ++nk;
          }
        }
        sort4(tk, rk);
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
  const unsigned long long a = *acc;
  return a >= kOne ? 1.f : float(a) * (1.f / kScale);
}

}  // namespace ugp
