// Free-flight sampling device code shared by the standalone query, the renderer and the batch
// server.
#pragma once

// Exact free-flight distribution sampling over the BVH (Sec. 5.2, Eq. 8-10).
//
// Definition (order-free).  With the clipped intervals [a_k, b_k] of the primitives along the
// ray and F(t) = 1/2 sum_k I_k(a_k, min(t, b_k)): the ray escapes if F(t1) <= u; otherwise
// t_u solves F(t_u) = u and the primitive is drawn among those whose interval contains t_u
// with probability G_k(x_{t_u}) / sum_j G_j(x_{t_u}).  The draw is an exponential race: each
// candidate k gets E_k = -ln U_k with U_k from Philox keyed by u2 and counter k, and the
// smallest E_k / G_k wins, so the result does not depend on the order candidates are seen in.
// Since u < 1, t_u lies before the saturating distance, so primitive k is chosen with
// probability 1/2 I_k(a_k, min(b_k, t_sat)).
//
// A BVH gives no front-to-back order (the paper's reason for a kd-tree, Sec. 5.1), so t_u is
// found in two exact passes, in the spirit of the paper's GPU binning (Sec. 5.2):
//
//  * scan (this header, one lane per ray, one traversal).  A nearest-first traversal adds
//    each interval's contribution to kB bins of the ray's span inside the scene box, [lo, hi];
//    bin j ends at lo + (hi - lo) ((j + 1) / kB)^2, so bins are finest near the ray's start,
//    where the crossing lies for rays that start in or near dense matter (their pruning limit
//    and finish bracket then shrink with the free path).  The first bin whose
//    prefix passes u, the crossing bin j, can only move earlier as intervals arrive, so subtrees
//    starting after its end are pruned, and bins after it are no longer updated.  The slots of
//    the primitives met before its end are recorded in the ray's slot list.  Afterwards F(e_j)
//    is exact from the bins, t_u lies in [e_j, e_j+1], and the list holds every primitive whose
//    interval meets that bin.
//  * finish (ugp_dense.cu, 16 lanes per ray, more for rays with many intervals): the lanes
//    rebuild the bin's intervals from the list, solve F(t_u) = u by a safeguarded Newton
//    iteration with F and F' = 1/2 sum G (Eq. 9) summed across them, and run the race as an
//    argmin across them.
//
// The scan runs on persistent lanes: a lane whose ray is done takes a new one, and the idle
// lanes of a warp fetch together (one atomic) once kRefill of them are idle, so a warp does not
// wait for its slowest ray before starting new ones (per-ray work varies several-fold; on camera
// rays of a 1M-primitive room the mean over a warp is 0.58 of its maximum). Each loop step is
// either a node step (every lane with nodes left visits one) or a leaf step: primitives met in
// node steps are held back until the warp holds 32 of them (or a lane's queue is nearly full or
// its traversal is over), and a leaf step then spreads them over the lanes, one per lane
// whichever ray it belongs to, so the expensive primitive test and binning run on all lanes
// (with one primitive per lane of its own ray, the leaf steps of a 5.5M-primitive room's path
// rays kept 10 of 32 lanes busy). A lane bins into the owning ray's bins with shared-memory atomics; the owner
// moves its crossing bin after the step. Holding a primitive back can only delay a lowering of
// the pruning limit, never skip a node that matters.
#include "ugp_dense.cuh"
#include "ugp_gauss.cuh"
#include "ugp_philox.cuh"
#include "ugp_trace.cuh"

namespace ugp {

constexpr int kLeafQ = 12;  // primitives a lane may hold back before they are tested (< 16)

// Bins hold 1/2 I in fixed point, units of 2^-28: integer sums do not depend on the order the
// contributions arrive in, so a ray's result does not depend on which rays share its warp or
// which lanes test its primitives. A contribution is capped at kBinCap, just above 1, and a bin
// that already holds kBinCap or more takes no more: the bins before the crossing bin sum to at
// most u <= 1, so such a bin lies at or after the crossing, where only "exceeds u" matters. A
// step adds to one ray's bins from at most kLeafQ lanes, so no bin or running sum passes
// (kLeafQ + 1) kBinCap < 2^32. Contributions below 2^-29 are dropped.
constexpr float kBinScale = 268435456.f;            // 2^28
constexpr float kBinUnit = 3.725290298461914e-09f;  // 2^-28
constexpr unsigned kBinCap = (1u << 28) + 1u;       // just above 1 in bin units
static_assert((kLeafQ + 1ull) * kBinCap < (1ull << 32), "bins must not wrap");
static_assert(kLeafQ < 16, "queue lengths are summed from four bit planes");

struct FFSmem {
  unsigned bin[kB][kFFBlock];  // fixed-point bins
  int stk[kFFStack][kFFBlock];
  int lq[kLeafQ][kFFBlock];    // held-back primitive slots
  unsigned below[kFFBlock];    // sum of the bins before the crossing bin (all bins while none)
  int nlist[kFFBlock];         // slots recorded in the ray's list
  int owner[kFFBlock];         // leaf steps: lane of each warp's k-th ray with queued primitives
};

// A ray as handed to and returned from the scan (Src::begin fills the ray fields, the driver
// the rest at the end).
struct ScanState {
  Ray ray;
  float t0, t1;
  int ex;
  float lo, hi;      // bins over [lo, hi] (bin_edge)
  int jc;            // crossing bin (kB: none)
  unsigned n_nodes, n_prims;
  uint8_t st;
  int* list;         // this ray's slot list (kListCap ints) or NULL
  int nlist;
};

#define FB(arr, i) sm.arr[(i)][tid]

// The scene's bounding box: the union of the root's children (binary node layout).
static __device__ __forceinline__ void scene_box(const TraceScene& sc, float3& lo, float3& hi) {
  const float4* nd = sc.nodes;
  const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
  const int4 n3 = __ldg(reinterpret_cast<const int4*>(nd) + 3);
  lo = make_float3(fminf(n0.x, n3.y != kEmptyChild ? n1.z : n0.x), fminf(n0.y, n3.y != kEmptyChild ? n1.w : n0.y),
                   fminf(n0.z, n3.y != kEmptyChild ? n2.x : n0.z));
  hi = make_float3(fmaxf(n0.w, n3.y != kEmptyChild ? n2.y : n0.w), fmaxf(n1.x, n3.y != kEmptyChild ? n2.z : n1.x),
                   fmaxf(n1.y, n3.y != kEmptyChild ? n2.w : n1.y));
}

// Span [entry, exit] of the ray inside the scene's bounding box, clipped to [lo, hi] and widened
// by a few ulps so that every clipped interval lies inside it.
static __device__ float2 scene_span(const TraceScene& sc, const Ray& r, float lo, float hi) {
  float3 bl, bh;
  scene_box(sc, bl, bh);
  const float x0 = (bl.x - r.o.x) * r.inv.x, x1 = (bh.x - r.o.x) * r.inv.x;
  const float y0 = (bl.y - r.o.y) * r.inv.y, y1 = (bh.y - r.o.y) * r.inv.y;
  const float z0 = (bl.z - r.o.z) * r.inv.z, z1 = (bh.z - r.o.z) * r.inv.z;
  const float tl = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fminf(z0, z1));
  const float th = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fmaxf(z0, z1));
  const float e = fminf(hi, fmaxf(lo, th * (1.f + 1e-6f) + 1e-6f));
  const float b = fminf(e, fmaxf(lo, tl - 1e-6f * fabsf(tl) - 1e-6f));
  return make_float2(b, e);
}

// Edge j of the scan's bins over [lo, hi] (L = hi - lo): lo + L (j / kB)^2, hi for j >= kB.
// (j / kB)^2 is exact in float and the products round monotonically, so edges never decrease.
__device__ __forceinline__ float bin_edge(float lo, float hi, float L, int j) {
  return j >= kB ? hi : fmaf(L, float(j * j) * (1.f / float(kB * kB)), lo);
}

// Result of a finished scan.
struct FFResult {
  int prim;          // -1: escape
  float t_u, t_spawn;
  bool pending;      // t_u is bracketed in [lo, hi] with F(lo) = Flo; the warp pass finishes it
  float lo, hi, Flo;
  int nlist;         // slots recorded in the ray's list
};

static __device__ FFResult scan_result(FFSmem& sm, int tid, const ScanState& s, bool traversed) {
  FFResult r{-1, s.t1, s.t1, false, 0.f, 0.f, 0.f, 0};
  if (!traversed || s.st != UGP_RAY_OK || s.jc == kB) return r;  // F(end) <= u: escape
  unsigned long long acc = 0;
  for (int k = 0; k < s.jc; ++k) acc += FB(bin, k);
  const float Flo = float(acc) * kBinUnit;
  r.pending = true;
  r.lo = bin_edge(s.lo, s.hi, s.hi - s.lo, s.jc);
  r.hi = bin_edge(s.lo, s.hi, s.hi - s.lo, s.jc + 1);
  r.Flo = Flo;
  r.nlist = s.nlist;
  return r;
}

#undef FB

constexpr int kRefill = 2;  // idle lanes of a warp that trigger a joint fetch of new rays

// Traversal context of one lane: the scene, the ray and its counters, as used by the
// persistent driver below.
struct ScanCtx {
  FFSmem& sm;
  int tid;
  TraceScene sc;
  Ray ray;
  float t0, t1;
  int ex;
  unsigned n_nodes, n_prims;
  uint8_t st;
  int* list;
};

// What a lane needs to test and bin a held-back primitive of another lane's ray (the owner).
struct OwnerRay {
  const float4* prims;
  const float4* wlo;
  float k2;
  Ray ray;
  float t0, t1;
  int ex;
  float lo, hi, L;
  int jc;     // the owner's crossing bin at the start of the step (it only moves earlier)
  int* list;
  int tid;    // the owner's thread index in the block (its column of the shared arrays)
  __device__ float edge(int j) const { return bin_edge(lo, hi, L, j); }
};

// Tests primitive `slot` against the owner's ray and adds its interval's contribution to the
// owner's bins up to the owner's crossing bin, with shared-memory atomics (other lanes may bin
// primitives of the same ray in the same step); contributions to bins before the crossing bin
// also go to the owner's running sum of them, and a primitive met before the crossing bin's end
// goes into the owner's slot list. The owner moves its crossing bin afterwards.
static __device__ void pooled_leaf(FFSmem& sm, const OwnerRay& w, int slot) {
  PrimHit h;
  if (!prim_test(w.prims, w.wlo, slot, w.ray, w.t0, w.t1, w.k2, w.ex, h)) return;
  const float x = fmaxf(h.a, w.lo), y = fminf(h.b, w.hi);
  if (!(x < y)) return;
  int j = min(kB - 1, max(0, int(float(kB) * sqrtf((x - w.lo) / w.L))));
  while (j > 0 && x < w.edge(j)) --j;
  while (j < kB - 1 && x >= w.edge(j + 1)) ++j;
  if (j > w.jc) return;  // starts after the crossing bin: cannot matter any more
  const int kend = w.jc < kB ? w.jc + 1 : kB;
  // The share of bin k is 1/2 I between consecutive cut points (App. A): a difference of erf
  // values, taken as erfc(|tau|) at each cut point (same-sign pairs without cancellation), so
  // each cut point costs one erfc however many bins the interval spans.
  const float amp = h.e0 * (0.25f * kSqrtPi) / h.s;
  float tp = (h.a_end && x == h.a) ? -h.th : tau_at(x, h.tn, h.ts, h.s);
  float ep = erfcf(fabsf(tp));
  unsigned long long dbelow = 0;
  float e_lo = w.edge(j);
  for (int k = j; k < kend; ++k) {
    const float e_hi = w.edge(k + 1);
    const float xa = fmaxf(x, e_lo), ya = fminf(y, e_hi);
    e_lo = e_hi;
    if (!(xa < y)) break;
    if (xa < ya) {
      const float tq = (h.b_end && ya == h.b) ? h.th : tau_at(ya, h.tn, h.ts, h.s);
      const float eq = erfcf(fabsf(tq));
      const float diff = tp >= 0.f ? ep - eq : (tq <= 0.f ? eq - ep : 2.f - ep - eq);
      const unsigned add = min(__float2uint_rn(fminf(fmaxf(amp * diff, 0.f) * kBinScale, 2.f * kBinScale)), kBinCap);
      unsigned* bp = &sm.bin[k][w.tid];
      if (add != 0u && *reinterpret_cast<volatile unsigned*>(bp) < kBinCap) {
        atomicAdd(bp, add);
        if (k < w.jc) dbelow += add;
      }
      tp = tq;
      ep = eq;
    }
  }
  // a share above kBinCap makes the running sum exceed u anyway: capping it keeps the sum within
  // 32 bits
  if (dbelow != 0ull) atomicAdd(&sm.below[w.tid], unsigned(dbelow < kBinCap ? dbelow : kBinCap));
  if (x < w.edge(w.jc + 1) && w.list) {
    const int pos = atomicAdd(&sm.nlist[w.tid], 1);
    if (pos < kListCap) w.list[pos] = slot;
  }
}

// Persistent-lane driver of the scan. Src supplies the rays:
//   __device__ int count() const                    rays in this launch
//   __device__ bool begin(int i, ScanState& s, float& u)   loads ray i (ray, t0, t1, ex, list);
//                                                  false: the ray is skipped (no result)
//   __device__ TraceScene scene() const             the current ray's scene
//   __device__ void finish(const ScanState& s, const FFResult& r)   writes the current ray's result
// Src is per thread and keeps what it needs of the current ray. `next` is a device counter,
// zero before the launch. The node step is written out in the loop with the traversal state in
// plain locals; kept in this form, the compiler holds the state in registers across the refill
// branch (the same steps written as helper functions over ScanState ran 1.4x slower).
template <class Src>
__device__ void scan_persistent(FFSmem& sm, Src& src, int* next) {
  const int lane = int(threadIdx.x) & 31;
  constexpr unsigned kFull = 0xffffffffu;
  const int n = src.count();
  ScanCtx c{sm, int(threadIdx.x), src.scene(), make_ray(make_float3(0.f, 0.f, 0.f), make_float3(0.f, 0.f, 1.f)), 0.f,
            0.f, -1, 0u, 0u, UGP_RAY_OK, nullptr};
  ScanState s;
  bool busy = false, exhausted = false, tdone = false;
  int node = 0, sp = 0, jc = kB, nq = 0;
  float lo = 0.f, hi = 0.f, L = 0.f, target = 0.f, limit = 0.f;
  for (;;) {
    const unsigned idle = __ballot_sync(kFull, !busy && !exhausted);
    unsigned working = __ballot_sync(kFull, busy);
    if (idle && (__popc(idle) >= kRefill || working == 0)) {
      int base = 0;
      const int leader = __ffs(idle) - 1;
      if (lane == leader) base = atomicAdd(next, __popc(idle));
      base = __shfl_sync(kFull, base, leader);
      if (!busy && !exhausted) {
        const int i = base + __popc(idle & ((1u << lane) - 1u));
        if (i >= n) {
          exhausted = true;
        } else {
          float u = 0.f;
          if (src.begin(i, s, u)) {
            c.sc = src.scene();
            c.ray = s.ray;
            c.t0 = s.t0;
            c.t1 = s.t1;
            c.ex = s.ex;
            c.n_nodes = c.n_prims = 0u;
            c.st = UGP_RAY_OK;
            c.list = s.list;
            target = u;
            lo = hi = c.t0;
            if (c.sc.n_prims > 0 && c.t0 < c.t1) {
              const float2 sp2 = scene_span(c.sc, c.ray, c.t0, c.t1);
              lo = sp2.x;
              hi = sp2.y;
            }
            if (!(lo < hi)) {  // nothing to traverse: the ray escapes
              s.n_nodes = s.n_prims = 0u;
              s.st = UGP_RAY_OK;
              s.nlist = 0;
              src.finish(s, scan_result(sm, c.tid, s, false));
            } else {
              L = hi - lo;
              for (int j = 0; j < kB; ++j) sm.bin[j][c.tid] = 0u;
              sm.below[c.tid] = 0u;
              sm.nlist[c.tid] = 0;
              jc = kB;
              limit = hi;
              node = 0;
              sp = 0;
              nq = 0;
              tdone = false;
              busy = true;
            }
          }
        }
      }
      working = __ballot_sync(kFull, busy);
    }
    if (working == 0) {
      if (__all_sync(kFull, exhausted)) break;
      continue;
    }
    const int mine = busy ? nq : 0;
    const int total = int(__reduce_add_sync(kFull, unsigned(mine)));
    // a node step may add four held-back primitives: it runs only while every lane has room
    const bool urgent = __any_sync(kFull, busy && (nq > kLeafQ - 4 || (tdone && nq > 0)));
    if (total > 0 && (total >= 32 || urgent)) {
      // ---- leaf step: the warp's held-back primitives, up to 32, one per lane whichever ray
      // they belong to; lane i takes item i of the lanes' queues laid end to end
      // each lane's exclusive prefix of the queue lengths (below 16) from four bit planes
      const unsigned below_me = (1u << lane) - 1u;
      const unsigned q0 = __ballot_sync(kFull, (mine & 1) != 0), q1 = __ballot_sync(kFull, (mine & 2) != 0),
                     q2 = __ballot_sync(kFull, (mine & 4) != 0), q3 = __ballot_sync(kFull, (mine & 8) != 0);
      const int off = __popc(q0 & below_me) + 2 * __popc(q1 & below_me) + 4 * __popc(q2 & below_me) +
                      8 * __popc(q3 & below_me);
      const unsigned has = q0 | q1 | q2 | q3;
      const unsigned starts = __reduce_or_sync(kFull, (mine > 0 && off < 32) ? (1u << off) : 0u);
      const bool work = lane < total;
      int* owner_of = sm.owner + (c.tid & ~31);
      if (mine > 0) owner_of[__popc(has & below_me)] = lane;
      __syncwarp();
      const int o = work ? owner_of[__popc(starts & (0xffffffffu >> (31 - lane))) - 1] : lane;
      const int off_o = __shfl_sync(kFull, off, o);
      const int nq_o = __shfl_sync(kFull, mine, o);
      OwnerRay w;
      w.prims = reinterpret_cast<const float4*>(
          __shfl_sync(kFull, reinterpret_cast<unsigned long long>(c.sc.prims), o));
      w.wlo = reinterpret_cast<const float4*>(__shfl_sync(kFull, reinterpret_cast<unsigned long long>(c.sc.wlo), o));
      w.k2 = __shfl_sync(kFull, c.sc.k2, o);
      w.ray.o = make_float3(__shfl_sync(kFull, c.ray.o.x, o), __shfl_sync(kFull, c.ray.o.y, o),
                            __shfl_sync(kFull, c.ray.o.z, o));
      w.ray.d = make_float3(__shfl_sync(kFull, c.ray.d.x, o), __shfl_sync(kFull, c.ray.d.y, o),
                            __shfl_sync(kFull, c.ray.d.z, o));
      w.ray.inv = make_float3(0.f, 0.f, 0.f);  // not used by the primitive test
      w.ray.inv_dd = __shfl_sync(kFull, c.ray.inv_dd, o);
      w.t0 = __shfl_sync(kFull, c.t0, o);
      w.t1 = __shfl_sync(kFull, c.t1, o);
      w.ex = __shfl_sync(kFull, c.ex, o);
      w.lo = __shfl_sync(kFull, lo, o);
      w.hi = __shfl_sync(kFull, hi, o);
      w.L = __shfl_sync(kFull, L, o);
      w.jc = __shfl_sync(kFull, jc, o);
      w.list = reinterpret_cast<int*>(__shfl_sync(kFull, reinterpret_cast<unsigned long long>(c.list), o));
      w.tid = (int(threadIdx.x) & ~31) | o;
      if (work) pooled_leaf(sm, w, sm.lq[nq_o - 1 - (lane - off_o)][w.tid]);
      __syncwarp();
      // each ray drops the items taken from the top of its queue and, when its running sum of
      // the bins before the crossing bin passes u, moves the crossing bin (bins are
      // non-negative, so while that sum is at most u no prefix passes u earlier)
      const int taken = min(mine, max(0, 32 - off));
      if (taken > 0) {
        nq = mine - taken;
        const unsigned tgt = unsigned(target * kBinScale);  // u <= 1, a multiple of 2^-24: exact
        if (sm.below[c.tid] > tgt) {
          unsigned long long acc = 0;
          for (int k = 0; k < jc; ++k) {
            const unsigned long long before = acc;
            acc += sm.bin[k][c.tid];
            if (acc > tgt) {
              jc = k;
              limit = bin_edge(lo, hi, L, jc + 1);
              sm.below[c.tid] = unsigned(before);
              break;
            }
          }
        }
      }
    } else if (busy && !tdone) {
      // ---- node step: one 4-wide node of the nearest-first traversal
      if (unsigned(node) >= unsigned(c.sc.n_nodes)) {
        c.st = UGP_RAY_BAD_NODE;
        node = 0;
      }
      float en[4];
      int ch[4];
      unsigned hm = node4_test(c.sc.nodes4, node, c.ray, lo, hi, en, ch);
      ++c.n_nodes;
      float tk[4];
      int rk[4];
      int nk = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        tk[k] = INFINITY;
        rk[k] = -1;
        if (!((hm >> k) & 1u)) continue;
        // a primitive's slot is checked here (its record is loaded by slot); a child node's
        // index is checked when it is visited
        if (ch[k] < 0 && unsigned(~ch[k]) >= unsigned(c.sc.n_prims)) c.st = UGP_RAY_BAD_NODE;
        if (en[k] > limit || c.st != UGP_RAY_OK) continue;
        if (ch[k] < 0) {
          ++c.n_prims;
          sm.lq[nq][c.tid] = ~ch[k];  // nq <= kLeafQ - 4 here: a node adds at most four
          ++nq;
        } else {
          tk[k] = en[k];
          rk[k] = ch[k];
          ++nk;
        }
      }
      sort4(tk, rk);
      if (c.st != UGP_RAY_OK) {
        tdone = true;
        nq = 0;
      } else if (nk > 0) {
        if (sp + nk - 1 > kFFStack) {
          c.st = UGP_RAY_STACK_OVERFLOW;
          tdone = true;
          nq = 0;
        } else {
          // the farther children go on the stack, farthest first, so the nearer pop first
#pragma unroll
          for (int k = 3; k >= 1; --k)
            if (rk[k] >= 0) {
              sm.stk[sp][c.tid] = rk[k];
              ++sp;
            }
          node = rk[0];
        }
      } else if (sp == 0) {
        tdone = true;
      } else {
        --sp;
        node = sm.stk[sp][c.tid];
      }
    }
    if (busy && tdone && nq == 0) {
      s.lo = lo;
      s.hi = hi;
      s.jc = jc;
      s.st = c.st;
      s.n_nodes = c.n_nodes;
      s.n_prims = c.n_prims;
      s.nlist = sm.nlist[c.tid];
      src.finish(s, scan_result(sm, c.tid, s, true));
      busy = false;
    }
  }
}

// Grid of a persistent scan launch: every SM filled with resident blocks.
int scan_grid(const void* kernel);

}  // namespace ugp
