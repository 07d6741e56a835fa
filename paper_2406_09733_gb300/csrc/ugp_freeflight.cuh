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
// either a node step (every lane with nodes left visits one) or a leaf step (every lane with
// held-back primitives tests one and bins it): primitives met in node steps are held back
// until kLeafBatch lanes have some (or a lane's queue is nearly full or its traversal is over),
// so the expensive primitive test and binning run with most lanes together instead of inside a
// node step that most lanes skip. Holding a primitive back can only delay a lowering of the
// pruning limit, never skip a node that matters.
#include "ugp_dense.cuh"
#include "ugp_gauss.cuh"
#include "ugp_philox.cuh"
#include "ugp_trace.cuh"

namespace ugp {

constexpr int kLeafQ = 6;      // primitives a lane may hold back before testing them
constexpr int kLeafBatch = 16;  // lanes with held-back primitives that start a joint leaf phase

// Bins hold 1/2 I in fixed point, units of 2^-30, with saturating adds: integer sums do not depend
// on the order the contributions arrive in, so a ray's result does not depend on which rays share
// its warp. Bins before the crossing bin sum to less than u <= 1; a bin that saturates (>= 2) lies
// at or after it, where only "exceeds u" matters. Contributions below 2^-31 are dropped.
constexpr float kBinScale = 1073741824.f;         // 2^30
constexpr float kBinUnit = 9.313225746154785e-10f;  // 2^-30

__device__ __forceinline__ int bin_add(int b, float v) {
  const float f = fminf(fmaxf(v, 0.f) * kBinScale, 2147483520.f);
  const long long t = (long long)b + (long long)__float2int_rn(f);
  return t > 2147483647ll ? 2147483647 : int(t);
}

struct FFSmem {
  int bin[kB][kFFBlock];     // fixed-point bins
  int stk[kFFStack][kFFBlock];
  int lq[kLeafQ][kFFBlock];  // held-back primitive slots
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
  long long acc = 0;
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

// Traversal context of one lane (the scene, the ray and its counters) and the bin visitor of a
// primitive met by the traversal, as used by the persistent driver below.
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
  int nlist;
};

struct ScanBins {
  ScanCtx& c;
  float lo, hi, L, target;
  int jc;           // crossing bin (kB: none yet)
  long long below;  // sum of the bins before the crossing bin (of all bins while there is none)
  __device__ float edge(int j) const { return bin_edge(lo, hi, L, j); }
  // The interval's contribution goes to the bins up to the crossing bin; the crossing bin (and
  // the pruning limit) may move earlier; primitives met before its end go into the slot list.
  __device__ void leaf(int slot, float& limit) {
    PrimHit h;
    if (!prim_test(c.sc.prims, c.sc.wlo, slot, c.ray, c.t0, c.t1, c.sc.k2, c.ex, h)) return;
    const float x = fmaxf(h.a, lo), y = fminf(h.b, hi);
    if (!(x < y)) return;
    int j = min(kB - 1, max(0, int(float(kB) * sqrtf((x - lo) / L))));
    while (j > 0 && x < edge(j)) --j;
    while (j < kB - 1 && x >= edge(j + 1)) ++j;
    if (j > jc) return;  // starts after the crossing bin: cannot matter any more
    const int kend = jc < kB ? jc + 1 : kB;
    // The share of bin k is 1/2 I between consecutive cut points (App. A): a difference of erf
    // values, taken as erfc(|tau|) at each cut point (same-sign pairs without cancellation), so
    // each cut point costs one erfc however many bins the interval spans.
    const float amp = h.e0 * (0.25f * kSqrtPi) / h.s;
    float tp = (h.a_end && x == h.a) ? -h.th : tau_at(x, h.tn, h.ts, h.s);
    float ep = erfcf(fabsf(tp));
    for (int k = j; k < kend; ++k) {
      const float xa = fmaxf(x, edge(k)), ya = fminf(y, edge(k + 1));
      if (!(xa < y)) break;
      if (xa < ya) {
        const float tq = (h.b_end && ya == h.b) ? h.th : tau_at(ya, h.tn, h.ts, h.s);
        const float eq = erfcf(fabsf(tq));
        const float diff = tp >= 0.f ? ep - eq : (tq <= 0.f ? eq - ep : 2.f - ep - eq);
        const int old = c.sm.bin[k][c.tid];
        const int nb = bin_add(old, amp * diff);
        c.sm.bin[k][c.tid] = nb;
        if (k < jc) below += nb - old;
        tp = tq;
        ep = eq;
      }
    }
    // Bins are non-negative, so while the bins before the crossing bin sum to at most u no
    // prefix passes u earlier, and the crossing bin stands; otherwise find the new one.
    const long long tgt = (long long)(target * kBinScale);  // u is a multiple of 2^-24: exact
    if (below > tgt) {
      long long acc = 0;
      for (int k = 0; k < jc; ++k) {
        const long long before = acc;
        acc += c.sm.bin[k][c.tid];
        if (acc > tgt) {
          jc = k;
          limit = edge(jc + 1);
          below = before;
          break;
        }
      }
    }
    if (x < edge(jc + 1) && c.list) {
      if (c.nlist < kListCap) c.list[c.nlist] = slot;
      ++c.nlist;
    }
  }
};

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
            0.f, -1, 0u, 0u, UGP_RAY_OK, nullptr, 0};
  ScanState s;
  bool busy = false, exhausted = false, tdone = false;
  int node = 0, sp = 0, jc = kB, nq = 0;
  long long below = 0;
  float lo = 0.f, hi = 0.f, L = 0.f, target = 0.f, limit = 0.f;
  for (;;) {
    const unsigned idle = __ballot_sync(kFull, !busy && !exhausted);
    const unsigned working = __ballot_sync(kFull, busy);
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
            c.nlist = 0;
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
              for (int j = 0; j < kB; ++j) sm.bin[j][c.tid] = 0;
              jc = kB;
              below = 0;
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
    }
    if (__ballot_sync(kFull, busy) == 0) {
      if (__all_sync(kFull, exhausted)) break;
      continue;
    }
    const unsigned pend = __ballot_sync(kFull, busy && nq > 0);
    // a node step may add four held-back primitives: it runs only while every lane has room
    const bool urgent = __any_sync(kFull, busy && (nq > kLeafQ - 4 || (tdone && nq > 0)));
    if (pend && (__popc(pend) >= kLeafBatch || urgent)) {
      // ---- leaf step: one held-back primitive per lane
      if (busy && nq > 0) {
        --nq;
        ScanBins v{c, lo, hi, L, target, jc, below};
        v.leaf(sm.lq[nq][c.tid], limit);
        jc = v.jc;
        below = v.below;
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
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        tk[k] = INFINITY;
        rk[k] = -1;
        if (!((hm >> k) & 1u)) continue;
        if ((ch[k] < 0 && ~ch[k] >= c.sc.n_prims) || (ch[k] >= 0 && ch[k] >= c.sc.n_nodes)) c.st = UGP_RAY_BAD_NODE;
        if (en[k] > limit || c.st != UGP_RAY_OK) continue;
        if (ch[k] < 0) {
          ++c.n_prims;
          sm.lq[nq][c.tid] = ~ch[k];  // nq <= kLeafQ - 4 here: a node adds at most four
          ++nq;
        } else {
          tk[k] = en[k];
          rk[k] = ch[k];
        }
      }
      sort4(tk, rk);
      const int nk = (rk[0] >= 0) + (rk[1] >= 0) + (rk[2] >= 0) + (rk[3] >= 0);
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
      s.nlist = c.nlist;
      src.finish(s, scan_result(sm, c.tid, s, true));
      busy = false;
    }
  }
}

// Grid of a persistent scan launch: every SM filled with resident blocks.
int scan_grid(const void* kernel);

}  // namespace ugp
