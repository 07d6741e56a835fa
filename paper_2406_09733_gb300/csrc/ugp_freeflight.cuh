// Free-flight sampling device code shared by the standalone query and the renderer.
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
//  * scan (this header, one thread per ray, one traversal).  A nearest-first traversal adds
//    each interval's contribution to kB equal bins of [t0, scene exit].  The first bin whose
//    prefix passes u, the crossing bin j, can only move earlier as intervals arrive, so subtrees
//    starting after its end are pruned.  The slots of the primitives met before that end are
//    recorded in the ray's slot list.  Afterwards F(e_j) is exact from the bins, t_u lies in
//    [e_j, e_j+1], and the list holds every primitive whose interval meets that bin.
//  * finish (ugp_dense.cu, one warp per ray): 32 lanes rebuild the bin's intervals from the list,
//    solve F(t_u) = u by a safeguarded Newton iteration with warp-reduced F and F' = 1/2 sum G
//    (Eq. 9), and run the race as a warp argmin.
#include "ugp_dense.cuh"
#include "ugp_gauss.cuh"
#include "ugp_philox.cuh"
#include "ugp_trace.cuh"

namespace ugp {

struct FFSmem {
  float bin[kB][kFFBlock];
  int stk[kFFStack][kFFBlock];
};

struct Ctx {  // per-ray state shared by the traversal visitors
  FFSmem& sm;
  int tid;
  const TraceScene& sc;
  Ray ray;
  float t0, t1;
  int ex;
  unsigned n_nodes, n_prims;
  uint8_t st;
  int* list;  // this ray's slot list (kListCap ints) or NULL
  int nlist;
};

#define FB(arr, i) c.sm.arr[(i)][c.tid]

// Nearest-first traversal of the leaves whose boxes meet [lo, hi].  The visitor may lower
// `limit`; children whose clipped entry lies beyond it are skipped and reported through
// vis.pruned(entry).
template <class V>
__device__ void traverse(Ctx& c, float lo, float hi, float& limit, V& vis) {
  int sp = 0, node = 0;
  while (true) {
    if (unsigned(node) >= unsigned(c.sc.n_nodes)) {
      c.st = UGP_RAY_BAD_NODE;
      return;
    }
    const float4* nd = c.sc.nodes + 4 * node;
    const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
    const int4 n3 = __ldg(reinterpret_cast<const int4*>(nd) + 3);
    ++c.n_nodes;
    const int ch[2] = {n3.x, n3.y};
    if ((ch[0] < 0 && ~ch[0] >= c.sc.n_prims) ||
        (ch[1] < 0 && ch[1] != kEmptyChild && ~ch[1] >= c.sc.n_prims)) {
      c.st = UGP_RAY_BAD_NODE;
      return;
    }
    float en[2];
    bool hc[2];
    hc[0] = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, c.ray, lo, hi, en[0]);
    hc[1] = ch[1] != kEmptyChild && slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, c.ray, lo, hi, en[1]);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (!hc[k]) continue;
      if (en[k] > limit) {
        vis.pruned(en[k]);
        hc[k] = false;
        continue;
      }
      if (ch[k] >= 0) continue;
      hc[k] = false;
      ++c.n_prims;
      vis.leaf(~ch[k], limit);
    }
    if (hc[0] && hc[1]) {
      const bool first0 = en[0] <= en[1];
      if (sp == kFFStack) {
        c.st = UGP_RAY_STACK_OVERFLOW;
        return;
      }
      FB(stk, sp) = first0 ? ch[1] : ch[0];
      ++sp;
      node = first0 ? ch[0] : ch[1];
    } else if (hc[0]) {
      node = ch[0];
    } else if (hc[1]) {
      node = ch[1];
    } else {
      if (sp == 0) return;
      --sp;
      node = FB(stk, sp);
    }
  }
}

// ---------------------------------------------------------------- scan visitor
struct ScanVisitor {
  Ctx& c;
  float lo, hi, w, target;  // bins of width w over [lo, hi]; target = u - F(lo)
  int jc;                   // current crossing bin (kB: none yet)
  __device__ float edge(int j) const { return j >= kB ? hi : lo + w * float(j); }
  __device__ void pruned(float) {}
  __device__ void leaf(int slot, float& limit) {
    PrimHit h;
    if (!prim_test(c.sc.prims, c.sc.wlo, slot, c.ray, c.t0, c.t1, c.sc.k2, c.ex, h)) return;
    const float x = fmaxf(h.a, lo), y = fminf(h.b, hi);
    if (!(x < y)) return;
    int j = min(kB - 1, max(0, int((x - lo) / w)));
    while (j > 0 && x < edge(j)) --j;
    while (j < kB - 1 && x >= edge(j + 1)) ++j;
    for (int k = j; k < kB && edge(k) < y; ++k) {
      const float xa = fmaxf(x, edge(k)), ya = fminf(y, edge(k + 1));
      if (xa < ya) FB(bin, k) += seg_half_integral(xa, ya, h.a, h.b, h.a_end, h.b_end, h.tn, h.ts, h.s, h.e0, h.th);
    }
    if (j <= jc) {  // the crossing bin can only move to or before this interval's first bin
      float acc = 0.f;
      for (int k = 0; k < jc; ++k) {
        acc += FB(bin, k);
        if (acc > target) {
          jc = k;
          limit = edge(jc + 1);
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

// Exit distance of the ray from the scene's bounding box (both children of the root).
static __device__ float scene_exit(const Ctx& c, float lo, float hi) {
  const float4* nd = c.sc.nodes;
  const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
  const int4 n3 = __ldg(reinterpret_cast<const int4*>(nd) + 3);
  const float lx = fminf(n0.x, n3.y != kEmptyChild ? n1.z : n0.x);
  const float ly = fminf(n0.y, n3.y != kEmptyChild ? n1.w : n0.y);
  const float lz = fminf(n0.z, n3.y != kEmptyChild ? n2.x : n0.z);
  const float hx = fmaxf(n0.w, n3.y != kEmptyChild ? n2.y : n0.w);
  const float hy = fmaxf(n1.x, n3.y != kEmptyChild ? n2.z : n1.x);
  const float hz = fmaxf(n1.y, n3.y != kEmptyChild ? n2.w : n1.y);
  const Ray& r = c.ray;
  const float x0 = (lx - r.o.x) * r.inv.x, x1 = (hx - r.o.x) * r.inv.x;
  const float y0 = (ly - r.o.y) * r.inv.y, y1 = (hy - r.o.y) * r.inv.y;
  const float z0 = (lz - r.o.z) * r.inv.z, z1 = (hz - r.o.z) * r.inv.z;
  const float th = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fmaxf(z0, z1));
  return fminf(hi, fmaxf(lo, th * (1.f + 1e-6f) + 1e-6f));
}

// Samples the free-flight distribution for the ray in `c` (see the file comment).
struct FFResult {
  int prim;          // -1: escape
  float t_u, t_spawn;
  bool pending;      // t_u is bracketed in [lo, hi] with F(lo) = Flo; the warp pass finishes it
  float lo, hi, Flo;
  int nlist;         // slots recorded in c.list
};

static __device__ FFResult ff_sample(Ctx& c, float u, float u2) {
  (void)u2;
  FFResult r{-1, c.t1, c.t1, false, 0.f, 0.f, 0.f, 0};
  if (!(c.sc.n_prims > 0 && c.t0 < c.t1)) return r;
  const float lo = c.t0, hi = scene_exit(c, c.t0, c.t1);
  if (!(lo < hi)) return r;
  for (int j = 0; j < kB; ++j) FB(bin, j) = 0.f;
  ScanVisitor v{c, lo, hi, (hi - lo) / float(kB), u, kB};
  float limit = hi;
  traverse(c, lo, hi, limit, v);
  if (c.st != UGP_RAY_OK || v.jc == kB) return r;  // F(end) <= u: escape
  float Flo = 0.f;
  for (int k = 0; k < v.jc; ++k) Flo += FB(bin, k);
  r.pending = true;
  r.lo = v.edge(v.jc);
  r.hi = v.edge(v.jc + 1);
  r.Flo = Flo;
  r.nlist = c.nlist;
  return r;
}

#undef FB

}  // namespace ugp
