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
// found in two exact steps, in the spirit of the paper's GPU binning (Sec. 5.2):
//
//  * scan (this header, one thread per ray, one traversal).  A nearest-first traversal adds
//    each interval's contribution to kB equal bins of [t0, scene exit].  The first bin whose
//    prefix passes u, the crossing bin j, can only move earlier as intervals arrive, so subtrees
//    starting after its end are pruned.  The thread also keeps the intervals that start before
//    that end in a kK-entry buffer, evicting the one that starts last when full and remembering
//    the smallest evicted start.  At the end F(e_j) is exact from the bins, and the buffer holds
//    every interval meeting [e_j, e_j+1] unless an evicted one starts before e_j+1.  If it does
//    hold them all, a safeguarded Newton iteration with F' = 1/2 sum G (Eq. 9) solves
//    F(t_u) = u inside the bin and the race picks the primitive.
//  * dense pass (ugp_dense.cu, one warp per ray) for the rays whose crossing bin holds more
//    intervals than the buffer, as inside dense aggregates: 32 lanes collect every interval of
//    the bin, solve with warp-reduced F and F', and run the race as a warp argmin.
#include "ugp_dense.cuh"
#include "ugp_gauss.cuh"
#include "ugp_philox.cuh"
#include "ugp_trace.cuh"

namespace ugp {

struct FFSmem {
  float a[kK][kFFBlock];
  float b[kK][kFFBlock];
  float tn[kK][kFFBlock];
  float ts[kK][kFFBlock];
  float s[kK][kFFBlock];
  float e0[kK][kFFBlock];
  float th[kK][kFFBlock];
  int id[kK][kFFBlock];   // index with the end-point flags (pack_id)
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

static __device__ __forceinline__ void put(Ctx& c, int pos, const PrimHit& h) {
  FB(a, pos) = h.a;
  FB(b, pos) = h.b;
  FB(tn, pos) = h.tn;
  FB(ts, pos) = h.ts;
  FB(s, pos) = h.s;
  FB(e0, pos) = h.e0;
  FB(th, pos) = h.th;
  FB(id, pos) = pack_id(h);
}

static __device__ __forceinline__ void move(Ctx& c, int to, int from) {
  FB(a, to) = FB(a, from);
  FB(b, to) = FB(b, from);
  FB(tn, to) = FB(tn, from);
  FB(ts, to) = FB(ts, from);
  FB(s, to) = FB(s, from);
  FB(e0, to) = FB(e0, from);
  FB(th, to) = FB(th, from);
  FB(id, to) = FB(id, from);
}

// 1/2 I of buffer entry e over [x, y].
static __device__ __forceinline__ float entry_integral(const Ctx& c, int e, float x, float y) {
  const int p = FB(id, e);
  return seg_half_integral(x, y, FB(a, e), FB(b, e), packed_a_end(p), packed_b_end(p), FB(tn, e), FB(ts, e),
                           FB(s, e), FB(e0, e), FB(th, e));
}

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
  int n;                    // buffer entries
  float lost_a;             // smallest start of an interval evicted from the full buffer
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
      for (int k = 0; k < kB; ++k) {
        acc += FB(bin, k);
        if (acc > target) {
          if (k < jc) {
            jc = k;
            limit = edge(jc + 1);
            int m = 0;  // intervals starting after the new end can no longer matter
            for (int e = 0; e < n; ++e) {
              if (FB(a, e) < limit) {
                if (m != e) move(c, m, e);
                ++m;
              }
            }
            n = m;
          }
          break;
        }
      }
    }
    if (!(x < edge(jc + 1))) return;
    if (c.list) {
      if (c.nlist < kListCap) c.list[c.nlist] = slot;
      ++c.nlist;
    }
    if (n < kK) {
      put(c, n++, h);
      return;
    }
    int far = 0;  // evict whichever of the buffer and the new interval starts last
    for (int e = 1; e < kK; ++e)
      if (FB(a, e) > FB(a, far)) far = e;
    if (FB(a, far) > h.a) {
      lost_a = fminf(lost_a, FB(a, far));
      put(c, far, h);
    } else {
      lost_a = fminf(lost_a, h.a);
    }
  }
};

// F(t) - u and F'(t) from the buffer entries [0, nE) on a window starting at lo with F(lo) = Flo.
static __device__ __forceinline__ void eval_F(Ctx& c, int nE, float lo, float Flo, float u, float t, float& f,
                                       float& fp) {
  f = Flo - u;
  fp = 0.f;
  for (int e = 0; e < nE; ++e) {
    const float x0 = fmaxf(FB(a, e), lo), x1 = fminf(FB(b, e), t);
    if (x0 < x1) f += entry_integral(c, e, x0, x1);
    if (FB(a, e) <= t && t <= FB(b, e)) fp += 0.5f * gauss_at(t, FB(tn, e), FB(ts, e), FB(s, e), FB(e0, e));
  }
}

// Root of F = u on [lo, hi] (F(lo) <= u < F(hi)) by Newton's method safeguarded with bisection:
// a Newton step is taken only if it stays in the bracket and shrinks it at least as fast as
// bisection would have two steps earlier.
static __device__ float solve_buffer(Ctx& c, int nE, float lo, float hi, float Flo, float u) {
  const float w_lo = lo;
  float t = 0.5f * (lo + hi);
  {
    float fh, fph;
    eval_F(c, nE, w_lo, Flo, u, hi, fh, fph);  // F(hi) - u > 0: start from the secant
    const float frac = (u - Flo) / (fh + u - Flo);
    const float ts = lo + frac * (hi - lo);
    if (ts > lo && ts < hi) t = ts;
  }
  float dx_old = hi - lo, dx = dx_old;
  for (int it = 0; it < kFFNewtonIters; ++it) {
    float f, fp;
    eval_F(c, nE, w_lo, Flo, u, t, f, fp);
    if (f == 0.f) return t;
    if (f < 0.f) lo = t; else hi = t;
    if (!(nextafterf(lo, INFINITY) < hi)) return t;  // bracket one float wide
    const float tn = fp > 0.f ? t - f / fp : lo;
    float tnew;
    if (fp > 0.f && tn > lo && tn < hi && fabsf(2.f * f) <= fabsf(dx_old * fp)) {
      dx_old = dx;
      dx = f / fp;
      tnew = tn;
    } else {
      dx_old = dx;
      dx = 0.5f * (hi - lo);
      tnew = lo + dx;
    }
    if (tnew == t) return t;
    t = tnew;
  }
  c.st = UGP_RAY_SOLVE_LIMIT;
  return t;
}

// Choice among buffer entries [0, nE) containing t by the exponential race (smallest E_k / G_k).
static __device__ int choose_buffer(Ctx& c, int nE, float t, float u2) {
  int pick = -1, pick_id = INT32_MAX;
  float best = INFINITY;
  for (int e = 0; e < nE; ++e) {
    if (!(FB(a, e) <= t && t <= FB(b, e))) continue;
    const int idv = unpack_id(FB(id, e));
    const float key = race_exponential(u2, idv) / gauss_at(t, FB(tn, e), FB(ts, e), FB(s, e), FB(e0, e));
    if (pick < 0 || key < best || (key == best && idv < pick_id)) {
      best = key;
      pick = e;
      pick_id = idv;
    }
  }
  return pick;
}

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
  FFResult r{-1, c.t1, c.t1, false, 0.f, 0.f, 0.f, 0};
  if (!(c.sc.n_prims > 0 && c.t0 < c.t1)) return r;
  const float lo = c.t0, hi = scene_exit(c, c.t0, c.t1);
  if (!(lo < hi)) return r;
  for (int j = 0; j < kB; ++j) FB(bin, j) = 0.f;
  ScanVisitor v{c, lo, hi, (hi - lo) / float(kB), u, kB, 0, INFINITY};
  float limit = hi;
  traverse(c, lo, hi, limit, v);
  if (c.st != UGP_RAY_OK || v.jc == kB) return r;  // F(end) <= u: escape
  float Flo = 0.f;
  for (int k = 0; k < v.jc; ++k) Flo += FB(bin, k);
  const float wlo = v.edge(v.jc), whi = v.edge(v.jc + 1);
  if (v.lost_a < whi) {  // the buffer misses intervals of the crossing bin
    r.pending = true;
    r.lo = wlo;
    r.hi = whi;
    r.Flo = Flo;
    r.nlist = c.nlist;
    return r;
  }
  // F is flat after the last interval ends, so the root lies before min(whi, max b)
  float t_hi = wlo;
  for (int e = 0; e < v.n; ++e) t_hi = fmaxf(t_hi, FB(b, e));
  t_hi = fminf(t_hi, whi);
  float f, fp;
  eval_F(c, v.n, wlo, Flo, u, t_hi, f, fp);
  const float t = f > 0.f ? solve_buffer(c, v.n, wlo, t_hi, Flo, u) : t_hi;
  const int pick = choose_buffer(c, v.n, t, u2);
  if (pick >= 0) {
    r.prim = unpack_id(FB(id, pick));
    r.t_u = t;
    r.t_spawn = 0.5f * (FB(a, pick) + FB(b, pick));
  }
  return r;
}

#undef FB

}  // namespace ugp
