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
// A BVH gives no front-to-back order (the paper's reason for a kd-tree, Sec. 5.1), so the
// kernel finds t_u in one of two ways, both exact:
//
//  * rounds (fast path).  A traversal collects the intervals with the smallest (a, index)
//    keys after a cursor into a per-ray shared-memory buffer of kK entries, next to the
//    intervals still active from the previous round.  Everything not kept starts at or after
//    t_w (the smallest dropped start, or the entry of a pruned subtree), so F on [t_c, t_w] is
//    known from the buffer; if it crosses u there, a safeguarded Newton iteration with
//    F' = 1/2 sum G (Eq. 9) finds t_u, else the window advances.
//  * dense mode (when more than kK intervals are active at once, as in dense aggregates, or
//    after kFFMaxRounds rounds).  In the spirit of the paper's GPU binning (Sec. 5.2), one
//    traversal adds each interval's contribution to kB equal bins of [t_c, scene exit],
//    pruning subtrees that start after the bin where the running sum passes u; this brackets
//    t_u in one bin.  If the intervals meeting the window fit the buffer the thread finishes
//    alone; otherwise the ray goes to a queue that a warp-per-ray pass (ugp_dense.cu) finishes:
//    32 lanes collect every interval of the bracket, solve F(t_u) = u by Newton with
//    warp-reduced F and F', and run the race as a warp argmin.
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
};

#define FB(arr, i) c.sm.arr[(i)][c.tid]

static __device__ __forceinline__ bool key_less(float a0, int i0, float a1, int i1) {
  return a0 < a1 || (a0 == a1 && i0 < i1);
}

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

// ---------------------------------------------------------------- rounds: collection visitor
struct RoundVisitor {
  Ctx& c;
  float t_c, cur_a;
  int cur_id, nC, cap, nNew;
  float t_next;
  __device__ void pruned(float en) { t_next = fminf(t_next, en); }
  __device__ void leaf(int slot, float& limit) {
    PrimHit h;
    if (!prim_test(c.sc.prims, c.sc.wlo, slot, c.ray, c.t0, c.t1, c.sc.k2, c.ex, h)) return;
    if (h.b <= t_c) return;                           // ends before the window
    if (!key_less(cur_a, cur_id, h.a, h.id)) return;  // kept in an earlier round
    int pos;
    if (nNew < cap) {
      pos = nC + nNew;
      ++nNew;
    } else {
      const int last = nC + nNew - 1;
      if (!key_less(h.a, h.id, FB(a, last), unpack_id(FB(id, last)))) {
        t_next = fminf(t_next, h.a);
        return;
      }
      t_next = fminf(t_next, FB(a, last));  // the evicted interval starts here
      pos = last;
    }
    while (pos > nC && key_less(h.a, h.id, FB(a, pos - 1), unpack_id(FB(id, pos - 1)))) {
      move(c, pos, pos - 1);
      --pos;
    }
    put(c, pos, h);
    if (nNew == cap) limit = FB(a, nC + nNew - 1);
  }
};

// ---------------------------------------------------------------- binned refinement visitor
struct BinVisitor {
  Ctx& c;
  float lo, hi, w, target;  // bins of width w over [lo, hi]; target = u - F(lo)
  int count;
  __device__ float edge(int j) const { return j >= kB ? hi : lo + w * float(j); }
  __device__ void pruned(float) {}
  __device__ void leaf(int slot, float& limit) {
    PrimHit h;
    if (!prim_test(c.sc.prims, c.sc.wlo, slot, c.ray, c.t0, c.t1, c.sc.k2, c.ex, h)) return;
    const float x = fmaxf(h.a, lo), y = fminf(h.b, hi);
    if (!(x < y)) return;
    if (count < kK) put(c, count, h);
    ++count;
    int j = min(kB - 1, max(0, int((x - lo) / w)));
    while (j > 0 && x < edge(j)) --j;
    while (j < kB - 1 && x >= edge(j + 1)) ++j;
    for (; j < kB && edge(j) < y; ++j) {
      const float xa = fmaxf(x, edge(j)), ya = fminf(y, edge(j + 1));
      if (xa < ya)
        FB(bin, j) += seg_half_integral(xa, ya, h.a, h.b, h.a_end, h.b_end, h.tn, h.ts, h.s, h.e0, h.th);
    }
    // the partial sums only grow, so once they pass the target the crossing is known to lie
    // at or before that bin's upper edge
    float acc = 0.f;
    for (int k = 0; k < kB; ++k) {
      acc += FB(bin, k);
      if (acc > target) {
        limit = fminf(limit, edge(k + 1));
        break;
      }
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
  unsigned rounds;
  bool dense;        // the rounds gave up (more than kK intervals active at once)
  bool pending;      // t_u is bracketed in [lo, hi] with F(lo) = Flo; the warp pass finishes it
  float lo, hi, Flo;
};

static __device__ FFResult ff_sample(Ctx& c, float u, float u2) {
  unsigned n_rounds = 0;
  int out_prim = -1;
  float out_tu = c.t1, out_tsp = c.t1;

  float t_c = c.t0, F_c = 0.f;
  float cur_a = -INFINITY;
  int cur_id = -1, nC = 0;
  bool done = !(c.sc.n_prims > 0 && c.t0 < c.t1);
  bool dense = false, pending = false;
  float p_lo = 0.f, p_hi = 0.f, p_Flo = 0.f;
  // ---------------- rounds ----------------
  while (!done) {
    if (n_rounds >= kFFMaxRounds || nC == kK) {
      dense = true;
      break;
    }
    ++n_rounds;
    RoundVisitor v{c, t_c, cur_a, cur_id, nC, kK - nC, 0, c.t1};
    float limit = c.t1;
    traverse(c, t_c, c.t1, limit, v);
    if (c.st != UGP_RAY_OK) break;
    const int nE = nC + v.nNew;
    const float t_w = fmaxf(v.t_next, t_c);
    float dF = 0.f;
    for (int e = 0; e < nE; ++e) {
      const float lo = fmaxf(FB(a, e), t_c), hi = fminf(FB(b, e), t_w);
      if (lo < hi) dF += entry_integral(c, e, lo, hi);
    }
    if (F_c + dF > u) {
      // F is flat after the last interval ends, so the root lies before min(t_w, max b)
      float t_hi = t_c;
      for (int e = 0; e < nE; ++e) t_hi = fmaxf(t_hi, FB(b, e));
      const float t = solve_buffer(c, nE, t_c, fminf(t_w, t_hi), F_c, u);
      const int pick = choose_buffer(c, nE, t, u2);
      if (pick >= 0) {
        out_prim = unpack_id(FB(id, pick));
        out_tu = t;
        out_tsp = 0.5f * (FB(a, pick) + FB(b, pick));
      }
      done = true;
      break;
    }
    F_c += dF;
    t_c = t_w;
    if (t_w >= c.t1) {
      done = true;  // escape
      break;
    }
    if (v.nNew > 0) {
      cur_a = FB(a, nE - 1);
      cur_id = unpack_id(FB(id, nE - 1));
    }
    int m = 0;  // carry the intervals still active after t_w
    for (int e = 0; e < nE; ++e) {
      if (FB(b, e) > t_w) {
        if (m != e) move(c, m, e);
        ++m;
      }
    }
    nC = m;
  }
  // ---------------- dense mode: binned bracket; the warp pass (ugp_dense.cu) finishes it ----------------
  if (dense && c.st == UGP_RAY_OK) {
    const float lo0 = t_c, hi0 = scene_exit(c, t_c, c.t1);
    for (int j = 0; j < kB; ++j) FB(bin, j) = 0.f;
    BinVisitor v{c, lo0, hi0, (hi0 - lo0) / float(kB), u - F_c, 0};
    float limit = hi0;
    traverse(c, lo0, hi0, limit, v);
    float t_u = -1.f;
    if (c.st == UGP_RAY_OK && v.count <= kK) {
      // every interval meeting [lo0, limit] is in the buffer
      float f, fp;
      eval_F(c, v.count, lo0, F_c, u, limit, f, fp);
      if (f > 0.f || limit < hi0) {
        float t_hi = lo0;
        for (int e = 0; e < v.count; ++e) t_hi = fmaxf(t_hi, FB(b, e));
        t_u = f > 0.f ? solve_buffer(c, v.count, lo0, fminf(limit, t_hi), F_c, u) : limit;
        const int pick = choose_buffer(c, v.count, t_u, u2);
        if (pick >= 0) {
          out_prim = unpack_id(FB(id, pick));
          out_tu = t_u;
          out_tsp = 0.5f * (FB(a, pick) + FB(b, pick));
        }
      }
    } else if (c.st == UGP_RAY_OK) {
      float acc = 0.f;
      int jx = -1;
      for (int j = 0; j < kB; ++j) {
        const float nxt = acc + FB(bin, j);
        if (nxt > u - F_c) {
          jx = j;
          break;
        }
        acc = nxt;
      }
      if (jx >= 0) {   // otherwise F(end) <= u: escape
        pending = true;
        p_lo = v.edge(jx);
        p_hi = v.edge(jx + 1);
        p_Flo = F_c + acc;
      }
    }
  }
  return FFResult{out_prim, out_tu, out_tsp, n_rounds, dense, pending, p_lo, p_hi, p_Flo};
}

#undef FB

}  // namespace ugp
