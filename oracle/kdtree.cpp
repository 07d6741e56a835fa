// FP64 oracle: the paper's own free-flight sampler (Sec. 5.2 and its listing), a diagnostic for
// the paper-faithful variant; the order-free sampler of geometry.cpp is the parity target.
//
// TEST INFRASTRUCTURE ONLY.
//  * An SAH kd-tree over the primitives' k-ellipsoid boxes (primitives straddling a plane go to
//    both sides), built by trying the box faces of every primitive as planes.
//  * Front-to-back traversal: each leaf covers a range [ta, tb] of the ray, and the leaves'
//    ranges partition [t0, t1]; a primitive contributes I_k over its clipped interval within the
//    range.
//  * In a leaf with one primitive, or whose contributions keep the running CDF below 1, the
//    primitives accumulate 1/2 I_k one by one (in the leaf's order) and the first one whose
//    running sum passes u is returned. Otherwise the leaf range is cut into segments of constant
//    active set; a segment with one primitive or whose CDF stays below 1 accumulates the same
//    way, and the segment where the CDF reaches 1 (the ambiguous one) solves F(t_u) = u and picks
//    among its active primitives proportionally to I_k(s0, t_u), with u_seg = F(s0) + u2 (u - F(s0)).
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "oracle_internal.h"

namespace orc {

namespace {

struct Box {
  double lo[3], hi[3];
};
double area(const Box& b) {
  const double e[3] = {b.hi[0] - b.lo[0], b.hi[1] - b.lo[1], b.hi[2] - b.lo[2]};
  return 2.0 * (e[0] * e[1] + e[1] * e[2] + e[2] * e[0]);
}

Box prim_box(const Prim& p, double k) {
  Box b;
  const double m[3] = {p.mu.x, p.mu.y, p.mu.z};
  for (int r = 0; r < 3; ++r) {
    double e2 = 0;
    for (int c = 0; c < 3; ++c) e2 += (p.R[3 * r + c] * p.s[c]) * (p.R[3 * r + c] * p.s[c]);
    b.lo[r] = m[r] - k * std::sqrt(e2);
    b.hi[r] = m[r] + k * std::sqrt(e2);
  }
  return b;
}

constexpr double kTraverse = 1.0, kIntersect = 1.5;
constexpr int kLeafMax = 4, kDepthMax = 24;

int build(KdTree& T, const std::vector<Box>& boxes, std::vector<int32_t> ids, const Box& nb, int depth) {
  const int me = int(T.nodes.size());
  T.nodes.push_back(KdNode{});
  const int n = int(ids.size());
  double best = kIntersect * n;  // cost of a leaf (relative to the node's area)
  int best_axis = -1;
  double best_pos = 0;
  if (n > kLeafMax && depth < kDepthMax) {
    const double a0 = area(nb);
    for (int ax = 0; ax < 3; ++ax) {
      std::vector<double> cand;
      for (int32_t i : ids) {
        cand.push_back(boxes[size_t(i)].lo[ax]);
        cand.push_back(boxes[size_t(i)].hi[ax]);
      }
      std::sort(cand.begin(), cand.end());
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
      for (double pos : cand) {
        if (!(pos > nb.lo[ax] && pos < nb.hi[ax])) continue;
        int nl = 0, nr = 0;
        for (int32_t i : ids) {
          if (boxes[size_t(i)].lo[ax] < pos) ++nl;
          if (boxes[size_t(i)].hi[ax] > pos) ++nr;
        }
        Box L = nb, R = nb;
        L.hi[ax] = pos;
        R.lo[ax] = pos;
        const double c = kTraverse + kIntersect * (area(L) * nl + area(R) * nr) / a0;
        if (c < best) {
          best = c;
          best_axis = ax;
          best_pos = pos;
        }
      }
    }
  }
  if (best_axis < 0) {
    T.nodes[size_t(me)].axis = -1;
    T.nodes[size_t(me)].first = int32_t(T.leaf_ids.size());
    T.nodes[size_t(me)].count = n;
    T.leaf_ids.insert(T.leaf_ids.end(), ids.begin(), ids.end());
    return me;
  }
  std::vector<int32_t> l, r;
  for (int32_t i : ids) {
    if (boxes[size_t(i)].lo[best_axis] < best_pos) l.push_back(i);
    if (boxes[size_t(i)].hi[best_axis] > best_pos) r.push_back(i);
  }
  ids.clear();
  Box L = nb, R = nb;
  L.hi[best_axis] = best_pos;
  R.lo[best_axis] = best_pos;
  const int cl = build(T, boxes, std::move(l), L, depth + 1);
  const int cr = build(T, boxes, std::move(r), R, depth + 1);
  KdNode& node = T.nodes[size_t(me)];
  node.axis = best_axis;
  node.pos = best_pos;
  node.child[0] = cl;
  node.child[1] = cr;
  return me;
}

}  // namespace

KdTree kd_build(const std::vector<Prim>& prims, double k) {
  KdTree T;
  std::vector<Box> boxes;
  Box root{{1e300, 1e300, 1e300}, {-1e300, -1e300, -1e300}};
  for (const Prim& p : prims) {
    boxes.push_back(prim_box(p, k));
    for (int a = 0; a < 3; ++a) {
      root.lo[a] = std::min(root.lo[a], boxes.back().lo[a]);
      root.hi[a] = std::max(root.hi[a], boxes.back().hi[a]);
    }
  }
  for (int a = 0; a < 3; ++a) {
    T.lo[a] = root.lo[a];
    T.hi[a] = root.hi[a];
  }
  std::vector<int32_t> ids(prims.size());
  for (size_t i = 0; i < ids.size(); ++i) ids[i] = int32_t(i);
  if (!prims.empty()) build(T, boxes, std::move(ids), root, 0);
  return T;
}

namespace {

// Running state of one sample along the ray.
struct KdSample {
  const std::vector<Prim>& prims;
  V3 o, d;
  double t0, t1, k, u, u2;
  double cdf = 0.0;
  int32_t result = -1;
  bool done = false;
  KdStats st;
};

// The part of primitive i's clipped interval within [ta, tb], if any.
bool part(const KdSample& S, int32_t i, double ta, double tb, Hit* h) {
  if (!ray_prim(S.prims[size_t(i)], i, S.o, S.d, S.t0, S.t1, S.k, h)) return false;
  h->a = std::max(h->a, ta);
  h->b = std::min(h->b, tb);
  return h->a < h->b;
}

void leaf(KdSample& S, const KdTree& T, const KdNode& nd, double ta, double tb) {
  std::vector<Hit> hs;
  for (int j = 0; j < nd.count; ++j) {
    Hit h;
    ++S.st.prims_tested;
    if (part(S, T.leaf_ids[size_t(nd.first + j)], ta, tb, &h)) hs.push_back(h);
  }
  if (hs.empty()) return;
  double sum = 0.0;
  for (const Hit& h : hs) sum += 0.5 * ray_integral(h, h.a, h.b);
  if (hs.size() == 1 || S.cdf + sum < 1.0) {
    for (const Hit& h : hs) {
      S.cdf += 0.5 * ray_integral(h, h.a, h.b);
      if (S.u < S.cdf) {
        S.result = h.id;
        S.done = true;
        return;
      }
    }
    return;
  }
  // segments of constant active set inside the leaf's range
  std::vector<double> ev;
  for (const Hit& h : hs) {
    ev.push_back(h.a);
    ev.push_back(h.b);
  }
  std::sort(ev.begin(), ev.end());
  ev.erase(std::unique(ev.begin(), ev.end()), ev.end());
  for (size_t s = 0; s + 1 < ev.size(); ++s) {
    const double s0 = ev[s], s1 = ev[s + 1];
    std::vector<const Hit*> act;
    for (const Hit& h : hs)
      if (h.a <= s0 && h.b >= s1) act.push_back(&h);
    if (act.empty()) continue;
    double dF = 0.0;
    for (const Hit* h : act) dF += 0.5 * ray_integral(*h, s0, s1);
    if (act.size() == 1 || S.cdf + dF < 1.0) {
      for (const Hit* h : act) {
        S.cdf += 0.5 * ray_integral(*h, s0, s1);
        if (S.u < S.cdf) {
          S.result = h->id;
          S.done = true;
          return;
        }
      }
      continue;
    }
    // ambiguous segment: u < 1 <= cdf + dF, so t_u lies inside; bracketed Newton
    double lo = s0, hi = s1, t = 0.5 * (s0 + s1);
    for (int it = 0; it < 400; ++it) {
      double f = S.cdf - S.u, fp = 0.0;
      for (const Hit* h : act) {
        f += 0.5 * ray_integral(*h, s0, t);
        fp += 0.5 * gauss_at(*h, t);
      }
      if (f == 0.0) break;
      if (f < 0) lo = t; else hi = t;
      double tn = fp > 0 ? t - f / fp : 0.5 * (lo + hi);
      if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
      const bool stop = std::fabs(tn - t) <= 1e-16 * std::max(1.0, std::fabs(t)) ||
                        hi - lo <= 1e-16 * std::max(1.0, std::fabs(t));
      t = tn;
      if (stop) break;
    }
    S.st.ambiguous_start = s0;
    const double u_seg = S.cdf + S.u2 * (S.u - S.cdf);
    for (const Hit* h : act) {
      S.cdf += 0.5 * ray_integral(*h, s0, t);
      if (u_seg < S.cdf) {
        S.result = h->id;
        S.done = true;
        return;
      }
    }
    S.result = act.back()->id;  // rounding: the running sum ends a hair below u_seg
    S.done = true;
    return;
  }
}

void traverse(KdSample& S, const KdTree& T, int node, double ta, double tb) {
  if (S.done || !(ta < tb)) return;
  ++S.st.nodes_visited;
  const KdNode& nd = T.nodes[size_t(node)];
  if (nd.axis < 0) {
    leaf(S, T, nd, ta, tb);
    return;
  }
  const double oa = nd.axis == 0 ? S.o.x : nd.axis == 1 ? S.o.y : S.o.z;
  const double da = nd.axis == 0 ? S.d.x : nd.axis == 1 ? S.d.y : S.d.z;
  const int nearc = (oa < nd.pos || (oa == nd.pos && da <= 0)) ? 0 : 1;
  if (da == 0.0) {
    traverse(S, T, nd.child[nearc], ta, tb);
    return;
  }
  const double ts = (nd.pos - oa) / da;
  if (ts >= tb || ts <= 0) {
    traverse(S, T, nd.child[nearc], ta, tb);
  } else if (ts <= ta) {
    traverse(S, T, nd.child[1 - nearc], ta, tb);
  } else {
    traverse(S, T, nd.child[nearc], ta, ts);
    traverse(S, T, nd.child[1 - nearc], ts, tb);
  }
}

}  // namespace

int32_t kd_sample_free_flight(const KdTree& T, const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1,
                              double k, double u, double u2, KdStats* stats) {
  KdSample S{prims, o, d, t0, t1, k, u, u2};
  S.st.ambiguous_start = std::numeric_limits<double>::quiet_NaN();
  if (!T.nodes.empty()) {
    // the ray's range inside the root box
    double ta = t0, tb = t1;
    const double ov[3] = {o.x, o.y, o.z}, dv[3] = {d.x, d.y, d.z};
    for (int a = 0; a < 3; ++a) {
      if (dv[a] == 0.0) {
        if (ov[a] < T.lo[a] || ov[a] > T.hi[a]) tb = ta;
        continue;
      }
      double x0 = (T.lo[a] - ov[a]) / dv[a], x1 = (T.hi[a] - ov[a]) / dv[a];
      if (x0 > x1) std::swap(x0, x1);
      ta = std::max(ta, x0);
      tb = std::min(tb, x1);
    }
    traverse(S, T, 0, ta, tb);
  }
  S.st.F_end = S.cdf;
  if (stats) *stats = S.st;
  return S.done ? S.result : -1;
}

}  // namespace orc
