// FP64 oracle: the paper's own free-flight sampler (Sec. 5.2, Eq. 8-10), a diagnostic for the
// paper-faithful variant; the order-free sampler of geometry.cpp is the parity target.
//
// TEST INFRASTRUCTURE ONLY.
//  * An SAH kd-tree over the primitives' k-ellipsoid boxes (primitives straddling a plane go to
//    both sides), built by trying the box faces of every primitive as planes.
//  * Front-to-back traversal: each leaf covers a range [ta, tb] of the ray, and the leaves'
//    ranges partition [t0, t1]; a primitive contributes I_k over its clipped interval within the
//    range.
//  * The CDF is the running sum of 1/2 I_k in the order the walk meets the primitives. A leaf
//    (or, inside a leaf, a segment of constant overlap set) that cannot bring it to 1 adds its
//    masses in order, and the sample is the primitive whose mass u falls in.
//  * Where the CDF reaches 1, no order can be trusted: t_u solves F(t_u) = u in that segment and
//    the primitive is chosen among the segment's overlapping ones with probability proportional
//    to I_k(s0, t_u) (Eq. 10), using u2.
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
  int nbins = 0;  // > 0: the paper's GPU partition of an ambiguous leaf into nbins equal bins
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

// Takes masses one after another (the front-to-back accumulation of Sec. 5.2): if u falls below
// cdf + the running sum, the primitive whose mass it falls in is the sample; otherwise the masses
// are added to cdf. Returns whether a primitive was chosen.
bool take_in_order(KdSample& S, const std::vector<int32_t>& ids, const std::vector<double>& mass) {
  double total = 0.0;
  for (double m : mass) total += m;
  if (!(S.u < S.cdf + total)) {
    S.cdf += total;
    return false;
  }
  double c = S.cdf;
  size_t k = 0;
  while (k + 1 < mass.size() && !(S.u < c + mass[k])) c += mass[k++];
  S.result = ids[k];
  S.done = true;
  return true;
}

// F(t) = u inside a segment [s0, s1] whose active primitives bring the CDF from S.cdf below u to
// at least 1 > u at s1 (Eq. 8-9): safeguarded Newton, F' = 1/2 sum G_k.
double solve_in_segment(const KdSample& S, const std::vector<const Hit*>& act, double s0, double s1) {
  double lo = s0, hi = s1, t = 0.5 * (s0 + s1);
  for (int it = 0; it < 400; ++it) {
    double f = S.cdf - S.u, fp = 0.0;
    for (const Hit* h : act) {
      f += 0.5 * ray_integral(*h, s0, t);
      fp += 0.5 * gauss_at(*h, t);
    }
    if (f == 0.0) break;
    (f < 0 ? lo : hi) = t;
    double tn = fp > 0 ? t - f / fp : 0.5 * (lo + hi);
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    const bool stop = std::fabs(tn - t) <= 1e-16 * std::max(1.0, std::fabs(t)) ||
                      hi - lo <= 1e-16 * std::max(1.0, std::fabs(t));
    t = tn;
    if (stop) break;
  }
  return t;
}

// One leaf of the front-to-back walk: the primitives' intervals clipped to the leaf's range
// [ta, tb] of the ray.
//  * If the leaf cannot bring the CDF to 1, or holds one primitive, its masses 1/2 I_k are taken
//    in the leaf's order.
//  * Otherwise the range splits at every interval end into segments of constant overlap set.
//    Segments before the one where the CDF reaches 1 (and any with one primitive) are taken the
//    same way; in the segment where it reaches 1, t_u solves F(t_u) = u and the primitive is
//    chosen with probability proportional to I_k(s0, t_u) (Eq. 10), using u2.
void leaf(KdSample& S, const KdTree& T, const KdNode& nd, double ta, double tb) {
  std::vector<Hit> hs;
  for (int j = 0; j < nd.count; ++j) {
    Hit h;
    ++S.st.prims_tested;
    if (part(S, T.leaf_ids[size_t(nd.first + j)], ta, tb, &h)) hs.push_back(h);
  }
  if (hs.empty()) return;
  std::vector<int32_t> ids;
  std::vector<double> mass;
  double leaf_mass = 0.0;
  for (const Hit& h : hs) {
    ids.push_back(h.id);
    mass.push_back(0.5 * ray_integral(h, h.a, h.b));
    leaf_mass += mass.back();
  }
  if (hs.size() == 1 || S.cdf + leaf_mass < 1.0) {
    take_in_order(S, ids, mass);
    return;
  }
  if (S.nbins > 0) {
    // the paper's GPU partition: equal bins of the ray-node interval [ta, tb], each classified
    // like a leaf; in the bin where the CDF reaches 1, t_u is solved from the bin's start and the
    // primitive drawn proportionally to I_k(bin start, t_u) among those overlapping the bin
    const double w = (tb - ta) / S.nbins;
    for (int b = 0; b < S.nbins; ++b) {
      const double s0 = ta + w * b, s1 = b + 1 == S.nbins ? tb : ta + w * (b + 1);
      std::vector<const Hit*> act;
      std::vector<int32_t> act_ids;
      std::vector<double> bin_mass;
      double bin_total = 0.0;
      for (const Hit& h : hs) {
        const double x = std::max(h.a, s0), y = std::min(h.b, s1);
        if (!(x < y)) continue;
        act.push_back(&h);
        act_ids.push_back(h.id);
        bin_mass.push_back(0.5 * ray_integral(h, x, y));
        bin_total += bin_mass.back();
      }
      if (act.empty()) continue;
      if (act.size() == 1 || S.cdf + bin_total < 1.0) {
        if (take_in_order(S, act_ids, bin_mass)) return;
        continue;
      }
      // F(t) = cdf + sum 1/2 I_k(max(a_k, s0), min(b_k, t)) = u, bracketed Newton
      auto F = [&](double t, double* fp) {
        double f = S.cdf - S.u, g = 0.0;
        for (const Hit* h : act) {
          const double x = std::max(h->a, s0), y = std::min(h->b, t);
          if (x < y) f += 0.5 * ray_integral(*h, x, y);
          if (h->a <= t && t <= h->b) g += 0.5 * gauss_at(*h, t);
        }
        *fp = g;
        return f;
      };
      double lo = s0, hi = s1, t = 0.5 * (s0 + s1);
      for (int it = 0; it < 400; ++it) {
        double fp;
        const double f = F(t, &fp);
        if (f == 0.0) break;
        (f < 0 ? lo : hi) = t;
        double tn = fp > 0 ? t - f / fp : 0.5 * (lo + hi);
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        const bool stop = std::fabs(tn - t) <= 1e-16 * std::max(1.0, std::fabs(t)) ||
                          hi - lo <= 1e-16 * std::max(1.0, std::fabs(t));
        t = tn;
        if (stop) break;
      }
      S.st.ambiguous_start = s0;
      std::vector<double> wk;
      double w_total = 0.0;
      for (const Hit* h : act) {
        const double x = std::max(h->a, s0), y = std::min(h->b, t);
        wk.push_back(x < y ? ray_integral(*h, x, y) : 0.0);
        w_total += wk.back();
      }
      double c = 0.0;
      size_t k = 0;
      while (k + 1 < wk.size() && !(wk[k] > 0.0 && S.u2 * w_total < c + wk[k])) c += wk[k++];
      S.result = act_ids[k];
      S.done = true;
      return;
    }
    return;
  }
  std::vector<double> ends;
  for (const Hit& h : hs) {
    ends.push_back(h.a);
    ends.push_back(h.b);
  }
  std::sort(ends.begin(), ends.end());
  ends.erase(std::unique(ends.begin(), ends.end()), ends.end());
  for (size_t s = 0; s + 1 < ends.size(); ++s) {
    const double s0 = ends[s], s1 = ends[s + 1];
    std::vector<const Hit*> act;
    std::vector<int32_t> act_ids;
    std::vector<double> seg_mass;
    double seg_total = 0.0;
    for (const Hit& h : hs)
      if (h.a <= s0 && h.b >= s1) {
        act.push_back(&h);
        act_ids.push_back(h.id);
        seg_mass.push_back(0.5 * ray_integral(h, s0, s1));
        seg_total += seg_mass.back();
      }
    if (act.empty()) continue;
    if (act.size() == 1 || S.cdf + seg_total < 1.0) {
      if (take_in_order(S, act_ids, seg_mass)) return;
      continue;
    }
    const double t_u = solve_in_segment(S, act, s0, s1);
    S.st.ambiguous_start = s0;
    std::vector<double> w;
    double w_total = 0.0;
    for (const Hit* h : act) {
      w.push_back(ray_integral(*h, s0, t_u));
      w_total += w.back();
    }
    double c = 0.0;
    size_t k = 0;
    while (k + 1 < w.size() && !(S.u2 * w_total < c + w[k])) c += w[k++];
    S.result = act_ids[k];
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
                              double k, double u, double u2, KdStats* stats, int nbins) {
  KdSample S{prims, o, d, t0, t1, k, u, u2};
  S.nbins = nbins;
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
