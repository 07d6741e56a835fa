// FP64 oracle: a plain bounding-volume hierarchy over the primitives' k-ellipsoid boxes, used to
// time the oracle's renderer on large scenes (the CPU baseline). It finds exactly the intervals
// the brute-force loop of all_hits finds, since a ray meets a primitive's ellipsoid only inside
// the primitive's box: the renderer's results do not change, only the order in which intervals
// are found, and every sum over them is ordered or order-free in double precision.
//
// TEST INFRASTRUCTURE ONLY. Build: recursive split at the median centroid along the longest
// centroid extent (std::nth_element), leaves of at most 8 primitives; boxes widened by a few
// ulps so that a grazing ray never misses a box its ellipsoid touches.
#include <algorithm>
#include <cmath>
#include <limits>

#include "oracle_internal.h"

namespace orc {

const Accel* g_accel = nullptr;

namespace {

constexpr int kAccelLeaf = 8;

void prim_bounds(const Prim& p, double k, double lo[3], double hi[3]) {
  const double m[3] = {p.mu.x, p.mu.y, p.mu.z};
  for (int r = 0; r < 3; ++r) {
    double e2 = 0;
    for (int c = 0; c < 3; ++c) e2 += (p.R[3 * r + c] * p.s[c]) * (p.R[3 * r + c] * p.s[c]);
    const double e = k * std::sqrt(e2) * (1.0 + 1e-12) + 1e-15 * std::fabs(m[r]);
    lo[r] = m[r] - e;
    hi[r] = m[r] + e;
  }
}

struct Build {
  const std::vector<Prim>& prims;
  double k;
  Accel& A;
  std::vector<double> lo, hi;  // 3 per primitive
  int node(int32_t b, int32_t e) {
    const int me = int(A.nodes.size());
    A.nodes.push_back(AccelNode{});
    double nlo[3], nhi[3], clo[3], chi[3];
    for (int a = 0; a < 3; ++a) {
      nlo[a] = clo[a] = std::numeric_limits<double>::infinity();
      nhi[a] = chi[a] = -std::numeric_limits<double>::infinity();
    }
    for (int32_t i = b; i < e; ++i) {
      const int32_t id = A.ids[size_t(i)];
      for (int a = 0; a < 3; ++a) {
        nlo[a] = std::min(nlo[a], lo[3 * size_t(id) + a]);
        nhi[a] = std::max(nhi[a], hi[3 * size_t(id) + a]);
        const double c = 0.5 * (lo[3 * size_t(id) + a] + hi[3 * size_t(id) + a]);
        clo[a] = std::min(clo[a], c);
        chi[a] = std::max(chi[a], c);
      }
    }
    for (int a = 0; a < 3; ++a) {
      A.nodes[size_t(me)].lo[a] = nlo[a];
      A.nodes[size_t(me)].hi[a] = nhi[a];
    }
    if (e - b <= kAccelLeaf) {
      A.nodes[size_t(me)].first = b;
      A.nodes[size_t(me)].count = e - b;
      return me;
    }
    int ax = 0;
    for (int a = 1; a < 3; ++a)
      if (chi[a] - clo[a] > chi[ax] - clo[ax]) ax = a;
    const int32_t mid = b + (e - b) / 2;
    std::nth_element(A.ids.begin() + b, A.ids.begin() + mid, A.ids.begin() + e, [&](int32_t x, int32_t y) {
      const double cx = lo[3 * size_t(x) + ax] + hi[3 * size_t(x) + ax];
      const double cy = lo[3 * size_t(y) + ax] + hi[3 * size_t(y) + ax];
      return cx < cy || (cx == cy && x < y);
    });
    const int l = node(b, mid);
    const int r = node(mid, e);
    A.nodes[size_t(me)].left = l;
    A.nodes[size_t(me)].right = r;
    return me;
  }
};

bool slab(const AccelNode& n, V3 o, V3 d, double t0, double t1) {
  const double ov[3] = {o.x, o.y, o.z}, dv[3] = {d.x, d.y, d.z};
  double a = t0, b = t1;
  for (int ax = 0; ax < 3; ++ax) {
    if (dv[ax] == 0.0) {
      if (ov[ax] < n.lo[ax] || ov[ax] > n.hi[ax]) return false;
      continue;
    }
    double x0 = (n.lo[ax] - ov[ax]) / dv[ax], x1 = (n.hi[ax] - ov[ax]) / dv[ax];
    if (x0 > x1) std::swap(x0, x1);
    a = std::max(a, x0);
    b = std::min(b, x1);
  }
  return a <= b * (1.0 + 1e-12) + 1e-300;
}

}  // namespace

Accel accel_build(const std::vector<Prim>& prims, double k) {
  Accel A;
  A.prims = &prims;
  if (prims.empty()) return A;
  A.ids.resize(prims.size());
  for (size_t i = 0; i < prims.size(); ++i) A.ids[i] = int32_t(i);
  Build B{prims, k, A, std::vector<double>(3 * prims.size()), std::vector<double>(3 * prims.size())};
  for (size_t i = 0; i < prims.size(); ++i) prim_bounds(prims[i], k, &B.lo[3 * i], &B.hi[3 * i]);
  B.node(0, int32_t(prims.size()));
  return A;
}

std::vector<Hit> accel_hits(const Accel& A, V3 o, V3 d, double t0, double t1, double k, int32_t exclude) {
  std::vector<Hit> hits;
  if (A.nodes.empty()) return hits;
  std::vector<int> stack{0};
  while (!stack.empty()) {
    const AccelNode& n = A.nodes[size_t(stack.back())];
    stack.pop_back();
    if (!slab(n, o, d, t0, t1)) continue;
    if (n.count > 0 || n.left < 0) {
      for (int32_t j = n.first; j < n.first + n.count; ++j) {
        const int32_t i = A.ids[size_t(j)];
        if (i == exclude) continue;
        Hit h;
        if (ray_prim((*A.prims)[size_t(i)], i, o, d, t0, t1, k, &h)) hits.push_back(h);
      }
      continue;
    }
    stack.push_back(n.right);
    stack.push_back(n.left);
  }
  // the brute-force loop's order (ascending index), so that every later step sees the same list
  std::sort(hits.begin(), hits.end(), [](const Hit& x, const Hit& y) { return x.id < y.id; });
  return hits;
}

}  // namespace orc
