// Light sampling toward emissive primitives (the paper renders its emitters only by
// unidirectional hits; this is the light-sampling technique for them, balanced against phase
// sampling).
//
// The free flight from a vertex x along w picks primitive j in [t, t + dt] with probability
// 1/2 G_j(x + t w) dt while t is below the saturating distance (Eq. 8 and the exact choice of
// Sec. 5.2). The direct emission of j is then 1/2 L_e,j int f_p(w(y)) G_j(y) 1[|y - x| < t_sat]
// / |y - x|^2 dy, and with j drawn with probability pi_j proportional to c_j mean(L_e,j) and y
// from G_j / (c_j m) inside the k-ellipsoid (m = P(chi_3 <= k)), one sample estimates it by
//   1/2 c_j m L_e,j f_p 1[T(x, y) > 0] / (|y - x|^2 pi_j)
// (the linear model needs only that y lies before saturation, no transmittance factor).
// Balance heuristic against phase sampling: 2 r_c^2 pi_j against c_j m p(w), r_c the distance
// from x to the emitter's mean (the two techniques' densities of (j, y) in volume measure, with
// r_c for |y - x| so that a path reaching j by phase sampling can form the same weight).
#pragma once

#include "ugp_internal.cuh"

namespace ugp {

// Table layout (device buffer, 256-byte aligned):
//   header (256 B): int64 n_em, double total, int64 n_prims
//   cdf   double[n_prims]  running sums of c mean(L_e) over the emitters, in caller order
//   rec   float4[4 n_prims] per emitter: (RS row 0, mu.x), (RS row 1, mu.y), (RS row 2, mu.z),
//                          (c m, L_e)
//   map   int32[n_prims]   caller index -> emitter index, -1 for other primitives
struct EmitterLayout {
  size_t cdf, rec, map, total;
};
inline EmitterLayout emitter_layout(int64_t n) {
  EmitterLayout L;
  L.cdf = 256;
  L.rec = L.cdf + align256(size_t(n) * 8);
  L.map = L.rec + align256(size_t(n) * 64);
  L.total = L.map + align256(size_t(n) * 4);
  return L;
}

struct EmitterDev {
  const long long* hdr;  // n_em, (total as double bits), n_prims
  const double* cdf;     // nullptr: no light sampling of emitters
  const float4* rec;
  const int* map;
  long long n_prims;     // the scene's, checked against the table's on the device
  float k, mass;         // ellipsoid cut-off and the Gaussian mass inside it
};

// Device view of a table from ugp_build_emitter_table (all null for table == NULL).
EmitterDev emitter_dev(const void* table, const ugp_bvh* bvh);

// CDF of the chi distribution with 3 degrees of freedom.
__device__ __forceinline__ float chi3_cdf_f(float r) {
  return erff(r * 0.70710678118654752f) - 0.79788456080286536f * r * expf(-0.5f * r * r);
}

// Radius with chi3_cdf_f(r) = target in [0, k): bracketed Newton, at most 40 steps.
__device__ __forceinline__ float chi3_radius(float target, float k) {
  float lo = 0.f, hi = k, r = fminf(1.5382f, 0.5f * k);
  for (int it = 0; it < 40; ++it) {
    const float f = chi3_cdf_f(r) - target;
    if (f < 0.f) lo = r; else hi = r;
    const float fp = 0.79788456080286536f * r * r * expf(-0.5f * r * r);
    float rn = fp > 0.f ? r - f / fp : 0.5f * (lo + hi);
    if (!(rn > lo && rn < hi)) rn = 0.5f * (lo + hi);
    const bool done = fabsf(rn - r) <= 1e-6f * r || hi - lo <= 1e-6f;
    r = rn;
    if (done) break;
  }
  return r;
}

__device__ __forceinline__ bool emitters_on(const EmitterDev& E) {
  return E.cdf != nullptr && E.hdr[0] > 0 && E.hdr[2] == E.n_prims;
}
__device__ __forceinline__ double emitters_total(const EmitterDev& E) { return __longlong_as_double(E.hdr[1]); }

// Probability pi of emitter e.
__device__ __forceinline__ float emitter_prob(const EmitterDev& E, long long e) {
  const double prev = e > 0 ? E.cdf[e - 1] : 0.0;
  return float((E.cdf[e] - prev) / emitters_total(E));
}

// Emitter whose CDF interval holds u in [0, 1): the first e with cdf[e] > u * total.
__device__ __forceinline__ long long emitter_pick(const EmitterDev& E, float u) {
  const double target = double(u) * emitters_total(E);
  long long lo = 0, hi = E.hdr[0] - 1;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (E.cdf[mid] > target) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

}  // namespace ugp
