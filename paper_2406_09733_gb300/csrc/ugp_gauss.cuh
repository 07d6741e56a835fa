// Device math of one Gaussian primitive along one ray (Eq. 1, Eq. 4, Eq. 6, App. A),
// written for float32 accuracy, plus the BVH slab test.
//
// Accuracy.  Thin primitives (scales ~1e-5 at distance ~1) make the textbook form
// A t^2 + B t + C cancel catastrophically in float32.  The test below therefore
//   1. forms p = o - mu exactly as a float pair (TwoSum),
//   2. moves the origin to the Euclidean closest approach t_n = -p.d / d.d, where the
//      residual q = p + t_n d is small and is formed with one FMA per component,
//   3. whitens q and d with W = S^-1 R^T and completes the square there:
//      |W(q + t' d)|^2 = A (t' - t_s)^2 + d2, A = |Wd|^2, t_s = -(Wq.Wd)/A.
// The closest approach of Eq. 6 is t* = t_n + t_s; the two parts are kept separate so
// that erf arguments tau(t) = sqrt(A/2) ((t - t_n) - t_s) keep full relative precision.
#pragma once

#include <math.h>

#include "ugp_internal.cuh"

namespace ugp {

constexpr float kSqrtPi = 1.7724538509055160f;

struct Ray {
  float3 o, d, inv;
  float inv_dd;
};

__device__ __forceinline__ Ray make_ray(float3 o, float3 d) {
  Ray r;
  r.o = o;
  r.d = d;
  const float tiny = 1e-30f;
  r.inv.x = 1.f / (fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x));
  r.inv.y = 1.f / (fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y));
  r.inv.z = 1.f / (fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z));
  r.inv_dd = 1.f / (d.x * d.x + d.y * d.y + d.z * d.z);
  return r;
}

// One clipped primitive interval with the quantities needed for its integral.
struct PrimHit {
  float a, b;   // [max(t0, t*-h), min(t1, t*+h)]
  float tn, ts; // t* = tn + ts
  float s;      // sqrt(A / 2)
  float e0;     // g0 exp(-d2 / 2): peak of G along the ray
  int id;       // caller's primitive index
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Tests primitive `slot` against the ray over [t0, t1].  Returns false if the ray misses the
// k-ellipsoid (d2 >= k^2), if the clipped interval is empty, if the primitive is the
// excluded one, or if it was flagged invalid at build time.
__device__ __forceinline__ bool prim_test(const float4* __restrict__ recs, int slot, const Ray& r,
                                          float t0, float t1, float k2, int exclude, PrimHit& h) {
  const float4 r3 = __ldg(recs + 4 * slot + 3);
  const int id = __float_as_int(r3.y);
  if (id == exclude || r3.z == 0.f) return false;
  const float4 r0 = __ldg(recs + 4 * slot + 0);
  const float4 r1 = __ldg(recs + 4 * slot + 1);
  const float4 r2 = __ldg(recs + 4 * slot + 2);
  float px, lx, py, ly, pz, lz;
  two_sum(r.o.x, -r0.w, px, lx);
  two_sum(r.o.y, -r1.w, py, ly);
  two_sum(r.o.z, -r2.w, pz, lz);
  const float tn = -fmaf(px, r.d.x, fmaf(py, r.d.y, pz * r.d.z)) * r.inv_dd;
  const float qx = fmaf(tn, r.d.x, px) + lx;
  const float qy = fmaf(tn, r.d.y, py) + ly;
  const float qz = fmaf(tn, r.d.z, pz) + lz;
  const float ox = fmaf(r0.x, qx, fmaf(r0.y, qy, r0.z * qz));
  const float oy = fmaf(r1.x, qx, fmaf(r1.y, qy, r1.z * qz));
  const float oz = fmaf(r2.x, qx, fmaf(r2.y, qy, r2.z * qz));
  const float dx = fmaf(r0.x, r.d.x, fmaf(r0.y, r.d.y, r0.z * r.d.z));
  const float dy = fmaf(r1.x, r.d.x, fmaf(r1.y, r.d.y, r1.z * r.d.z));
  const float dz = fmaf(r2.x, r.d.x, fmaf(r2.y, r.d.y, r2.z * r.d.z));
  const float A = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float invA = 1.f / A;
  const float ts = -fmaf(ox, dx, fmaf(oy, dy, oz * dz)) * invA;
  const float cx = fmaf(ts, dx, ox), cy = fmaf(ts, dy, oy), cz = fmaf(ts, dz, oz);
  const float d2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
  if (!(d2 < k2)) return false;
  const float half = sqrtf((k2 - d2) * invA);
  const float tc = tn + ts;
  const float a = fmaxf(t0, tc - half), b = fminf(t1, tc + half);
  if (!(a < b)) return false;
  h.a = a;
  h.b = b;
  h.tn = tn;
  h.ts = ts;
  h.s = sqrtf(0.5f * A);
  h.e0 = r3.x * expf(-0.5f * d2);
  h.id = id;
  return true;
}

__device__ __forceinline__ float tau_at(float t, float tn, float ts, float s) { return s * ((t - tn) - ts); }

// 1/2 I(x, y) of App. A: 1/2 g0 e^{-d2/2} sqrt(pi / 2A) [erf(tau_y) - erf(tau_x)], with
// sqrt(pi / 2A) = sqrt(pi) / (2 s).  Same-sign arguments use erfc to avoid cancellation.
__device__ __forceinline__ float half_integral(float x, float y, float tn, float ts, float s, float e0) {
  const float tx = tau_at(x, tn, ts, s), ty = tau_at(y, tn, ts, s);
  float diff;
  if (tx >= 0.f)
    diff = erfcf(tx) - erfcf(ty);
  else if (ty <= 0.f)
    diff = erfcf(-ty) - erfcf(-tx);
  else
    diff = erff(ty) - erff(tx);
  return e0 * (0.25f * kSqrtPi) / s * diff;
}

// G(x_t) of Eq. 1 along the ray: e0 exp(-tau^2).
__device__ __forceinline__ float gauss_at(float t, float tn, float ts, float s, float e0) {
  const float tt = tau_at(t, tn, ts, s);
  return e0 * expf(-tt * tt);
}

// Slab test of a box against [tmin, tmax]; tent receives the clipped entry distance.
__device__ __forceinline__ bool slab(float lx, float ly, float lz, float hx, float hy, float hz,
                                     const Ray& r, float tmin, float tmax, float& tent) {
  const float x0 = (lx - r.o.x) * r.inv.x, x1 = (hx - r.o.x) * r.inv.x;
  const float y0 = (ly - r.o.y) * r.inv.y, y1 = (hy - r.o.y) * r.inv.y;
  const float z0 = (lz - r.o.z) * r.inv.z, z1 = (hz - r.o.z) * r.inv.z;
  const float tl = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), tmin));
  const float th = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), tmax));
  tent = tl;
  // a few ulps of slack keep the test conservative against rounding
  return tl <= th + 4e-7f * fabsf(th);
}

__device__ __forceinline__ float3 ld3(const float* __restrict__ p, int64_t i) {
  return make_float3(__ldg(p + 3 * i), __ldg(p + 3 * i + 1), __ldg(p + 3 * i + 2));
}

// Warp-aggregated statistics update (threads of a warp that already returned are left out):
// nodes loaded, primitive records loaded, rays, traversal rounds, rays that needed the binned mode.
__device__ __forceinline__ void add_counters(unsigned long long* ctr, unsigned a, unsigned b,
                                             unsigned c, unsigned d, unsigned e) {
  const unsigned mask = __activemask();
  a = __reduce_add_sync(mask, a);
  b = __reduce_add_sync(mask, b);
  c = __reduce_add_sync(mask, c);
  d = __reduce_add_sync(mask, d);
  e = __reduce_add_sync(mask, e);
  if ((threadIdx.x & 31) == unsigned(__ffs(mask) - 1)) {
    atomicAdd(ctr + 0, (unsigned long long)a);
    atomicAdd(ctr + 1, (unsigned long long)b);
    atomicAdd(ctr + 2, (unsigned long long)c);
    atomicAdd(ctr + 3, (unsigned long long)d);
    if (e) atomicAdd(ctr + 4, (unsigned long long)e);
  }
}

}  // namespace ugp
