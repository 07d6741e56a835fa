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
  float th;     // tau at the ellipsoid's exit, sqrt((k^2 - d2) / 2) (-th at its entry)
  int id;       // caller's primitive index
  bool a_end;   // a is the ellipsoid entry (not clipped by t0)
  bool b_end;   // b is the ellipsoid exit (not clipped by t1)
};

// An interval end that is the ellipsoid boundary has the exact erf argument -th / +th; taking
// it from the float32 end point instead would cost s * ulp(t), large for thin primitives.
// Flags travel in the two top bits of a stored index (indices are below 2^30).
constexpr int kIdMask = 0x3fffffff;
__device__ __forceinline__ int pack_id(const PrimHit& h) {
  return h.id | (h.a_end ? 0x40000000 : 0) | (h.b_end ? int(0x80000000u) : 0);
}
__device__ __forceinline__ int unpack_id(int p) { return p & kIdMask; }
__device__ __forceinline__ bool packed_a_end(int p) { return (p & 0x40000000) != 0; }
__device__ __forceinline__ bool packed_b_end(int p) { return (p & int(0x80000000u)) != 0; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// ---- double-float helpers (value = h + l), built from correctly rounded intrinsics so the
// compiler cannot contract them into FMAs ---------------------------------------------------
struct dsf {
  float h, l;
};
__device__ __forceinline__ dsf ds_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dsf ds_norm(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dsf ds_add(dsf a, dsf b) {
  const dsf s = ds_two_sum(a.h, b.h);
  return ds_norm(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dsf ds_mul(dsf a, dsf b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = __fmaf_rn(a.h, b.h, -p);
  return ds_norm(p, __fadd_rn(e, __fadd_rn(__fmul_rn(a.h, b.l), __fmul_rn(a.l, b.h))));
}
__device__ __forceinline__ dsf ds_div(dsf a, dsf b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const dsf r = ds_add(a, ds_mul({-q1, 0.f}, b));
  return ds_norm(q1, __fdiv_rn(r.h, b.h));
}

// Whitened coordinates of a ray relative to one primitive, in double-float arithmetic:
// q = p + tn d (p = o - mu as an exact pair), o' = W q, d' = W d with W = hi + lo, then the
// closest approach t_s = -(o'.d')/A and d2 = |o' + t_s d'|^2.  Used only for hits whose float32
// evaluation is ill-conditioned (large whitened terms cancelling to a small result).
static __device__ __noinline__ void refine_ds(const float4 r0, const float4 r1, const float4 r2,
                                       const float4* __restrict__ lo3, const float3 ph, const float3 pl,
                                       float tn, const float3 d, float& A_out, float& ts_out, float& d2_out) {
  const float4 l0 = __ldg(lo3), l1 = __ldg(lo3 + 1), l2 = __ldg(lo3 + 2);
  const float phv[3] = {ph.x, ph.y, ph.z}, plv[3] = {pl.x, pl.y, pl.z}, dv[3] = {d.x, d.y, d.z};
  dsf q[3];
  for (int j = 0; j < 3; ++j) {
    const float P = __fmul_rn(tn, dv[j]);
    const float Pe = __fmaf_rn(tn, dv[j], -P);
    const dsf S = ds_two_sum(phv[j], P);
    q[j] = ds_norm(S.h, __fadd_rn(S.l, __fadd_rn(Pe, plv[j])));
  }
  const float Wh[9] = {r0.x, r0.y, r0.z, r1.x, r1.y, r1.z, r2.x, r2.y, r2.z};
  const float Wl[9] = {l0.x, l0.y, l0.z, l1.x, l1.y, l1.z, l2.x, l2.y, l2.z};
  dsf o[3], w[3];
  for (int i = 0; i < 3; ++i) {
    dsf so = {0.f, 0.f}, sd = {0.f, 0.f};
    for (int j = 0; j < 3; ++j) {
      const dsf W = {Wh[3 * i + j], Wl[3 * i + j]};
      so = ds_add(so, ds_mul(W, q[j]));
      sd = ds_add(sd, ds_mul(W, {dv[j], 0.f}));
    }
    o[i] = so;
    w[i] = sd;
  }
  dsf A = {0.f, 0.f}, od = {0.f, 0.f};
  for (int i = 0; i < 3; ++i) {
    A = ds_add(A, ds_mul(w[i], w[i]));
    od = ds_add(od, ds_mul(o[i], w[i]));
  }
  dsf ts = ds_div(od, A);
  ts = {-ts.h, -ts.l};
  dsf d2 = {0.f, 0.f};
  for (int i = 0; i < 3; ++i) {
    const dsf ci = ds_add(o[i], ds_mul(ts, w[i]));
    d2 = ds_add(d2, ds_mul(ci, ci));
  }
  A_out = A.h;
  ts_out = ts.h;
  d2_out = __fadd_rn(d2.h, d2.l);
}

// Whitened magnitude above which a hit is recomputed in double-float arithmetic: the float32
// error of d is about 1e-7 times the largest |W_ij q_j|, so below this it stays under 1e-6.
constexpr float kRefineAbove = 8.f;

// Tests primitive `slot` against the ray over [t0, t1].  Returns false if the ray misses the
// k-ellipsoid (d2 >= k^2), if the clipped interval is empty, if the primitive is the
// excluded one, or if it was flagged invalid at build time.
__device__ __forceinline__ bool prim_test(const float4* __restrict__ recs, const float4* __restrict__ wlo,
                                          int slot, const Ray& r, float t0, float t1, float k2, int exclude,
                                          PrimHit& h) {
  // the whole 64-byte record in one round of loads (the exclusion and validity test rarely ends
  // the test, so the other three loads need not wait for it)
  const float4 r0 = __ldg(recs + 4 * slot + 0);
  const float4 r1 = __ldg(recs + 4 * slot + 1);
  const float4 r2 = __ldg(recs + 4 * slot + 2);
  const float4 r3 = __ldg(recs + 4 * slot + 3);
  const int id = __float_as_int(r3.y);
  if (id == exclude || r3.z == 0.f) return false;
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
  float A = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  float ts = -fmaf(ox, dx, fmaf(oy, dy, oz * dz)) / A;
  const float cx = fmaf(ts, dx, ox), cy = fmaf(ts, dy, oy), cz = fmaf(ts, dz, oz);
  float d2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
  if (!(d2 < k2 * 1.0001f)) return false;
  // conditioning: largest whitened term that took part in a cancellation
  const float aqx = fabsf(qx), aqy = fabsf(qy), aqz = fabsf(qz);
  const float m0 = fabsf(r0.x) * aqx + fabsf(r0.y) * aqy + fabsf(r0.z) * aqz;
  const float m1 = fabsf(r1.x) * aqx + fabsf(r1.y) * aqy + fabsf(r1.z) * aqz;
  const float m2 = fabsf(r2.x) * aqx + fabsf(r2.y) * aqy + fabsf(r2.z) * aqz;
  if (fmaxf(m0, fmaxf(m1, m2)) > kRefineAbove)
    refine_ds(r0, r1, r2, wlo + 3 * slot, make_float3(px, py, pz), make_float3(lx, ly, lz), tn, r.d, A, ts, d2);
  if (!(d2 < k2)) return false;
  const float half = sqrtf((k2 - d2) / A);
  const float tc = tn + ts;
  const float a = fmaxf(t0, tc - half), b = fminf(t1, tc + half);
  if (!(a < b)) return false;
  h.a = a;
  h.b = b;
  h.tn = tn;
  h.ts = ts;
  h.s = sqrtf(0.5f * A);
  h.e0 = r3.x * expf(-0.5f * d2);
  h.th = sqrtf(0.5f * (k2 - d2));
  h.id = id;
  h.a_end = tc - half >= t0;
  h.b_end = tc + half <= t1;
  return true;
}

__device__ __forceinline__ float tau_at(float t, float tn, float ts, float s) { return s * ((t - tn) - ts); }

// 1/2 I between erf arguments tx <= ty (App. A): 1/2 g0 e^{-d2/2} sqrt(pi / 2A) [erf(ty) - erf(tx)],
// with sqrt(pi / 2A) = sqrt(pi) / (2 s).  Same-sign arguments use erfc to avoid cancellation.
__device__ __forceinline__ float half_integral_tau(float tx, float ty, float s, float e0) {
  float diff;
  if (tx >= 0.f)
    diff = erfcf(tx) - erfcf(ty);
  else if (ty <= 0.f)
    diff = erfcf(-ty) - erfcf(-tx);
  else
    diff = erff(ty) - erff(tx);
  return e0 * (0.25f * kSqrtPi) / s * diff;
}

// 1/2 I(x, y) for a sub-range [x, y] of a clipped interval [a, b].
__device__ __forceinline__ float seg_half_integral(float x, float y, float a, float b, bool a_end, bool b_end,
                                                   float tn, float ts, float s, float e0, float th) {
  const float tx = (a_end && x == a) ? -th : tau_at(x, tn, ts, s);
  const float ty = (b_end && y == b) ? th : tau_at(y, tn, ts, s);
  return half_integral_tau(tx, ty, s, e0);
}

// 1/2 I over a hit's whole clipped interval.
__device__ __forceinline__ float hit_half_integral(const PrimHit& h) {
  return seg_half_integral(h.a, h.b, h.a, h.b, h.a_end, h.b_end, h.tn, h.ts, h.s, h.e0, h.th);
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

// Byte c of w as a float: the byte goes into the low mantissa of 2^23 (exact), which is then
// subtracted.
__device__ __forceinline__ float byte_f(uint32_t w, int c) {
  const uint32_t sel = uint32_t(c) | 0x7440u;  // bytes: (w.c, 0, 0, 0x4B) from {0x4B000000 : w}
  return __uint_as_float(__byte_perm(w, 0x4B000000u, sel)) - 8388608.f;
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Slab test of the four children of a 4-wide quantised node (layout in ugp_internal.cuh)
// against [tmin, tmax]: returns the mask of children hit and writes their references and entry
// distances. Child c's face along axis a is o_a + q 2^e_a, so its ray distance is
// q (2^e_a inv_a) + (o_a - ray.o_a) inv_a: two products per axis and node, one fma per face.
// The ray's direction signs pick, once per node, which face of each axis is met first, so a
// child's entry and exit are a three-way max and min (the same values as the min/max pairs).
__device__ __forceinline__ unsigned node4_test(const uint4* __restrict__ n4, int node, const Ray& r, float tmin,
                                               float tmax, float en[4], int ch[4]) {
  const uint4* nd = n4 + 4 * size_t(node);
  const uint4 w0 = __ldg(nd), w1 = __ldg(nd + 1), w2 = __ldg(nd + 2), w3 = __ldg(nd + 3);
  // 2^e from the stored byte e + 128: the float exponent field is e + 127
  const float sx = __uint_as_float(((w0.w & 255u) - 1u) << 23);
  const float sy = __uint_as_float((((w0.w >> 8) & 255u) - 1u) << 23);
  const float sz = __uint_as_float((((w0.w >> 16) & 255u) - 1u) << 23);
  const float ax = sx * r.inv.x, bx = (__uint_as_float(w0.x) - r.o.x) * r.inv.x;
  const float ay = sy * r.inv.y, by = (__uint_as_float(w0.y) - r.o.y) * r.inv.y;
  const float az = sz * r.inv.z, bz = (__uint_as_float(w0.z) - r.o.z) * r.inv.z;
  const bool px = r.inv.x >= 0.f, py = r.inv.y >= 0.f, pz = r.inv.z >= 0.f;
  const uint32_t nx = px ? w1.x : w1.w, fx = px ? w1.w : w1.x;  // near and far faces
  const uint32_t ny = py ? w1.y : w2.x, fy = py ? w2.x : w1.y;
  const uint32_t nz = pz ? w1.z : w2.y, fz = pz ? w2.y : w1.z;
  ch[0] = int(w3.x);
  ch[1] = int(w3.y);
  ch[2] = int(w3.z);
  ch[3] = int(w3.w);
  unsigned hit = 0u;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float tl = fmaxf(max3f(fmaf(byte_f(nx, c), ax, bx), fmaf(byte_f(ny, c), ay, by), fmaf(byte_f(nz, c), az, bz)),
                           tmin);
    const float th = fminf(min3f(fmaf(byte_f(fx, c), ax, bx), fmaf(byte_f(fy, c), ay, by), fmaf(byte_f(fz, c), az, bz)),
                           tmax);
    en[c] = tl;
    if (tl <= th + 4e-7f * fabsf(th)) hit |= 1u << c;  // never for an empty slot (inverted box)
  }
  return hit;
}

// Orders (t, ref) pairs of the children hit by entry distance (misses last), a sorting network
// on four entries.
__device__ __forceinline__ void sort4(float t[4], int r[4]) {
  auto cs = [&](int i, int j) {
    if (t[j] < t[i]) {
      const float tt = t[i]; t[i] = t[j]; t[j] = tt;
      const int rr = r[i]; r[i] = r[j]; r[j] = rr;
    }
  };
  cs(0, 1); cs(2, 3); cs(0, 2); cs(1, 3); cs(1, 2);
}

__device__ __forceinline__ float3 ld3(const float* __restrict__ p, int64_t i) {
  return make_float3(__ldg(p + 3 * i), __ldg(p + 3 * i + 1), __ldg(p + 3 * i + 2));
}

// Warp-aggregated statistics update (threads of a warp that already returned are left out):
// nodes loaded, primitive records loaded, rays, traversal passes, rays handed to the dense pass.
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
