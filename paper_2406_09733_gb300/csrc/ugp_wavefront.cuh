// Device records and helpers of the wavefront path tracer, shared by the single-image renderer
// (ugp_render.cu) and the batched server (ugp_batch.cu).
#pragma once
#include <cooperative_groups.h>

#include <math.h>

#include "ugp_phase.cuh"
#include "ugp_philox.cuh"
#include "ugp_trace.cuh"

namespace ugp {

// Path state, one column per field (structure of arrays, indexed by path slot).
struct PathSoA {
  float *ox, *oy, *oz, *dx, *dy, *dz;
  float *br, *bg, *bb;   // throughput beta
  float *lr, *lg, *lb;   // radiance so far
  float* pdf_prev;       // approximate phase pdf of the last scattering (< 0: none)
  int* excl;             // primitive the current ray skips
  int* prim;             // free-flight result
  float* tsp;            // spawn distance along the current ray
  float* tq;             // distance to the area light along the current ray
  int* qflag;            // 0 no light hit, 1 front face, 2 back face
  float *fu, *fu2;       // free-flight uniforms of the current ray (u, u2)
};

struct ShadowSoA {
  int* path;
  float *ox, *oy, *oz, *dx, *dy, *dz, *dist;
  int* excl;
  float *cr, *cg, *cb;   // contribution if unoccluded
};

struct LightsDev {
  int has_quad;
  float3 corner, e1, e2, Le, bg, nrm;  // nrm = unit e1 x e2
  float area;
};

struct CameraDev {
  float3 eye, fwd, right, up;
  float th, aspect;
  int width, height;
};

struct MatDev {
  const float* sggx6;
  const uint8_t* type;
  const float* albedo3;
  const float* roughness;
  const float* emission3;
  const float* disney9;  // may be null (published defaults for type 3)
};

namespace wf {
namespace cg = cooperative_groups;

__device__ __forceinline__ float4 rng(uint2 key, int pixel, int sample, int bounce, int slot) {
  const uint4 x = philox4x32_10(make_uint4(uint32_t(pixel), uint32_t(sample), uint32_t(16 * bounce + slot), 0u), key);
  return make_float4(u24(x.x), u24(x.y), u24(x.z), u24(x.w));
}

__device__ __forceinline__ int load_count(const int* c) { return *reinterpret_cast<const volatile int*>(c); }

// Ray / parallelogram intersection with t in (0, tmax).
__device__ __forceinline__ int quad_hit(const LightsDev& L, float3 o, float3 d, float& t) {
  if (!L.has_quad) return 0;
  const float den = dot3(d, L.nrm);
  if (fabsf(den) < 1e-30f) return 0;
  const float tt = dot3(L.corner - o, L.nrm) / den;
  if (!(tt > 0.f && tt < 1e30f)) return 0;
  const float3 q = o + tt * d - L.corner;
  const float e11 = dot3(L.e1, L.e1), e22 = dot3(L.e2, L.e2), e12 = dot3(L.e1, L.e2);
  const float q1 = dot3(q, L.e1), q2 = dot3(q, L.e2);
  const float det = e11 * e22 - e12 * e12;
  const float al = (q1 * e22 - q2 * e12) / det, be = (q2 * e11 - q1 * e12) / det;
  if (al < 0.f || al > 1.f || be < 0.f || be > 1.f) return 0;
  t = tt;
  return den < 0.f ? 1 : 2;
}

// Appends the calling thread to a queue; the threads of a warp that take the same call share
// one atomic.
__device__ __forceinline__ int queue_append(int* counter) {
  cg::coalesced_group g = cg::coalesced_threads();
  int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(counter, int(g.size()));
  base = g.shfl(base, 0);
  return base + int(g.thread_rank());
}

}  // namespace wf
using wf::rng;
using wf::load_count;
using wf::quad_hit;
using wf::queue_append;

__device__ __forceinline__ Material load_material(const MatDev& m, int k) {
  Material M;
  M.type = m.type[k];
  M.albedo = f3(m.albedo3[3 * k], m.albedo3[3 * k + 1], m.albedo3[3 * k + 2]);
  M.alpha = m.roughness[k];
  for (int j = 0; j < 6; ++j) M.S[j] = m.sggx6[6 * k + j];
  if (M.type == kMatDisney) {
    if (m.disney9) {
      for (int j = 0; j < 9; ++j) M.dis[j] = m.disney9[9 * size_t(k) + j];
    } else {
      const float def[9] = {0.f, 0.f, 0.5f, 0.f, 0.5f, 0.f, 0.5f, 0.f, 1.f};
      for (int j = 0; j < 9; ++j) M.dis[j] = def[j];
    }
  }
  return M;
}

inline float3 h3(const float* v) { return make_float3(v[0], v[1], v[2]); }

// Device form of the lights (one-sided parallelogram with its unit normal and area).
inline LightsDev lights_dev(const ugp_lights* lights) {
  LightsDev Ld;
  Ld.has_quad = lights->has_quad != 0;
  Ld.corner = h3(lights->quad_corner);
  Ld.e1 = h3(lights->quad_e1);
  Ld.e2 = h3(lights->quad_e2);
  Ld.Le = h3(lights->quad_Le);
  Ld.bg = h3(lights->bg);
  const double e1[3] = {lights->quad_e1[0], lights->quad_e1[1], lights->quad_e1[2]};
  const double e2[3] = {lights->quad_e2[0], lights->quad_e2[1], lights->quad_e2[2]};
  const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  const double a = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  Ld.area = float(a);
  Ld.nrm = a > 0 ? make_float3(float(c[0] / a), float(c[1] / a), float(c[2] / a)) : make_float3(0.f, 0.f, 1.f);
  if (Ld.has_quad && !(a > 0)) Ld.has_quad = 0;
  return Ld;
}

// Device form of the pinhole camera (orthonormal frame, tan of half the vertical field of view).
inline ugp_status camera_dev(const ugp_camera* camera, const char* fn, CameraDev* out) {
  const int W = camera->width, H = camera->height;
  double f[3] = {double(camera->look[0]) - camera->eye[0], double(camera->look[1]) - camera->eye[1],
                 double(camera->look[2]) - camera->eye[2]};
  const double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  if (!(fl > 0)) return fail(UGP_ERR_INVALID_ARG, "%s: eye and look coincide", fn);
  for (double& v : f) v /= fl;
  const double up[3] = {camera->up[0], camera->up[1], camera->up[2]};
  double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
  const double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (!(rl > 0)) return fail(UGP_ERR_INVALID_ARG, "%s: up is parallel to the view direction", fn);
  for (double& v : r) v /= rl;
  const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
  CameraDev cd;
  cd.eye = h3(camera->eye);
  cd.fwd = make_float3(float(f[0]), float(f[1]), float(f[2]));
  cd.right = make_float3(float(r[0]), float(r[1]), float(r[2]));
  cd.up = make_float3(float(u[0]), float(u[1]), float(u[2]));
  cd.th = float(tan(0.5 * double(camera->vfov_deg) * 3.14159265358979323846 / 180.0));
  cd.aspect = float(double(W) / double(H));
  cd.width = W;
  cd.height = H;
  *out = cd;
  return UGP_OK;
}

// Inputs of the next free flight of path slot `slot` (ray o + t d at `bounce`): the light-hit
// distance and face, and the free-flight uniforms (Philox slot 0). Computed where the ray is made
// (camera or shading), so the scan only loads them.
__device__ __forceinline__ void prepare_extend(const PathSoA& ps, int slot, const LightsDev& L, uint2 key, int pixel,
                                               int sample, int bounce, float3 o, float3 d) {
  float tq = 1e30f;
  const int qf = quad_hit(L, o, d, tq);
  const float4 U = rng(key, pixel, sample, bounce, 0);
  ps.tq[slot] = tq;
  ps.qflag[slot] = qf;
  ps.fu[slot] = U.x;
  ps.fu2[slot] = U.y;
}

// Pinhole camera ray through pixel p of the image at the Philox jitter of (sample, bounce 15).
__device__ __forceinline__ float3 camera_dir(const CameraDev& cam, uint2 key, int p, int sample) {
  const int px = p % cam.width, py = p / cam.width;
  const float4 U = rng(key, p, sample, 15, 0);
  const float x = (2.f * (float(px) + U.x) / float(cam.width) - 1.f) * cam.th * cam.aspect;
  const float y = (1.f - 2.f * (float(py) + U.y) / float(cam.height)) * cam.th;
  return normalize3(cam.fwd + x * cam.right + y * cam.up);
}

}  // namespace ugp
