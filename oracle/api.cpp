// C entry points of the FP64 oracle (loaded by the tests through ctypes).
//
// TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
// CPU-baseline leg call these; the CUDA library never does.
#include <algorithm>
#include <cstring>

#include "oracle_internal.h"

#ifdef _OPENMP
#include <omp.h>
#endif

using namespace orc;

extern "C" {

typedef struct {
  int64_t n;
  const float* mean3;
  const float* quat4;
  const float* scale3;
  const float* magnitude;
  const float* sggx6;
  const uint8_t* type;
  const float* albedo3;
  const float* roughness;
  const float* emission3;
} orc_scene;

static SceneIn scene_in(const orc_scene* s) {
  SceneIn r;
  std::memcpy(&r, s, sizeof(r));
  return r;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

void orc_philox4x32_10(const uint32_t* ctr4, const uint32_t* key2, uint32_t* out4) {
  philox4x32_10(ctr4, key2, out4);
}

// Per-primitive whitening matrix (row-major, 9), normaliser g0 and bounding-ellipsoid AABB
// (lo xyz, hi xyz) with the half extent k * sqrt(sum_j (R_ij s_j)^2).
void orc_prim_setup(const orc_scene* s, double cutoff_eps, double* W9, double* g0, double* aabb6) {
  const double k = cutoff_k(cutoff_eps);
  for (int64_t i = 0; i < s->n; ++i) {
    const Prim p = make_prim(s->mean3 + 3 * i, s->quat4 + 4 * i, s->scale3 + 3 * i, s->magnitude[i]);
    for (int j = 0; j < 9; ++j) W9[9 * i + j] = p.W[j];
    g0[i] = p.g0;
    const double m[3] = {p.mu.x, p.mu.y, p.mu.z};
    for (int r = 0; r < 3; ++r) {
      double e2 = 0;
      for (int c = 0; c < 3; ++c) e2 += (p.R[3 * r + c] * p.s[c]) * (p.R[3 * r + c] * p.s[c]);
      const double e = k * std::sqrt(e2);
      aabb6[6 * i + r] = m[r] - e;
      aabb6[6 * i + 3 + r] = m[r] + e;
    }
  }
}

// Ray integral of primitive i over [ta, tb] without the ellipsoid cut-off (App. A).
double orc_prim_integral(const orc_scene* s, int64_t i, const float* o3, const float* d3, double ta,
                         double tb) {
  const Prim p = make_prim(s->mean3 + 3 * i, s->quat4 + 4 * i, s->scale3 + 3 * i, s->magnitude[i]);
  Hit h;
  h.id = int32_t(i);
  h.g0 = p.g0;
  ray_prim_quadratic(p, load3(o3), load3(d3), &h.A, &h.tstar, &h.d2);
  h.a = ta;
  h.b = tb;
  return ray_integral(h, ta, tb);
}

// Hits of one ray (ascending id): writes up to cap entries, returns the total count.
int64_t orc_hits(const orc_scene* s, double cutoff_eps, const float* o3, const float* d3, float t0,
                 float t1, int32_t exclude, int32_t* ids, double* a, double* b, double* d2,
                 double* half_I, int64_t cap) {
  const std::vector<Prim> prims = make_prims(scene_in(s));
  const std::vector<Hit> hits =
      all_hits(prims, load3(o3), load3(d3), t0, t1, cutoff_k(cutoff_eps), exclude);
  for (size_t i = 0; i < hits.size() && int64_t(i) < cap; ++i) {
    ids[i] = hits[i].id;
    a[i] = hits[i].a;
    b[i] = hits[i].b;
    d2[i] = hits[i].d2;
    half_I[i] = 0.5 * ray_integral(hits[i], hits[i].a, hits[i].b);
  }
  return int64_t(hits.size());
}

// Batched transmittance (Eq. 7) by brute force.
void orc_transmittance(const orc_scene* s, double cutoff_eps, int64_t nr, const float* o3,
                       const float* d3, const float* t0, const float* t1, const int32_t* exclude,
                       double* T_out, double* tau_out, int32_t* nhit_out) {
  const std::vector<Prim> prims = make_prims(scene_in(s));
  const double k = cutoff_k(cutoff_eps);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nr; ++r) {
    const int32_t ex = exclude ? exclude[r] : -1;
    const V3 o = load3(o3 + 3 * r), d = load3(d3 + 3 * r);
    double tau = 0;
    T_out[r] = transmittance(prims, o, d, t0[r], t1[r], k, ex, &tau);
    if (tau_out) tau_out[r] = tau;
    if (nhit_out) nhit_out[r] = int32_t(all_hits(prims, o, d, t0[r], t1[r], k, ex).size());
  }
}

// Batched exact free-flight sampling (Sec. 5.2) with caller-supplied uniforms (u, u2).
void orc_sample_free_flight(const orc_scene* s, double cutoff_eps, int64_t nr, const float* o3,
                            const float* d3, const float* t0, const float* t1,
                            const int32_t* exclude, const float* u, const float* u2,
                            int32_t* prim_out, double* t_u_out, double* t_spawn_out,
                            double* F_end_out, int32_t* n_active_out) {
  const std::vector<Prim> prims = make_prims(scene_in(s));
  const double k = cutoff_k(cutoff_eps);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nr; ++r) {
    const int32_t ex = exclude ? exclude[r] : -1;
    const FreeFlight f = sample_free_flight(prims, load3(o3 + 3 * r), load3(d3 + 3 * r), t0[r],
                                            t1[r], k, ex, u[r], u2[r]);
    prim_out[r] = f.prim;
    t_u_out[r] = f.t_u;
    t_spawn_out[r] = f.t_spawn;
    if (F_end_out) F_end_out[r] = f.F_end;
    if (n_active_out) n_active_out[r] = f.n_active;
  }
}

// App. A quantities of primitive i along a ray (no clipping): A, t* = -B/2A, d2 = C - B^2/4A.
void orc_prim_quadratic(const orc_scene* s, int64_t i, const float* o3, const float* d3, double* out3) {
  const Prim p = make_prim(s->mean3 + 3 * i, s->quat4 + 4 * i, s->scale3 + 3 * i, s->magnitude[i]);
  ray_prim_quadratic(p, load3(o3), load3(d3), &out3[0], &out3[1], &out3[2]);
}

double orc_erfinv(double y) { return erfinv(y); }

}  // extern "C"
