// C entry points of the FP64 oracle (loaded by the tests through ctypes).
//
// TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
// CPU-baseline leg call these; the CUDA library never does.
#include <algorithm>
#include <cstring>

#include "oracle_internal.h"
#include "oracle_phase.h"

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
  const float* disney9;  // n x 9 Disney parameters of type-3 primitives, or NULL
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
                            double* F_end_out, int32_t* n_active_out, double* race_margin_out) {
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
    if (race_margin_out) race_margin_out[r] = f.race_margin;
  }
}

// Batched radiance-field render (Sec. 7, Eq. rf) by brute force.
void orc_radiance_field(const orc_scene* s, double cutoff_eps, int64_t nr, const float* o3, const float* d3,
                        const float* t0, const float* t1, const float* emission3, const double* background3,
                        double t_shift_ulps, double* rgb_out, double* t_sat_out, double* F_end_out) {
  const std::vector<Prim> prims = make_prims(scene_in(s));
  const double k = cutoff_k(cutoff_eps);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nr; ++r)
    radiance_field(prims, load3(o3 + 3 * r), load3(d3 + 3 * r), t0[r], t1[r], k, emission3, background3,
                   t_shift_ulps, rgb_out + 3 * r, t_sat_out ? t_sat_out + r : nullptr,
                   F_end_out ? F_end_out + r : nullptr);
}

// Batched analog decomposition tracking of the exponential variant, one uniform u per ray
// (the key of the per-primitive variates).
void orc_sample_free_flight_exponential(const orc_scene* s, double cutoff_eps, int64_t nr, const float* o3,
                                        const float* d3, const float* t0, const float* t1,
                                        const int32_t* exclude, const float* u, int32_t* prim_out,
                                        double* t_out, double* t_second_out, double* margin_out, double* amp_out,
                                        double* G_out, double* depth_out) {
  const std::vector<Prim> prims = make_prims(scene_in(s));
  const double k = cutoff_k(cutoff_eps);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nr; ++r) {
    const ExpFreeFlight f = sample_free_flight_exponential(prims, load3(o3 + 3 * r), load3(d3 + 3 * r), t0[r],
                                                           t1[r], k, exclude ? exclude[r] : -1, u[r]);
    prim_out[r] = f.prim;
    t_out[r] = f.t;
    t_second_out[r] = f.t_second;
    margin_out[r] = f.margin;
    amp_out[r] = f.amp;
    G_out[r] = f.G_t;
    depth_out[r] = f.depth;
  }
}

// Batched exponential transmittance exp(-sum_k I_k).
void orc_transmittance_exponential(const orc_scene* s, double cutoff_eps, int64_t nr, const float* o3,
                                   const float* d3, const float* t0, const float* t1, const int32_t* exclude,
                                   double* T_out, double* depth_out) {
  const std::vector<Prim> prims = make_prims(scene_in(s));
  const double k = cutoff_k(cutoff_eps);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nr; ++r)
    T_out[r] = transmittance_exponential(prims, load3(o3 + 3 * r), load3(d3 + 3 * r), t0[r], t1[r], k,
                                         exclude ? exclude[r] : -1, depth_out ? depth_out + r : nullptr);
}

// Rays whose hit set is decided at rounding level (the epsilon band of the parity contract):
// some primitive with |sqrt(d2) - k| < rel k whose closest approach lies in [t0, t1], or an
// ellipsoid end point within rel (t1 - t0) of t0 or t1. flag_out[r] = 1 for such a ray.
void orc_band_rays(const orc_scene* s, double cutoff_eps, int64_t nr, const float* o3, const float* d3,
                   const float* t0, const float* t1, double rel, int32_t* flag_out) {
  const std::vector<Prim> prims = make_prims(scene_in(s));
  const double k = cutoff_k(cutoff_eps);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nr; ++r) {
    const V3 o = load3(o3 + 3 * r), d = load3(d3 + 3 * r);
    const double a = t0[r], b = t1[r], tol = rel * (b - a);
    int32_t flag = 0;
    for (size_t i = 0; i < prims.size() && !flag; ++i) {
      double A, ts, d2;
      ray_prim_quadratic(prims[i], o, d, &A, &ts, &d2);
      const double dist = std::sqrt(std::max(d2, 0.0));
      if (std::fabs(dist - k) < rel * k && ts >= a && ts <= b) flag = 1;
      if (d2 < k * k) {
        const double half = std::sqrt((k * k - d2) / A);
        for (double e : {ts - half, ts + half})
          if (std::fabs(e - a) <= tol || std::fabs(e - b) <= tol) flag = 1;
      }
    }
    flag_out[r] = flag;
  }
}

// Batched free-flight sampling by the paper's own disambiguation rule (a bias diagnostic).
void orc_sample_free_flight_paper_rule(const orc_scene* s, double cutoff_eps, int64_t nr, const float* o3,
                                       const float* d3, const float* t0, const float* t1, const float* u,
                                       const float* u2, int32_t* prim_out) {
  const std::vector<Prim> prims = make_prims(scene_in(s));
  const double k = cutoff_k(cutoff_eps);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nr; ++r)
    prim_out[r] = sample_free_flight_paper_rule(all_hits(prims, load3(o3 + 3 * r), load3(d3 + 3 * r), t0[r], t1[r],
                                                         k, -1),
                                                t0[r], t1[r], u[r], u2[r]);
}

// The paper's own sampler over an SAH kd-tree (built once per call): primitive (-1: escape),
// the start of the ambiguous segment it used (NaN if none), and the nodes and primitives it visited.
// The paper's sampler over a kd-tree given as arrays (interior node: axis, plane as float bits,
// left, right; leaf: 3, count, first reference, 0; references are primitive indices), with the
// root box, and the ambiguous leaf partitioned into nbins equal bins (0: exact segments).
void orc_kd_sample_tree(const orc_scene* s, double cutoff_eps, const int32_t* nodes4, int64_t n_nodes,
                        const int32_t* refs, int64_t n_refs, const float* box6, int32_t nbins, int64_t nr,
                        const float* o3, const float* d3, const float* t0, const float* t1, const float* u,
                        const float* u2, int32_t* prim_out, double* ambiguous_start_out) {
  const std::vector<Prim> prims = make_prims(scene_in(s));
  const double k = cutoff_k(cutoff_eps);
  KdTree T;
  T.nodes.resize(size_t(n_nodes));
  for (int64_t i = 0; i < n_nodes; ++i) {
    const int32_t* q = nodes4 + 4 * i;
    KdNode& nd = T.nodes[size_t(i)];
    if (q[0] == 3) {
      nd.axis = -1;
      nd.count = q[1];
      nd.first = q[2];
    } else {
      float pos;
      std::memcpy(&pos, &q[1], 4);
      nd.axis = q[0];
      nd.pos = pos;
      nd.child[0] = q[2];
      nd.child[1] = q[3];
    }
  }
  T.leaf_ids.assign(refs, refs + n_refs);
  for (int a = 0; a < 3; ++a) {
    T.lo[a] = box6[a];
    T.hi[a] = box6[3 + a];
  }
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nr; ++r) {
    KdStats st;
    prim_out[r] = kd_sample_free_flight(T, prims, load3(o3 + 3 * r), load3(d3 + 3 * r), t0[r], t1[r], k, u[r], u2[r],
                                        &st, nbins);
    ambiguous_start_out[r] = st.ambiguous_start;
  }
}

void orc_kd_sample_free_flight(const orc_scene* s, double cutoff_eps, int64_t nr, const float* o3, const float* d3,
                               const float* t0, const float* t1, const float* u, const float* u2, int32_t* prim_out,
                               double* ambiguous_start_out, int64_t* nodes_out, int64_t* prims_out) {
  const std::vector<Prim> prims = make_prims(scene_in(s));
  const double k = cutoff_k(cutoff_eps);
  const KdTree T = kd_build(prims, k);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nr; ++r) {
    KdStats st;
    prim_out[r] = kd_sample_free_flight(T, prims, load3(o3 + 3 * r), load3(d3 + 3 * r), t0[r], t1[r], k, u[r], u2[r],
                                        &st);
    ambiguous_start_out[r] = st.ambiguous_start;
    nodes_out[r] = st.nodes_visited;
    prims_out[r] = st.prims_tested;
  }
}

double orc_decomposition_exponential(double u, int32_t k) { return decomposition_exponential(u, k); }

// App. A quantities of primitive i along a ray (no clipping): A, t* = -B/2A, d2 = C - B^2/4A.
void orc_prim_quadratic(const orc_scene* s, int64_t i, const float* o3, const float* d3, double* out3) {
  const Prim p = make_prim(s->mean3 + 3 * i, s->quat4 + 4 * i, s->scale3 + 3 * i, s->magnitude[i]);
  ray_prim_quadratic(p, load3(o3), load3(d3), &out3[0], &out3[1], &out3[2]);
}

double orc_erfinv(double y) { return erfinv(y); }
double orc_race_exponential(double u2, int32_t k) { return race_exponential(u2, k); }

// ------------------------------------------------------------------ appearance (Sec. 6, App. B)
static V3 d3v(const double* p) { return v3(p[0], p[1], p[2]); }
static void put3(double* p, V3 v) { p[0] = v.x; p[1] = v.y; p[2] = v.z; }
static Material mat_of(int type, const double* albedo3, double alpha, const double* S6) {
  Material m;
  m.type = type;
  m.albedo = d3v(albedo3);
  m.alpha = alpha;
  m.emission = v3(0, 0, 0);
  for (int k = 0; k < 6; ++k) m.S[k] = S6[k];
  return m;
}

// sigma(w) and D(n = w) of the SGGX distribution S6 for n directions.
void orc_sggx_eval(const double* S6, int64_t n, const double* w3, double* sigma, double* D) {
  for (int64_t i = 0; i < n; ++i) {
    sigma[i] = sggx_sigma(S6, d3v(w3 + 3 * i));
    D[i] = sggx_D(S6, d3v(w3 + 3 * i));
  }
}
void orc_sggx_dvis(const double* S6, const double* wo, int64_t n, const double* n3, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = sggx_Dvis(S6, d3v(wo), d3v(n3 + 3 * i));
}
void orc_sggx_sample_vndf(const double* S6, const double* wo, int64_t n, const double* U2, double* n3) {
  for (int64_t i = 0; i < n; ++i) put3(n3 + 3 * i, sggx_sample_vndf(S6, d3v(wo), U2[2 * i], U2[2 * i + 1]));
}
void orc_sggx_roughen(const double* S6, double alpha, double* out6) { sggx_roughen(S6, alpha, out6); }

// Cosine-weighted base BSDF f(wi, wo; n) <n.wi> for type 0 (Lambertian) or 1 (GGX).
void orc_base_bsdf(int type, const double* albedo3, double alpha, int64_t n, const double* wi3,
                   const double* wo, const double* nrm, double* out3) {
  for (int64_t i = 0; i < n; ++i) {
    const V3 wi = d3v(wi3 + 3 * i);
    const V3 f = type == kMatGGX ? ggx_f(d3v(albedo3), alpha, wi, d3v(wo), d3v(nrm))
                                 : lambert_f(d3v(albedo3), wi, d3v(wo), d3v(nrm));
    put3(out3 + 3 * i, f);
  }
}
// GGX visible-normal samples h (n3 out) and micro-normal samples around a half vector.
void orc_ggx_sample_vn(double alpha, const double* wo, const double* nrm, int64_t n, const double* U2,
                       double* h3) {
  for (int64_t i = 0; i < n; ++i) put3(h3 + 3 * i, ggx_sample_vn(alpha, d3v(wo), d3v(nrm), U2[2 * i], U2[2 * i + 1]));
}
void orc_micro_sample(double alpha, const double* h, int64_t n, const double* U2, double* n3) {
  for (int64_t i = 0; i < n; ++i) put3(n3 + 3 * i, micro_sample(alpha, d3v(h), U2[2 * i], U2[2 * i + 1]));
}

// Phase function values for n incident directions.  mode 0: as used by the renderer (closed form
// for isotropic flakes with a Lambertian base, else stochastic), 1: stochastic estimator,
// 2: Lambert-sphere closed form.  U6 holds six uniforms per direction.
void orc_phase_eval(int type, const double* albedo3, double alpha, const double* S6, const double* wo,
                    int64_t n, const double* wi3, const double* U6, int mode, double* out3) {
  const Material m = mat_of(type, albedo3, alpha, S6);
  for (int64_t i = 0; i < n; ++i) {
    const V3 wi = d3v(wi3 + 3 * i);
    V3 f;
    if (mode == 1) f = phase_eval_stochastic(m, wi, d3v(wo), U6 + 6 * i);
    else if (mode == 2) f = phase_eval_lambert_sphere(m.albedo, wi, d3v(wo));
    else f = phase_eval(m, wi, d3v(wo), U6 + 6 * i);
    put3(out3 + 3 * i, f);
  }
}

void orc_phase_sample(int type, const double* albedo3, double alpha, const double* S6, const double* wo,
                      int64_t n, const double* U4, double* wi3, double* weight3, int32_t* ok) {
  const Material m = mat_of(type, albedo3, alpha, S6);
  for (int64_t i = 0; i < n; ++i) {
    V3 wi = v3(0, 0, 0), w = v3(0, 0, 0);
    ok[i] = phase_sample(m, d3v(wo), U4 + 4 * i, &wi, &w) ? 1 : 0;
    put3(wi3 + 3 * i, wi);
    put3(weight3 + 3 * i, w);
  }
}

void orc_phase_pdf_approx(int type, const double* albedo3, double alpha, const double* S6, const double* wo,
                          int64_t n, const double* wi3, double* out) {
  const Material m = mat_of(type, albedo3, alpha, S6);
  for (int64_t i = 0; i < n; ++i) out[i] = phase_pdf_approx(m, d3v(wi3 + 3 * i), d3v(wo));
}

// ------------------------------------------------------------------ Disney base BSDF
static Material disney_mat(const double* C3, const double* dis9, const double* S6) {
  Material m = mat_of(kMatDisney, C3, 0.0, S6);
  for (int k = 0; k < 9; ++k) m.dis[k] = dis9[k];
  return m;
}
static const double kIdentityS6[6] = {1, 1, 1, 0, 0, 0};

// Cosine-weighted base BSDF f <n.wi> at n directions wi3 (normal nrm, outgoing wo).
void orc_disney_f(const double* C3, const double* dis9, int64_t n, const double* wi3, const double* wo,
                  const double* nrm, double* out3) {
  const Material m = disney_mat(C3, dis9, kIdentityS6);
  for (int64_t i = 0; i < n; ++i) put3(out3 + 3 * i, disney_f(m, d3v(wi3 + 3 * i), d3v(wo), d3v(nrm)));
}
void orc_disney_pdf(const double* C3, const double* dis9, const double* wo, const double* nrm, int64_t n,
                    const double* wi3, double* out) {
  const Material m = disney_mat(C3, dis9, kIdentityS6);
  for (int64_t i = 0; i < n; ++i) out[i] = disney_pdf(m, d3v(wi3 + 3 * i), d3v(wo), d3v(nrm));
}
void orc_disney_sample(const double* C3, const double* dis9, const double* wo, const double* nrm, int64_t n,
                       const double* U2, double* wi3, double* weight3, int32_t* ok) {
  const Material m = disney_mat(C3, dis9, kIdentityS6);
  for (int64_t i = 0; i < n; ++i) {
    V3 wi = v3(0, 0, 0), w = v3(0, 0, 0);
    ok[i] = disney_sample(m, d3v(wo), d3v(nrm), U2 + 2 * i, &wi, &w) ? 1 : 0;
    put3(wi3 + 3 * i, wi);
    put3(weight3 + 3 * i, w);
  }
}
// The diffuse, subsurface and sheen part alone (times <n.wi>), so that tests can pin it apart from
// the glossy lobes.
void orc_disney_f_diffuse(const double* C3, const double* dis9, int64_t n, const double* wi3, const double* wo,
                          const double* nrm, double* out3) {
  const Material m = disney_mat(C3, dis9, kIdentityS6);
  for (int64_t i = 0; i < n; ++i) put3(out3 + 3 * i, disney_f_diffuse(m, d3v(wi3 + 3 * i), d3v(wo), d3v(nrm)));
}
double orc_gtr1_D(double a, double c) { return gtr1_D(a, c); }

// The phase function of Eq. 12 with a Disney base: stochastic evaluation, sampling, App. B pdf.
void orc_phase_eval_disney(const double* C3, const double* dis9, const double* S6, const double* wo, int64_t n,
                           const double* wi3, const double* U6, double* out3) {
  const Material m = disney_mat(C3, dis9, S6);
  for (int64_t i = 0; i < n; ++i) put3(out3 + 3 * i, phase_eval(m, d3v(wi3 + 3 * i), d3v(wo), U6 + 6 * i));
}
void orc_phase_sample_disney(const double* C3, const double* dis9, const double* S6, const double* wo, int64_t n,
                             const double* U4, double* wi3, double* weight3, int32_t* ok) {
  const Material m = disney_mat(C3, dis9, S6);
  for (int64_t i = 0; i < n; ++i) {
    V3 wi = v3(0, 0, 0), w = v3(0, 0, 0);
    ok[i] = phase_sample(m, d3v(wo), U4 + 4 * i, &wi, &w) ? 1 : 0;
    put3(wi3 + 3 * i, wi);
    put3(weight3 + 3 * i, w);
  }
}
void orc_phase_pdf_approx_disney(const double* C3, const double* dis9, const double* S6, const double* wo,
                                 int64_t n, const double* wi3, double* out) {
  const Material m = disney_mat(C3, dis9, S6);
  for (int64_t i = 0; i < n; ++i) out[i] = phase_pdf_approx(m, d3v(wi3 + 3 * i), d3v(wo));
}

// ------------------------------------------------------------------ path tracer (Table 1)
typedef struct {
  float eye[3], look[3], up[3];
  float vfov_deg;
  int32_t width, height;
} orc_camera;
typedef struct {
  int32_t has_quad;
  float corner[3], e1[3], e2[3], Le[3], bg[3];
} orc_lights;
typedef struct {
  double pos_lo[3], pos_hi[3];
  double kappa_min, kappa_max;
  int32_t round_bf16;
} orc_guide_cfg;
typedef struct {
  int32_t spp, spp_begin, max_depth;
  uint64_t seed;
  double cutoff_eps;
  int32_t nee, spawn_mode;
  const float* guide;  // flat guide parameters (NULL: plain phase sampling)
  orc_guide_cfg guide_cfg;
  double guide_alpha;
  int32_t nee_emitters;  // 1: next-event estimation toward emissive primitives as well
  int32_t accel;         // 1: intervals found with a BVH (the same ones; for timing large scenes)
  double guide_min_roughness;  // glossier vertices scatter by phase sampling alone
  int32_t crop_x0, crop_x1;    // columns [crop_x0, crop_x1) of the range only (x1 <= x0: all)
} orc_params;

static GuideCfg guide_cfg_of(const orc_guide_cfg* g) {
  GuideCfg c;
  for (int a = 0; a < 3; ++a) {
    c.pos_lo[a] = g->pos_lo[a];
    c.pos_hi[a] = g->pos_hi[a];
  }
  c.kappa_min = g->kappa_min;
  c.kappa_max = g->kappa_max;
  c.round_bf16 = g->round_bf16;
  return c;
}

// Adds the per-pixel sums of sample values and of their squares (3 channels) for pixels
// [p_begin, p_end) (within columns [crop_x0, crop_x1) when those are set) into accum /
// accum_sq (full-image arrays).  counts[0] += extend queries,
// counts[1] += shadow queries.
void orc_render(const orc_scene* s, const orc_camera* c, const orc_lights* l, const orc_params* p,
                int64_t p_begin, int64_t p_end, double* accum, double* accum_sq, int64_t* counts) {
  Camera cam{load3(c->eye), load3(c->look), load3(c->up), c->vfov_deg, c->width, c->height};
  Lights L{l->has_quad != 0, load3(l->corner), load3(l->e1), load3(l->e2), load3(l->Le), load3(l->bg)};
  RenderParams P{p->spp, p->spp_begin, p->max_depth, p->seed, p->cutoff_eps, p->nee, p->spawn_mode};
  P.guide = p->guide;
  P.guide_cfg = guide_cfg_of(&p->guide_cfg);
  P.guide_alpha = p->guide_alpha;
  P.nee_emitters = p->nee_emitters;
  P.accel = p->accel;
  P.guide_min_roughness = p->guide_min_roughness;
  P.crop_x0 = p->crop_x0;
  P.crop_x1 = p->crop_x1;
  int64_t ne = 0, ns = 0;
  render_pixels(scene_in(s), cam, L, P, p_begin, p_end, accum, accum_sq, &ne, &ns);
  if (counts) {
    counts[0] += ne;
    counts[1] += ns;
  }
}

// Points of primitive i from its Gaussian restricted to the k-ellipsoid (three uniforms each).
void orc_sample_in_ellipsoid(const orc_scene* s, int64_t i, double cutoff_eps, int64_t n, const double* U3,
                             double* y3) {
  const Prim p = make_prim(s->mean3 + 3 * i, s->quat4 + 4 * i, s->scale3 + 3 * i, s->magnitude[i]);
  const double k = cutoff_k(cutoff_eps);
  for (int64_t r = 0; r < n; ++r) put3(y3 + 3 * r, sample_in_ellipsoid(p, k, U3 + 3 * r));
}

// Sum and sum of squares of n light estimates toward the scene's emitters (no MIS weight) at the
// vertex x3 with outgoing direction wo3 and the given material.
void orc_emitter_nee(const orc_scene* s, double cutoff_eps, const double* x3, const double* wo3, int32_t exclude,
                     int32_t mtype, const double* albedo3, double alpha, const double* S6, int64_t n, uint64_t seed,
                     double* sum3, double* sq3) {
  emitter_nee_sums(scene_in(s), cutoff_eps, mat_of(mtype, albedo3, alpha, S6), d3v(x3), d3v(wo3), exclude, n, seed,
                   sum3, sq3);
}

double orc_chi3_cdf(double r) { return chi3_cdf(r); }

// ------------------------------------------------------------------ learned guide
int64_t orc_guide_nparams() { return kGNParams; }

void orc_bf16_round(int64_t n, const double* x, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = bf16_round(x[i]);
}

void orc_guide_encode(const orc_guide_cfg* g, int64_t n, const float* x3, const float* wo3, double* out) {
  const GuideCfg c = guide_cfg_of(g);
  for (int64_t i = 0; i < n; ++i) guide_encode(c, load3(x3 + 3 * i), load3(wo3 + 3 * i), out + kGWidth * i);
}

// Head outputs (n x 40) and the mixture (n x 40: per lobe mu (3), kappa, pi); either may be NULL.
void orc_guide_forward(const orc_guide_cfg* g, const float* params, int64_t n, const float* x3, const float* wo3,
                       double* Y_out, double* mix_out) {
  const GuideCfg c = guide_cfg_of(g);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double Y[kGOut];
    guide_forward(c, params, load3(x3 + 3 * i), load3(wo3 + 3 * i), Y, nullptr);
    if (Y_out) std::memcpy(Y_out + kGOut * i, Y, sizeof(Y));
    if (mix_out) {
      const Mixture m = guide_mixture(c, Y);
      for (int j = 0; j < kGLobes; ++j) {
        double* o = mix_out + kGOut * i + 5 * j;
        o[0] = m.mu[j].x; o[1] = m.mu[j].y; o[2] = m.mu[j].z; o[3] = m.kappa[j]; o[4] = m.pi[j];
      }
    }
  }
}

static Mixture mixture_of(const double* mx) {
  Mixture m;
  for (int j = 0; j < kGLobes; ++j) {
    m.mu[j] = v3(mx[5 * j], mx[5 * j + 1], mx[5 * j + 2]);
    m.kappa[j] = mx[5 * j + 3];
    m.pi[j] = mx[5 * j + 4];
  }
  return m;
}

void orc_mixture_pdf(int64_t n, const double* mix, const double* wi3, double* pdf_out) {
  for (int64_t i = 0; i < n; ++i) pdf_out[i] = mixture_pdf(mixture_of(mix + kGOut * i), d3v(wi3 + 3 * i));
}

// Directions from uniforms U3 = (lobe choice, u1, u2) per row, and their mixture pdf.
void orc_mixture_sample(int64_t n, const double* mix, const double* U3, double* wi_out, double* pdf_out) {
  for (int64_t i = 0; i < n; ++i) {
    const Mixture m = mixture_of(mix + kGOut * i);
    const V3 w = mixture_sample(m, U3 + 3 * i);
    put3(wi_out + 3 * i, w);
    if (pdf_out) pdf_out[i] = mixture_pdf(m, w);
  }
}

double orc_mixture_loss_grad(const orc_guide_cfg* g, const double* Y, const double* wi, double w, double* dY) {
  return mixture_loss_grad(guide_cfg_of(g), Y, d3v(wi), w, dY);
}

double orc_guide_loss_grad(const orc_guide_cfg* g, const float* params, int64_t n, const float* x3, const float* wo3,
                           const float* wi3, const float* weight, double* grad) {
  return guide_loss_grad(guide_cfg_of(g), params, n, x3, wo3, wi3, weight, grad);
}

void orc_adam_step(int64_t n, double* theta, double* m, double* v, const double* g, int64_t t, double lr, double b1,
                   double b2, double eps) {
  adam_step(n, theta, m, v, g, t, lr, b1, b2, eps);
}

}  // extern "C"
