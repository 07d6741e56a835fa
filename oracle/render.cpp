// FP64 oracle: the volumetric path tracer of Table 1 (right column), brute force.
//
// TEST INFRASTRUCTURE ONLY. Each camera path is traced with the exact free-flight sampler and
// exact transmittance of geometry.cpp (all primitives tested, no acceleration structure).
//
// Readings of the paper used here (the CUDA renderer follows the same ones):
//  * max_depth D allows at most D scattering vertices: the loop samples up to D+1 free
//    flights, the last one only to collect emission, and no light sampling happens from a
//    vertex that cannot scatter further, so light sampling and phase sampling cover the same
//    path lengths.
//  * Emissive primitives are pure emitters: choosing one adds beta * L_e and ends the path.
//  * Escape adds the constant background, or the area light's radiance if the ray reaches
//    the front of the light (one-sided, emitting towards e1 x e2).
//  * Scattered and shadow rays start at the centre of the chosen primitive's clipped
//    interval and skip that primitive (Sec. 6, "Importance Sampling").
//  * MIS (Table 1) is the balance heuristic between light sampling and phase sampling,
//    with the approximate phase pdf of App. B.
//  * Random numbers: Philox4x32-10 with key (seed lo, seed hi) and counter
//    (pixel, sample, 16 * bounce + slot, 0); slot 0 free flight, 1 phase sampling, 2 guide
//    (lobe choice, technique choice, two for the vMF lobe), 3 light point, 4-5 stochastic
//    phase evaluation of the light sample, 6-7 stochastic phase evaluation of a guide sample;
//    the camera jitter uses bounce 15, slot 0.
//  * With a guide, one-sample MIS between the guide (probability alpha) and phase sampling
//    (1 - alpha), balance heuristic with the approximate phase pdf p~ of App. B:
//      guide sample:  weight = f(wi) / (alpha q(wi) + (1 - alpha) p~(wi))
//      phase sample:  weight = (f / p)(wi) * p~(wi) / (alpha q(wi) + (1 - alpha) p~(wi))
//    The two weights of the balance heuristic sum to one at every direction, so the estimate
//    stays unbiased for any q and any approximation p~ (Sec. 6). The mixture pdf
//    alpha q + (1 - alpha) p~ replaces p~ in the MIS with light sampling.
//  * Optionally (nee_emitters), next-event estimation toward emissive primitives as well
//    (slot 8: emitter choice and point, slots 9-10: stochastic phase evaluation), balanced
//    against phase sampling; see emitter_nee below.
#include <algorithm>
#include <cmath>

#include "oracle_phase.h"

namespace orc {

static const double kPi = 3.14159265358979323846;

Material material_of(const SceneIn& s, int64_t i) {
  Material m;
  m.type = s.type[i];
  m.albedo = load3(s.albedo3 + 3 * i);
  m.alpha = s.roughness[i];
  m.emission = load3(s.emission3 + 3 * i);
  for (int k = 0; k < 6; ++k) m.S[k] = s.sggx6[6 * i + k];
  if (m.type == kMatDisney) {
    // Burley's published defaults where the scene gives no parameters: metallic 0, subsurface 0,
    // specular 0.5, specular tint 0, roughness 0.5, sheen 0, sheen tint 0.5, clearcoat 0, gloss 1
    static const double kDefault[9] = {0, 0, 0.5, 0, 0.5, 0, 0.5, 0, 1};
    for (int k = 0; k < 9; ++k) m.dis[k] = s.disney9 ? double(s.disney9[9 * i + k]) : kDefault[k];
  }
  return m;
}

static void rng4(uint64_t seed, uint32_t pixel, uint32_t sample, uint32_t bounce, uint32_t slot,
                 double out[4]) {
  const uint32_t ctr[4] = {pixel, sample, 16u * bounce + slot, 0u};
  const uint32_t key[2] = {uint32_t(seed & 0xffffffffu), uint32_t(seed >> 32)};
  uint32_t x[4];
  philox4x32_10(ctr, key, x);
  for (int k = 0; k < 4; ++k) out[k] = u24(x[k]);
}

// Pinhole camera: ray through pixel (px, py) at sub-pixel position (jx, jy).
static void camera_ray(const Camera& c, int px, int py, double jx, double jy, V3* o, V3* d) {
  const V3 f = normalize(c.look - c.eye);
  const V3 r = normalize(cross(f, c.up));
  const V3 up = cross(r, f);
  const double th = std::tan(0.5 * c.vfov_deg * kPi / 180.0);
  const double aspect = double(c.width) / double(c.height);
  const double x = (2.0 * (px + jx) / c.width - 1.0) * th * aspect;
  const double y = (1.0 - 2.0 * (py + jy) / c.height) * th;
  *o = c.eye;
  *d = normalize(f + x * r + y * up);
}

// Ray / parallelogram (corner, e1, e2) intersection with t in (0, tmax).
static bool quad_hit(const Lights& L, V3 o, V3 d, double tmax, double* t, bool* front) {
  const V3 n = cross(L.e1, L.e2);
  const double den = dot(d, n);
  if (std::fabs(den) < 1e-300) return false;
  const double tt = dot(L.corner - o, n) / den;
  if (!(tt > 0.0 && tt < tmax)) return false;
  const V3 q = o + tt * d - L.corner;
  const double e11 = dot(L.e1, L.e1), e22 = dot(L.e2, L.e2), e12 = dot(L.e1, L.e2);
  const double q1 = dot(q, L.e1), q2 = dot(q, L.e2);
  const double det = e11 * e22 - e12 * e12;
  const double al = (q1 * e22 - q2 * e12) / det, be = (q2 * e11 - q1 * e12) / det;
  if (al < 0 || al > 1 || be < 0 || be > 1) return false;
  *t = tt;
  *front = den < 0;
  return true;
}

static double mis2(double a, double b) { return a + b > 0 ? a / (a + b) : 0.0; }

// ---- next-event estimation toward emissive primitives ------------------------------------
// The free flight from x along w picks primitive j at a distance in [t, t + dt] with
// probability 1/2 G_j(x + t w) dt for t below the saturating distance (Eq. 8 and the exact
// choice of Sec. 5.2). Its direct emission is therefore
//   int f_p(w) P_j(w) L_e,j dw = 1/2 L_e,j int f_p(w(y)) G_j(y) 1[|y - x| < t_sat] / |y - x|^2 dy,
// and with y drawn from G_j / (c_j m) inside the ellipsoid (m its Gaussian mass) and j with
// probability pi_j, one sample estimates it by 1/2 c_j m L_e,j f_p 1[T(x, y) > 0] / (r^2 pi_j):
// the linear model needs only that y lies before saturation, not a transmittance factor.
// The balance heuristic against phase sampling compares the two densities of (j, y) in volume
// measure, pi_j G_j(y) / (c_j m) and p(w) 1/2 G_j(y) / r^2, in which G_j(y) cancels: 2 r^2 pi_j
// against c_j m p(w). The weights use r_c, the distance from x to the emitter's mean, in place of
// r: a weight that depends on (j, x, w) only is available to a path that reaches the emitter by
// phase sampling without knowing where inside it the free flight stopped, and any weights that
// sum to one over the two techniques keep the estimate unbiased.
double chi3_cdf(double r) {
  return std::erf(r / std::sqrt(2.0)) - std::sqrt(2.0 / kPi) * r * std::exp(-0.5 * r * r);
}

EmitterTable emitter_table(const SceneIn& s, double k) {
  EmitterTable E;
  E.mass = chi3_cdf(k);
  for (int64_t i = 0; i < s.n; ++i) {
    if (s.type[i] != kMatEmissive) continue;
    const double w = double(s.magnitude[i]) *
                     (double(s.emission3[3 * i]) + s.emission3[3 * i + 1] + s.emission3[3 * i + 2]) / 3.0;
    if (!(w > 0)) continue;
    E.total += w;
    E.ids.push_back(int32_t(i));
    E.cdf.push_back(E.total);
  }
  return E;
}

V3 sample_in_ellipsoid(const Prim& p, double k, const double U[3]) {
  // radius: invert the chi-3 CDF on [0, k] by bracketed Newton (pdf sqrt(2/pi) r^2 e^{-r^2/2})
  const double target = U[0] * chi3_cdf(k);
  double lo = 0.0, hi = k, r = 0.5 * k;
  for (int it = 0; it < 200; ++it) {
    const double f = chi3_cdf(r) - target;
    if (f == 0.0) break;
    if (f < 0) lo = r; else hi = r;
    const double fp = std::sqrt(2.0 / kPi) * r * r * std::exp(-0.5 * r * r);
    double rn = fp > 0 ? r - f / fp : 0.5 * (lo + hi);
    if (!(rn > lo && rn < hi)) rn = 0.5 * (lo + hi);
    if (std::fabs(rn - r) <= 1e-15 * std::max(1.0, r) || hi - lo <= 1e-15) {
      r = rn;
      break;
    }
    r = rn;
  }
  const double cz = 1.0 - 2.0 * U[1], sz = std::sqrt(std::max(0.0, 1.0 - cz * cz)), ph = 2.0 * kPi * U[2];
  const double z[3] = {r * sz * std::cos(ph) * p.s[0], r * sz * std::sin(ph) * p.s[1], r * cz * p.s[2]};
  return p.mu + v3(p.R[0] * z[0] + p.R[1] * z[1] + p.R[2] * z[2], p.R[3] * z[0] + p.R[4] * z[1] + p.R[5] * z[2],
                   p.R[6] * z[0] + p.R[7] * z[1] + p.R[8] * z[2]);
}

bool emitter_nee(const SceneIn& s, const std::vector<Prim>& prims, const EmitterTable& E, double k,
                 const Material& m, V3 x, V3 wo, int32_t exclude, const double U4[4], const double Uf[6],
                 V3* contrib, V3* dir, double* p_light, double* p_scatter_scale, int64_t* shadow_rays) {
  if (E.ids.empty()) return false;
  size_t q = size_t(std::upper_bound(E.cdf.begin(), E.cdf.end(), U4[0] * E.total) - E.cdf.begin());
  if (q >= E.ids.size()) q = E.ids.size() - 1;
  const int32_t j = E.ids[q];
  const double pj = (E.cdf[q] - (q ? E.cdf[q - 1] : 0.0)) / E.total;
  const V3 y = sample_in_ellipsoid(prims[size_t(j)], k, U4 + 1);
  const V3 w = y - x;
  const double r2 = dot(w, w);
  if (!(r2 > 0)) return false;
  const V3 wl = (1.0 / std::sqrt(r2)) * w;
  const V3 f = phase_eval(m, wl, wo, Uf);
  if (!(f.x > 0 || f.y > 0 || f.z > 0)) return false;
  ++*shadow_rays;
  if (!(transmittance(prims, x, wl, 0.0, std::sqrt(r2), k, exclude, nullptr) > 0)) return false;
  const double cm = double(s.magnitude[j]) * E.mass;
  *contrib = (0.5 * cm / (r2 * pj)) * (f * load3(s.emission3 + 3 * size_t(j)));
  *dir = wl;
  const V3 c = prims[size_t(j)].mu - x;
  *p_light = 2.0 * dot(c, c) * pj;
  *p_scatter_scale = cm;
  return true;
}

// Balance weight of emitter j reached by phase sampling from the vertex x (scattering pdf p
// there): the complement of the light-sampling weight above.
static double emitter_hit_weight(const SceneIn& s, const std::vector<Prim>& prims, const EmitterTable& E, int32_t j,
                                 V3 x, double p) {
  const auto it = std::lower_bound(E.ids.begin(), E.ids.end(), j);
  if (it == E.ids.end() || *it != j) return 1.0;
  const size_t q = size_t(it - E.ids.begin());
  const double pj = (E.cdf[q] - (q ? E.cdf[q - 1] : 0.0)) / E.total;
  const V3 c = prims[size_t(j)].mu - x;
  return mis2(double(s.magnitude[j]) * E.mass * p, 2.0 * dot(c, c) * pj);
}

void emitter_nee_sums(const SceneIn& s, double cutoff_eps, const Material& m, V3 x, V3 wo, int32_t exclude,
                      int64_t n, uint64_t seed, double sum[3], double sq[3]) {
  const std::vector<Prim> prims = make_prims(s);
  const double k = cutoff_k(cutoff_eps);
  const EmitterTable E = emitter_table(s, k);
  double a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
#pragma omp parallel for schedule(static) reduction(+ : a[:3], b[:3])
  for (int64_t i = 0; i < n; ++i) {
    double Ue[4], Uf[6], U10[4];
    rng4(seed, 0u, uint32_t(i), 0u, 8, Ue);
    rng4(seed, 0u, uint32_t(i), 0u, 9, Uf);
    rng4(seed, 0u, uint32_t(i), 0u, 10, U10);
    Uf[4] = U10[0];
    Uf[5] = U10[1];
    V3 c{0, 0, 0}, wl;
    double pl, cm;
    int64_t shd = 0;
    if (!emitter_nee(s, prims, E, k, m, x, wo, exclude, Ue, Uf, &c, &wl, &pl, &cm, &shd)) c = v3(0, 0, 0);
    a[0] += c.x; a[1] += c.y; a[2] += c.z;
    b[0] += c.x * c.x; b[1] += c.y * c.y; b[2] += c.z * c.z;
  }
  for (int c = 0; c < 3; ++c) {
    sum[c] = a[c];
    sq[c] = b[c];
  }
}

void render_pixels(const SceneIn& s, const Camera& cam, const Lights& L, const RenderParams& P,
                   int64_t p_begin, int64_t p_end, double* accum, double* accum_sq, int64_t* n_extend,
                   int64_t* n_shadow) {
  const std::vector<Prim> prims = make_prims(s);
  const double k = cutoff_k(P.cutoff_eps);
  const V3 ln = cross(L.e1, L.e2);
  const double area = length(ln);
  const V3 lnh = area > 0 ? (1.0 / area) * ln : v3(0, 0, 1);
  const EmitterTable E = P.nee_emitters ? emitter_table(s, k) : EmitterTable{};
  // The BVH of the last scene rendered with it is kept (a timing aid: repeated calls over the
  // same arrays, such as a build-only call followed by the timed one, build it once). The key is
  // the arrays' address, size, cut-off and a sample of the means.
  static Accel cached;
  static std::vector<double> cached_key;
  if (P.accel) {
    std::vector<double> key{double(reinterpret_cast<uintptr_t>(s.mean3)), double(s.n), k};
    for (int64_t i = 0; i < s.n; i += std::max<int64_t>(1, s.n / 64)) key.push_back(s.mean3[3 * i]);
    if (key != cached_key || cached.prims == nullptr) {
      cached = accel_build(prims, k);
      cached_key = key;
    }
    cached.prims = &prims;
    g_accel = &cached;
  }
  int64_t ext = 0, shd = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : ext, shd)
  for (int64_t p = p_begin; p < p_end; ++p) {
    const int px = int(p % cam.width), py = int(p / cam.width);
    if (P.crop_x1 > P.crop_x0 && (px < P.crop_x0 || px >= P.crop_x1)) continue;
    double sum[3] = {0, 0, 0}, sq[3] = {0, 0, 0};
    for (int si = 0; si < P.spp; ++si) {
      const uint32_t sample = uint32_t(P.spp_begin + si);
      double U[4];
      rng4(P.seed, uint32_t(p), sample, 15, 0, U);
      V3 o, d;
      camera_ray(cam, px, py, U[0], U[1], &o, &d);
      V3 beta = v3(1, 1, 1), Lr = v3(0, 0, 0);
      double pdf_prev = -1.0;  // < 0: the previous vertex cannot be reached by light sampling
      int32_t excl = -1;
      for (int b = 0; b <= P.max_depth; ++b) {
        double t1 = 1e30, tq = 0;
        bool front = false;
        const bool hq = L.has_quad && quad_hit(L, o, d, 1e30, &tq, &front);
        if (hq) t1 = tq;
        rng4(P.seed, uint32_t(p), sample, uint32_t(b), 0, U);
        const FreeFlight ff = sample_free_flight(prims, o, d, 0.0, t1, k, excl, U[0], U[1]);
        ++ext;
        if (ff.prim < 0) {
          if (hq) {
            if (front) {
              double w = 1.0;
              if (P.nee && pdf_prev >= 0) {
                const double cl = -dot(d, lnh);
                const double pl = tq * tq / (area * cl);
                w = mis2(pdf_prev, pl);
              }
              Lr = Lr + w * (beta * L.Le);
            }
          } else {
            Lr = Lr + beta * L.bg;
          }
          break;
        }
        const Material m = material_of(s, ff.prim);
        if (m.type == kMatEmissive) {
          const double w = (P.nee_emitters && pdf_prev >= 0) ? emitter_hit_weight(s, prims, E, ff.prim, o, pdf_prev) : 1.0;
          Lr = Lr + w * (beta * m.emission);
          break;
        }
        if (b == P.max_depth) break;
        const V3 x = o + (P.spawn_mode == 1 ? ff.t_u : ff.t_spawn) * d;
        const V3 wo = -d;
        const bool guided = P.guide != nullptr;
        const bool smooth = (m.type == kMatGGX && m.alpha < P.guide_min_roughness) ||
                            (m.type == kMatDisney && std::max(1e-3, double(m.dis[4]) * m.dis[4]) < P.guide_min_roughness);
        const double al = smooth ? 0.0 : P.guide_alpha;
        Mixture mix{};
        if (guided) {
          double Y[kGOut];
          guide_forward(P.guide_cfg, P.guide, x, wo, Y, nullptr);
          mix = guide_mixture(P.guide_cfg, Y);
        }
        // Density of the scattering technique (the MIS partner of light sampling).
        auto p_scatter = [&](V3 w) {
          const double pt = phase_pdf_approx(m, w, wo);
          return guided ? al * mixture_pdf(mix, w) + (1 - al) * pt : pt;
        };
        if (P.nee && L.has_quad && area > 0) {
          rng4(P.seed, uint32_t(p), sample, uint32_t(b), 3, U);
          const V3 y = L.corner + U[0] * L.e1 + U[1] * L.e2;
          const V3 w = y - x;
          const double r2 = dot(w, w), r = std::sqrt(r2);
          const V3 wl = (1.0 / r) * w;
          const double cl = -dot(wl, lnh);
          if (cl > 0) {
            const double pl = r2 / (area * cl);
            double Ue[6], U5[4];
            rng4(P.seed, uint32_t(p), sample, uint32_t(b), 4, Ue);
            rng4(P.seed, uint32_t(p), sample, uint32_t(b), 5, U5);
            Ue[4] = U5[0];
            Ue[5] = U5[1];
            const V3 f = phase_eval(m, wl, wo, Ue);
            if (f.x > 0 || f.y > 0 || f.z > 0) {
              const double tr = transmittance(prims, x, wl, 0.0, r, k, ff.prim, nullptr);
              ++shd;
              if (tr > 0) {
                const double wmis = mis2(pl, p_scatter(wl));
                Lr = Lr + (tr * wmis / pl) * (beta * (f * L.Le));
              }
            }
          }
        }
        if (P.nee_emitters && !E.ids.empty()) {
          double Ue[4], Uf[6], U10[4];
          rng4(P.seed, uint32_t(p), sample, uint32_t(b), 8, Ue);
          rng4(P.seed, uint32_t(p), sample, uint32_t(b), 9, Uf);
          rng4(P.seed, uint32_t(p), sample, uint32_t(b), 10, U10);
          Uf[4] = U10[0];
          Uf[5] = U10[1];
          V3 c, wl;
          double pl, cm;
          if (emitter_nee(s, prims, E, k, m, x, wo, ff.prim, Ue, Uf, &c, &wl, &pl, &cm, &shd))
            Lr = Lr + mis2(pl, cm * p_scatter(wl)) * (beta * c);
        }
        V3 wi, wgt;
        if (!guided) {
          rng4(P.seed, uint32_t(p), sample, uint32_t(b), 1, U);
          if (!phase_sample(m, wo, U, &wi, &wgt)) break;
          pdf_prev = phase_pdf_approx(m, wi, wo);
        } else {
          double G[4];
          rng4(P.seed, uint32_t(p), sample, uint32_t(b), 2, G);
          if (G[1] < al) {
            const double Gs[3] = {G[0], G[2], G[3]};
            wi = mixture_sample(mix, Gs);
            double Ug[6], U7[4];
            rng4(P.seed, uint32_t(p), sample, uint32_t(b), 6, Ug);
            rng4(P.seed, uint32_t(p), sample, uint32_t(b), 7, U7);
            Ug[4] = U7[0];
            Ug[5] = U7[1];
            const V3 f = phase_eval(m, wi, wo, Ug);
            const double pm = p_scatter(wi);
            if (!(pm > 0)) break;
            wgt = (1.0 / pm) * f;
            pdf_prev = pm;
          } else {
            rng4(P.seed, uint32_t(p), sample, uint32_t(b), 1, U);
            V3 w0;
            if (!phase_sample(m, wo, U, &wi, &w0)) break;
            const double pt = phase_pdf_approx(m, wi, wo);
            const double pm = al * mixture_pdf(mix, wi) + (1 - al) * pt;
            if (!(pm > 0)) break;
            wgt = (pt / pm) * w0;
            pdf_prev = pm;
          }
        }
        beta = beta * wgt;
        if (beta.x <= 0 && beta.y <= 0 && beta.z <= 0) break;
        o = x;
        d = wi;
        excl = ff.prim;
      }
      sum[0] += Lr.x; sum[1] += Lr.y; sum[2] += Lr.z;
      sq[0] += Lr.x * Lr.x; sq[1] += Lr.y * Lr.y; sq[2] += Lr.z * Lr.z;
    }
    for (int c = 0; c < 3; ++c) {
      accum[3 * p + c] += sum[c];
      accum_sq[3 * p + c] += sq[c];
    }
  }
  if (n_extend) *n_extend += ext;
  if (n_shadow) *n_shadow += shd;
  g_accel = nullptr;
}

}  // namespace orc
