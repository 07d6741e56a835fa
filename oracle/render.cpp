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

void render_pixels(const SceneIn& s, const Camera& cam, const Lights& L, const RenderParams& P,
                   int64_t p_begin, int64_t p_end, double* accum, double* accum_sq, int64_t* n_extend,
                   int64_t* n_shadow) {
  const std::vector<Prim> prims = make_prims(s);
  const double k = cutoff_k(P.cutoff_eps);
  const V3 ln = cross(L.e1, L.e2);
  const double area = length(ln);
  const V3 lnh = area > 0 ? (1.0 / area) * ln : v3(0, 0, 1);
  int64_t ext = 0, shd = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : ext, shd)
  for (int64_t p = p_begin; p < p_end; ++p) {
    const int px = int(p % cam.width), py = int(p / cam.width);
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
          Lr = Lr + beta * m.emission;
          break;
        }
        if (b == P.max_depth) break;
        const V3 x = o + (P.spawn_mode == 1 ? ff.t_u : ff.t_spawn) * d;
        const V3 wo = -d;
        const bool guided = P.guide != nullptr;
        const double al = P.guide_alpha;
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
}

}  // namespace orc
