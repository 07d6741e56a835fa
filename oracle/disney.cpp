// FP64 oracle: the Disney principled base BSDF (Burley 2012, isotropic; the paper's Sec. 6 base
// BSDF with 12 parameters), cosine-weighted like the other base BSDFs, with its sampling and pdf.
//
// TEST INFRASTRUCTURE ONLY. Parameters: base colour C (3) and, in Material::dis, metallic,
// subsurface, specular, specular tint, roughness, sheen, sheen tint, clearcoat, clearcoat gloss.
// Written from the published model:
//  * diffuse: C / pi (1 + (F_D90 - 1)(1 - cos_l)^5)(1 + (F_D90 - 1)(1 - cos_v)^5),
//    F_D90 = 1/2 + 2 roughness cos_d^2, blended with the Hanrahan-Krueger-like subsurface term
//    1.25 (F_ss (1 / (cos_l + cos_v) - 1/2) + 1/2), F_ss90 = roughness cos_d^2;
//  * sheen: (1 - cos_d)^5 sheen mix(1, C_tint, sheen tint), C_tint = C / lum(C);
//    diffuse and sheen are scaled by (1 - metallic);
//  * specular: GGX with alpha = max(1e-3, roughness^2), height-correlated Smith masking and
//    Schlick Fresnel from C_spec0 = mix(0.08 specular mix(1, C_tint, specular tint), C, metallic)
//    (the oracle's GGX base with that F0);
//  * clearcoat: 1/4 clearcoat GTR1(alpha_c = mix(0.1, 0.001, gloss)) Schlick(0.04) with separable
//    Smith masking of roughness 0.25.
// lum(C) = 0.3 R + 0.6 G + 0.1 B as in the published model.
// Pins: the GGX reduction (metallic 1, no clearcoat), the normal-incidence values of the diffuse,
// subsurface and sheen terms, their grazing and 60-degree values where the published formulas
// reduce to exact numbers (retro-reflection (1/2 + 2 roughness)^2 at grazing, the Schlick weight,
// F_ss90, the sheen colour at theta_d = 90 degrees; a hand-derived fixture), reciprocity, the GTR1
// normalisation, and the sampler against its pdf and the albedo by quadrature.
#include <algorithm>
#include <cmath>

#include "oracle_phase.h"

namespace orc {

static const double kPi = 3.14159265358979323846;

static double lum(V3 c) { return 0.3 * c.x + 0.6 * c.y + 0.1 * c.z; }
static double pow5(double x) {
  const double c = std::min(1.0, std::max(0.0, x));
  return c * c * c * c * c;
}
static V3 mix3(V3 a, V3 b, double t) { return v3(a.x + (b.x - a.x) * t, a.y + (b.y - a.y) * t, a.z + (b.z - a.z) * t); }

// Generalised-Trowbridge-Reitz with exponent 1 (clearcoat), normalised so that
// int D(n.h) (n.h) dh = 1.
double gtr1_D(double a, double cos_h) {
  if (cos_h <= 0) return 0.0;
  if (a >= 1.0) return 1.0 / kPi;
  const double a2 = a * a;
  const double t = 1.0 + (a2 - 1.0) * cos_h * cos_h;
  return (a2 - 1.0) / (kPi * std::log(a2) * t);
}
// GGX Smith masking G1 for the separable clearcoat term.
static double smith_g1(double cos_t, double a) {
  const double c2 = cos_t * cos_t, a2 = a * a;
  return 2.0 * cos_t / (cos_t + std::sqrt(a2 + c2 - a2 * c2));
}

DisneyLobes disney_lobes(const Material& m) {
  DisneyLobes L;
  const V3 C = m.albedo;
  const double l = lum(C);
  const V3 tint = l > 0 ? (1.0 / l) * C : v3(1, 1, 1);
  const double metallic = m.dis[0], specular = m.dis[2], spec_tint = m.dis[3], rough = m.dis[4];
  const double sheen_tint = m.dis[6], clearcoat = m.dis[7], gloss = m.dis[8];
  L.spec0 = mix3((0.08 * specular) * mix3(v3(1, 1, 1), tint, spec_tint), C, metallic);
  L.sheen = mix3(v3(1, 1, 1), tint, sheen_tint);
  L.alpha = std::max(1e-3, rough * rough);
  L.alpha_c = 0.1 + (0.001 - 0.1) * gloss;
  // lobe choice for sampling, by rough energy: any positive weights keep sampling unbiased
  const double wd = (1.0 - metallic) * l;
  const double ws = lum(L.spec0) + 0.04;
  const double wc = 0.25 * clearcoat * 0.04 + (clearcoat > 0 ? 0.02 : 0.0);
  const double s = wd + ws + wc;
  L.p_diffuse = wd / s;
  L.p_spec = ws / s;
  L.p_coat = wc / s;
  return L;
}

// Diffuse, subsurface and sheen part (times <n.wi>), zero outside the upper hemisphere.
V3 disney_f_diffuse(const Material& m, V3 wi, V3 wo, V3 n) {
  const double cl = dot(n, wi), cv = dot(n, wo);
  if (cl <= 0 || cv <= 0) return v3(0, 0, 0);
  const DisneyLobes L = disney_lobes(m);
  const V3 h = normalize(wi + wo);
  const double cd = dot(wi, h);
  const double FL = pow5(1.0 - cl), FV = pow5(1.0 - cv), FH = pow5(1.0 - cd);
  const double rough = m.dis[4];
  const double fd90 = 0.5 + 2.0 * cd * cd * rough;
  const double Fd = (1.0 + (fd90 - 1.0) * FL) * (1.0 + (fd90 - 1.0) * FV);
  const double fss90 = cd * cd * rough;
  const double Fss = (1.0 + (fss90 - 1.0) * FL) * (1.0 + (fss90 - 1.0) * FV);
  const double ss = 1.25 * (Fss * (1.0 / (cl + cv) - 0.5) + 0.5);
  const double diff = (Fd + (ss - Fd) * m.dis[1]) / kPi;
  const V3 sheen = (FH * m.dis[5]) * L.sheen;
  return ((1.0 - m.dis[0]) * cl) * (diff * m.albedo + sheen);
}

// Specular and clearcoat part (times <n.wi>).
V3 disney_f_glossy(const Material& m, V3 wi, V3 wo, V3 n) {
  const double cl = dot(n, wi), cv = dot(n, wo);
  if (cl <= 0 || cv <= 0) return v3(0, 0, 0);
  const DisneyLobes L = disney_lobes(m);
  V3 f = ggx_f(L.spec0, L.alpha, wi, wo, n);
  if (m.dis[7] > 0) {
    const V3 h = normalize(wi + wo);
    const double Fr = 0.04 + 0.96 * pow5(1.0 - dot(wi, h));
    const double Gr = smith_g1(cl, 0.25) * smith_g1(cv, 0.25);
    const double c = 0.25 * m.dis[7] * Fr * gtr1_D(L.alpha_c, dot(n, h)) * Gr / (4.0 * cv);
    f = f + v3(c, c, c);
  }
  return f;
}

V3 disney_f(const Material& m, V3 wi, V3 wo, V3 n) { return disney_f_diffuse(m, wi, wo, n) + disney_f_glossy(m, wi, wo, n); }

// Density of the base sampler below: the lobe mixture of cosine, GGX visible-normal and GTR1
// half-vector sampling (reflection about the sampled half vector).
double disney_pdf(const Material& m, V3 wi, V3 wo, V3 n) {
  const double cl = dot(n, wi), cv = dot(n, wo);
  if (cl <= 0 || cv <= 0) return 0.0;
  const DisneyLobes L = disney_lobes(m);
  const V3 h = normalize(wi + wo);
  const double ch = dot(n, h), oh = dot(wo, h);
  double p = L.p_diffuse * cl / kPi;
  const double G1o = 1.0 / (1.0 + ggx_Lambda(L.alpha, cv));
  p += L.p_spec * G1o * ggx_D(L.alpha, ch) / (4.0 * cv);
  if (L.p_coat > 0 && oh > 0) p += L.p_coat * gtr1_D(L.alpha_c, ch) * ch / (4.0 * oh);
  return p;
}

// One sample from two uniforms: U[0] picks the lobe and, rescaled to [0, 1) within the lobe's
// share, drives the lobe's sampler with U[1]. The weight is f <n.wi> / pdf of the whole mixture.
bool disney_sample(const Material& m, V3 wo, V3 n, const double U[2], V3* wi, V3* weight) {
  const DisneyLobes L = disney_lobes(m);
  *weight = v3(0, 0, 0);
  if (dot(n, wo) <= 0) return false;
  const double u = U[0];
  if (u < L.p_diffuse) {
    *wi = cos_sample(n, u / L.p_diffuse, U[1]);
  } else if (u < L.p_diffuse + L.p_spec || L.p_coat <= 0) {
    const double u1 = std::min(1.0 - 1e-16, (u - L.p_diffuse) / L.p_spec);
    const V3 h = ggx_sample_vn(L.alpha, wo, n, u1, U[1]);
    *wi = normalize((2.0 * dot(wo, h)) * h - wo);
  } else {
    const double u1 = std::min(1.0 - 1e-16, (u - L.p_diffuse - L.p_spec) / L.p_coat);
    const double a2 = L.alpha_c * L.alpha_c;
    const double c2 = (1.0 - std::pow(a2, 1.0 - u1)) / (1.0 - a2);
    const double c = std::sqrt(std::max(0.0, std::min(1.0, c2))), s = std::sqrt(std::max(0.0, 1.0 - c * c));
    V3 t1, t2;
    onb(n, &t1, &t2);
    const double ph = 2.0 * kPi * U[1];
    const V3 h = normalize((s * std::cos(ph)) * t1 + (s * std::sin(ph)) * t2 + c * n);
    *wi = normalize((2.0 * dot(wo, h)) * h - wo);
  }
  const double p = disney_pdf(m, *wi, wo, n);
  if (!(p > 0)) return false;
  *weight = (1.0 / p) * disney_f(m, *wi, wo, n);
  return true;
}

}  // namespace orc
