// FP64 oracle: appearance of a Gaussian primitive (Sec. 6, App. B).
//
// TEST INFRASTRUCTURE ONLY. The phase function is the SGGX visible-normal distribution
// (Eq. 11) combined with a cosine-weighted base BSDF (Eq. 12). Directions point away from
// the scattering point: wo towards the viewer, wi towards the light.
#include <algorithm>
#include <cmath>

#include "oracle_phase.h"

namespace orc {

static const double kPi = 3.14159265358979323846;

// Orthonormal basis (b1, b2) completing the unit vector n (Duff et al., JCGT 2017).
void onb(V3 n, V3* b1, V3* b2) {
  const double sg = n.z >= 0 ? 1.0 : -1.0;
  const double a = -1.0 / (sg + n.z);
  const double b = n.x * n.y * a;
  *b1 = v3(1.0 + sg * n.x * n.x * a, sg * b, -sg * n.x);
  *b2 = v3(b, sg + n.y * n.y * a, -n.y);
}

// ------------------------------------------------------------------------------- SGGX
// S is stored as (Sxx, Syy, Szz, Sxy, Sxz, Syz).
static void sym(const double s6[6], double M[9]) {
  M[0] = s6[0]; M[1] = s6[3]; M[2] = s6[4];
  M[3] = s6[3]; M[4] = s6[1]; M[5] = s6[5];
  M[6] = s6[4]; M[7] = s6[5]; M[8] = s6[2];
}
static double quad_form(const double M[9], V3 a, V3 b) {
  return a.x * (M[0] * b.x + M[1] * b.y + M[2] * b.z) + a.y * (M[3] * b.x + M[4] * b.y + M[5] * b.z) +
         a.z * (M[6] * b.x + M[7] * b.y + M[8] * b.z);
}
static double det3(const double M[9]) {
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
         M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// Projected area sigma(w) = sqrt(w^T S w) (Heitz et al. 2015; Eq. 11).
double sggx_sigma(const double s6[6], V3 w) {
  double M[9];
  sym(s6, M);
  return std::sqrt(std::max(0.0, quad_form(M, w, w)));
}

// D(n) = 1 / (pi sqrt|S| (n^T S^-1 n)^2).
double sggx_D(const double s6[6], V3 n) {
  double M[9];
  sym(s6, M);
  const double det = det3(M);
  // n^T S^-1 n = n^T adj(S) n / det(S)
  double adj[9];
  adj[0] = M[4] * M[8] - M[5] * M[7]; adj[1] = M[2] * M[7] - M[1] * M[8]; adj[2] = M[1] * M[5] - M[2] * M[4];
  adj[3] = M[5] * M[6] - M[3] * M[8]; adj[4] = M[0] * M[8] - M[2] * M[6]; adj[5] = M[2] * M[3] - M[0] * M[5];
  adj[6] = M[3] * M[7] - M[4] * M[6]; adj[7] = M[1] * M[6] - M[0] * M[7]; adj[8] = M[0] * M[4] - M[1] * M[3];
  const double q = quad_form(adj, n, n) / det;
  return 1.0 / (kPi * std::sqrt(det) * q * q);
}

// Visible normal distribution D_wo(n) = <n.wo> D(n) / sigma(wo) (Eq. 11).
double sggx_Dvis(const double s6[6], V3 wo, V3 n) {
  const double c = dot(n, wo);
  if (c <= 0) return 0.0;
  return c * sggx_D(s6, n) / sggx_sigma(s6, wo);
}

// Visible-normal sampling.  The SGGX flakes are the normals of the ellipsoid {x : x^T S x <= 1},
// whose normal at x is proportional to S x.  Seen from wo, the visible half is sampled by drawing
// a point uniformly on the projected ellipse: in the frame (k, j, i = wo) write S = M M^T with the
// i-row of M equal to (0, 0, m_ii); a uniform point (u, v) of the unit disk lifted to the visible
// unit hemisphere w = (u, v, sqrt(1 - u^2 - v^2)) maps to the normal M w.  Solving M M^T = S row by
// row from the i-th row upwards gives the triangular factor used below.
V3 sggx_sample_vndf(const double s6[6], V3 wo, double U1, double U2) {
  double M[9];
  sym(s6, M);
  V3 wk, wj;
  onb(wo, &wk, &wj);
  const V3 wi = wo;
  const double Skk = quad_form(M, wk, wk), Sjj = quad_form(M, wj, wj), Sii = quad_form(M, wi, wi);
  const double Skj = quad_form(M, wk, wj), Ski = quad_form(M, wk, wi), Sji = quad_form(M, wj, wi);
  const double f = std::sqrt(Sii);
  const double e = Sji / f, d = Ski / f;
  const double c = std::sqrt(std::max(0.0, Sjj - e * e));
  const double b = (Skj - d * e) / c;
  const double a = std::sqrt(std::max(0.0, Skk - b * b - d * d));
  const double r = std::sqrt(U1), phi = 2 * kPi * U2;
  const double u = r * std::cos(phi), v = r * std::sin(phi);
  const double w = std::sqrt(std::max(0.0, 1.0 - u * u - v * v));
  // n_local = u * (a,0,0) + v * (b,c,0) + w * (d,e,f) in the (k, j, i) frame
  const V3 nl = v3(u * a + v * b + w * d, v * c + w * e, w * f);
  return normalize(nl.x * wk + nl.y * wj + nl.z * wi);
}

// Roughened SGGX of App. B: eigenvalues (s1 + a^2 s3, s2 + a^2 s3, s3), s1 <= s2 <= s3, same
// eigenvectors.  Eigen-decomposition by cyclic Jacobi rotations.
void sggx_roughen(const double s6[6], double alpha, double out6[6]) {
  double A[9], V[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  sym(s6, A);
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    if (off < 1e-30) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        const double apq = A[3 * p + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double th = (A[3 * q + q] - A[3 * p + p]) / (2 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1));
        const double cs = 1 / std::sqrt(t * t + 1), sn = t * cs;
        for (int k = 0; k < 3; ++k) {  // A <- J^T A J
          const double akp = A[3 * k + p], akq = A[3 * k + q];
          A[3 * k + p] = cs * akp - sn * akq;
          A[3 * k + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < 3; ++k) {
          const double apk = A[3 * p + k], aqk = A[3 * q + k];
          A[3 * p + k] = cs * apk - sn * aqk;
          A[3 * q + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const double vkp = V[3 * k + p], vkq = V[3 * k + q];
          V[3 * k + p] = cs * vkp - sn * vkq;
          V[3 * k + q] = sn * vkp + cs * vkq;
        }
      }
  }
  // App. B keeps the largest eigenvalue s3 and adds alpha^2 s3 to the other two. Where the
  // largest eigenvalue is shared (isotropic flakes), the eigenvector of the last such axis is
  // kept.
  const double ev[3] = {A[0], A[4], A[8]};
  int m = 0;
  for (int i = 1; i < 3; ++i)
    if (ev[i] >= ev[m]) m = i;
  const double s3 = ev[m];
  double nv[3];
  for (int i = 0; i < 3; ++i) nv[i] = i == m ? s3 : ev[i] + alpha * alpha * s3;
  double R[9] = {0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) R[3 * i + j] += V[3 * i + k] * nv[k] * V[3 * j + k];
  out6[0] = R[0]; out6[1] = R[4]; out6[2] = R[8]; out6[3] = R[1]; out6[4] = R[2]; out6[5] = R[5];
}

// ------------------------------------------------------------------------------- base BSDFs
// Cosine-weighted Lambertian: rho / pi <n.wi>, defined for normals facing wo.
V3 lambert_f(V3 rho, V3 wi, V3 wo, V3 n) {
  const double ci = dot(n, wi);
  if (ci <= 0 || dot(n, wo) <= 0) return v3(0, 0, 0);
  return (ci / kPi) * rho;
}

// GGX (isotropic, roughness alpha) with height-correlated Smith masking and Schlick Fresnel
// with F0 = albedo (Walter et al. 2007; Heitz 2014).
double ggx_D(double alpha, double cos_h) {
  if (cos_h <= 0) return 0.0;
  const double a2 = alpha * alpha;
  const double t = cos_h * cos_h * (a2 - 1.0) + 1.0;
  return a2 / (kPi * t * t);
}
double ggx_Lambda(double alpha, double cos_t) {
  const double c2 = cos_t * cos_t;
  const double tan2 = std::max(0.0, 1.0 - c2) / c2;
  return 0.5 * (-1.0 + std::sqrt(1.0 + alpha * alpha * tan2));
}
static V3 schlick(V3 F0, double c) {
  const double m = std::pow(std::max(0.0, 1.0 - c), 5.0);
  return v3(F0.x + (1 - F0.x) * m, F0.y + (1 - F0.y) * m, F0.z + (1 - F0.z) * m);
}
// f(wi, wo; n) <n.wi> = F D G2 / (4 <n.wo>)
V3 ggx_f(V3 F0, double alpha, V3 wi, V3 wo, V3 n) {
  const double ci = dot(n, wi), co = dot(n, wo);
  if (ci <= 0 || co <= 0) return v3(0, 0, 0);
  const V3 h = normalize(wi + wo);
  const double D = ggx_D(alpha, dot(n, h));
  const double G2 = 1.0 / (1.0 + ggx_Lambda(alpha, co) + ggx_Lambda(alpha, ci));
  return (D * G2 / (4.0 * co)) * schlick(F0, dot(wo, h));
}

// GGX visible-normal sampling (Heitz, JCGT 2018) in the frame of n: stretch the view direction
// to the unit-roughness configuration, sample the projected hemisphere with the half-disk warp,
// unstretch.  Returns the micro-normal h.
V3 ggx_sample_vn(double alpha, V3 wo, V3 n, double U1, double U2) {
  V3 t1, t2;
  onb(n, &t1, &t2);
  const V3 vl = v3(dot(wo, t1), dot(wo, t2), dot(wo, n));
  const V3 vh = normalize(v3(alpha * vl.x, alpha * vl.y, vl.z));
  const double l2 = vh.x * vh.x + vh.y * vh.y;
  const V3 T1 = l2 > 0 ? (1.0 / std::sqrt(l2)) * v3(-vh.y, vh.x, 0) : v3(1, 0, 0);
  const V3 T2 = cross(vh, T1);
  const double r = std::sqrt(U1), phi = 2 * kPi * U2;
  const double p1 = r * std::cos(phi);
  double p2 = r * std::sin(phi);
  const double sblend = 0.5 * (1.0 + vh.z);
  p2 = (1.0 - sblend) * std::sqrt(std::max(0.0, 1.0 - p1 * p1)) + sblend * p2;
  const V3 nh = p1 * T1 + p2 * T2 + std::sqrt(std::max(0.0, 1.0 - p1 * p1 - p2 * p2)) * vh;
  const V3 hl = normalize(v3(alpha * nh.x, alpha * nh.y, std::max(1e-12, nh.z)));
  return normalize(hl.x * t1 + hl.y * t2 + hl.z * n);
}

// pdf of n around h with density D(n.h) <n.h> (the "reversed" micro-normal sampling of Sec. 6).
double micro_pdf(double alpha, V3 n, V3 h) {
  const double c = dot(n, h);
  return c > 0 ? ggx_D(alpha, c) * c : 0.0;
}
V3 micro_sample(double alpha, V3 h, double U1, double U2) {
  const double a2 = alpha * alpha;
  const double c2 = (1.0 - U1) / (1.0 + (a2 - 1.0) * U1);
  const double c = std::sqrt(std::max(0.0, c2)), s = std::sqrt(std::max(0.0, 1.0 - c2));
  const double phi = 2 * kPi * U2;
  V3 t1, t2;
  onb(h, &t1, &t2);
  return normalize((s * std::cos(phi)) * t1 + (s * std::sin(phi)) * t2 + c * h);
}

V3 cos_sample(V3 n, double U1, double U2) {
  const double r = std::sqrt(U1), phi = 2 * kPi * U2;
  V3 t1, t2;
  onb(n, &t1, &t2);
  const double x = r * std::cos(phi), y = r * std::sin(phi);
  return normalize(x * t1 + y * t2 + std::sqrt(std::max(0.0, 1.0 - U1)) * n);
}

static double mis(double a, double b) { return a + b > 0 ? a / (a + b) : 0.0; }

static V3 base_f(const Material& m, V3 wi, V3 wo, V3 n) {
  if (m.type == kMatDisney) return disney_f(m, wi, wo, n);
  return m.type == kMatGGX ? ggx_f(m.albedo, m.alpha, wi, wo, n) : lambert_f(m.albedo, wi, wo, n);
}

bool sggx_isotropic(const double s6[6]) {
  return s6[0] == s6[1] && s6[1] == s6[2] && s6[3] == 0 && s6[4] == 0 && s6[5] == 0 && s6[0] > 0;
}

// Improved stochastic evaluation of Eq. 12 (Sec. 6, "Evaluation"): one VNDF sample n1 and one
// "reversed" base-BSDF sample, combined by the one-sample balance heuristic.  Specular base:
// n2 drawn around the half vector with density D(n.h)<n.h>; diffuse base: n3 drawn from the
// cosine lobe about wi.  U holds six uniforms.
V3 phase_eval_stochastic(const Material& m, V3 wi, V3 wo, const double U[6]) {
  const double* s6 = m.S;
  const V3 n1 = sggx_sample_vndf(s6, wo, U[0], U[1]);
  const double p1 = sggx_Dvis(s6, wo, n1);
  if (m.type == kMatDisney) {
    // each part with its own pair of techniques: the glossy part (specular and clearcoat) with
    // n2 around the half vector, the diffuse part (diffuse, subsurface, sheen) with n3 about wi
    const double a = disney_lobes(m).alpha;
    const V3 h = normalize(wi + wo);
    const V3 n2 = micro_sample(a, h, U[2], U[3]);
    const double q2 = micro_pdf(a, n2, h);
    V3 est = mis(p1, micro_pdf(a, n1, h)) * disney_f_glossy(m, wi, wo, n1);
    if (q2 > 0) {
      const double dv = sggx_Dvis(s6, wo, n2);
      est = est + (dv / q2 * mis(q2, dv)) * disney_f_glossy(m, wi, wo, n2);
    }
    const V3 n3 = cos_sample(wi, U[4], U[5]);
    const double q3 = std::max(0.0, dot(n3, wi)) / kPi;
    est = est + mis(p1, std::max(0.0, dot(n1, wi)) / kPi) * disney_f_diffuse(m, wi, wo, n1);
    if (q3 > 0) {
      const double dv = sggx_Dvis(s6, wo, n3);
      est = est + (dv / q3 * mis(q3, dv)) * disney_f_diffuse(m, wi, wo, n3);
    }
    return est;
  }
  if (m.type == kMatGGX) {
    const V3 h = normalize(wi + wo);
    const V3 n2 = micro_sample(m.alpha, h, U[2], U[3]);
    const double q2 = micro_pdf(m.alpha, n2, h);
    V3 est = mis(p1, micro_pdf(m.alpha, n1, h)) * base_f(m, wi, wo, n1);
    if (q2 > 0) {
      const double dv = sggx_Dvis(s6, wo, n2);
      est = est + (dv / q2 * mis(q2, dv)) * base_f(m, wi, wo, n2);
    }
    return est;
  }
  const V3 n3 = cos_sample(wi, U[4], U[5]);
  const double q3 = std::max(0.0, dot(n3, wi)) / kPi;
  V3 est = mis(p1, std::max(0.0, dot(n1, wi)) / kPi) * base_f(m, wi, wo, n1);
  if (q3 > 0) {
    const double dv = sggx_Dvis(s6, wo, n3);
    est = est + (dv / q3 * mis(q3, dv)) * base_f(m, wi, wo, n3);
  }
  return est;
}

// Isotropic flakes (S = I) with a Lambertian base: with D = 1/pi, Eq. 12 reduces to
// rho / pi^2 int <n.wo><n.wi> dn = rho * 2 / (3 pi^2) [(pi - g) cos g + sin g], g = angle(wi, wo).
V3 phase_eval_lambert_sphere(V3 rho, V3 wi, V3 wo) {
  const double c = std::max(-1.0, std::min(1.0, dot(wi, wo)));
  const double g = std::acos(c);
  const double v = 2.0 / (3.0 * kPi * kPi) * ((kPi - g) * c + std::sin(g));
  return v * rho;
}

V3 phase_eval(const Material& m, V3 wi, V3 wo, const double U[6]) {
  if (m.type == kMatDiffuse && sggx_isotropic(m.S)) return phase_eval_lambert_sphere(m.albedo, wi, wo);
  return phase_eval_stochastic(m, wi, wo, U);
}

// Importance sampling (Sec. 6): n ~ D_wo, then wi from the base BSDF around n; the weight
// f / pdf is the base BSDF's own (the VNDF sampling is exact).  U holds four uniforms.
bool phase_sample(const Material& m, V3 wo, const double U[4], V3* wi, V3* weight) {
  const V3 n = sggx_sample_vndf(m.S, wo, U[0], U[1]);
  if (m.type == kMatDisney) return disney_sample(m, wo, n, U + 2, wi, weight);
  if (m.type == kMatGGX) {
    const V3 h = ggx_sample_vn(m.alpha, wo, n, U[2], U[3]);
    const double oh = dot(wo, h);
    *wi = normalize((2.0 * oh) * h - wo);
    const double ci = dot(n, *wi), co = dot(n, wo);
    if (ci <= 0 || co <= 0 || oh <= 0) {
      *weight = v3(0, 0, 0);
      return false;
    }
    const double L_o = ggx_Lambda(m.alpha, co), L_i = ggx_Lambda(m.alpha, ci);
    const double w = (1.0 + L_o) / (1.0 + L_o + L_i);  // G2 / G1(wo)
    *weight = w * schlick(m.albedo, oh);
    return true;
  }
  *wi = cos_sample(n, U[2], U[3]);
  *weight = m.albedo;
  return true;
}

// Approximate pdf of App. B, taken as written: specular part D~_wo(w_h) with the roughened
// SGGX, diffuse part <w_h.wo> / pi, where w_h = normalize(wi + wo).
double phase_pdf_approx(const Material& m, V3 wi, V3 wo) {
  const V3 s = wi + wo;
  const double l = length(s);
  if (l <= 1e-12) return 0.0;
  const V3 h = (1.0 / l) * s;
  if (m.type == kMatGGX) {
    double r6[6];
    sggx_roughen(m.S, m.alpha, r6);
    return sggx_Dvis(r6, wo, h);
  }
  if (m.type == kMatDisney) {
    // the lobes weighted as the sampler picks them (by metallic and base-colour luminance)
    const DisneyLobes L = disney_lobes(m);
    double r6[6];
    sggx_roughen(m.S, L.alpha, r6);
    double p = L.p_spec * sggx_Dvis(r6, wo, h) + L.p_diffuse * std::max(0.0, dot(h, wo)) / kPi;
    if (L.p_coat > 0) {
      sggx_roughen(m.S, L.alpha_c, r6);
      p += L.p_coat * sggx_Dvis(r6, wo, h);
    }
    return p;
  }
  return std::max(0.0, dot(h, wo)) / kPi;
}

}  // namespace orc
