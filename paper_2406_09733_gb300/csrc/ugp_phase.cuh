// Appearance of a Gaussian primitive (Sec. 6, Eq. 11-12, App. B) in float32 device code.
//
// The phase function is the SGGX visible-normal distribution D_wo(n) (Heitz et al. 2015)
// combined with a cosine-weighted base BSDF f(wi, wo; n): Lambertian (rho / pi <n.wi>), GGX
// (F D G2 / (4 <n.wo>), height-correlated Smith, Schlick Fresnel with F0 = albedo), or the
// isotropic Disney principled BRDF with its 12 parameters (base colour and nine scalars).
// Directions point away from the scattering point: wo to the viewer, wi to the light.
#pragma once

#include <math.h>

namespace ugp {

constexpr float kPiF = 3.14159265358979f;
constexpr int kMatDiffuse = 0, kMatGGX = 1, kMatEmissive = 2, kMatDisney = 3;

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize3(float3 a) { return rsqrtf(dot3(a, a)) * a; }

struct Material {
  int type;
  float3 albedo;  // albedo, F0 of the GGX base, or the Disney base colour
  float alpha;
  float S[6];  // SGGX matrix (Sxx, Syy, Szz, Sxy, Sxz, Syz)
  // Disney parameters (type 3 only): metallic, subsurface, specular, specular tint, roughness,
  // sheen, sheen tint, clearcoat, clearcoat gloss.
  float dis[9];
};

// Orthonormal basis completing a unit vector (Duff et al., JCGT 2017).
__device__ __forceinline__ void onb3(float3 n, float3& b1, float3& b2) {
  const float sg = n.z >= 0.f ? 1.f : -1.f;
  const float a = -1.f / (sg + n.z);
  const float b = n.x * n.y * a;
  b1 = f3(1.f + sg * n.x * n.x * a, sg * b, -sg * n.x);
  b2 = f3(b, sg + n.y * n.y * a, -n.y);
}

// ---------------------------------------------------------------------------- SGGX
__device__ __forceinline__ float sggx_form(const float S[6], float3 a, float3 b) {
  return a.x * (S[0] * b.x + S[3] * b.y + S[4] * b.z) + a.y * (S[3] * b.x + S[1] * b.y + S[5] * b.z) +
         a.z * (S[4] * b.x + S[5] * b.y + S[2] * b.z);
}
__device__ __forceinline__ float sggx_sigma(const float S[6], float3 w) { return sqrtf(fmaxf(0.f, sggx_form(S, w, w))); }

// D(n) = 1 / (pi sqrt|S| (n^T S^-1 n)^2), with n^T S^-1 n = n^T adj(S) n / |S|.
__device__ __forceinline__ float sggx_D(const float S[6], float3 n) {
  const float xx = S[0], yy = S[1], zz = S[2], xy = S[3], xz = S[4], yz = S[5];
  const float a00 = yy * zz - yz * yz, a11 = xx * zz - xz * xz, a22 = xx * yy - xy * xy;
  const float a01 = xz * yz - xy * zz, a02 = xy * yz - xz * yy, a12 = xy * xz - xx * yz;
  const float det = xx * a00 + xy * a01 + xz * a02;
  const float q = (n.x * n.x * a00 + n.y * n.y * a11 + n.z * n.z * a22 +
                   2.f * (n.x * n.y * a01 + n.x * n.z * a02 + n.y * n.z * a12)) / det;
  return 1.f / (kPiF * sqrtf(det) * q * q);
}

__device__ __forceinline__ float sggx_dvis(const float S[6], float3 wo, float3 n) {
  const float c = dot3(n, wo);
  return c > 0.f ? c * sggx_D(S, n) / sggx_sigma(S, wo) : 0.f;
}

// Visible-normal sample.  The flakes are the normals of the ellipsoid {x : x^T S x <= 1}; seen
// from wo, a uniform point of the projected ellipse lifted to the visible surface has normal M w,
// where w is the corresponding point of the visible unit hemisphere and M M^T = S in the frame
// (k, j, i = wo) with the i-row of M reduced to (0, 0, m_ii).
__device__ __forceinline__ float3 sggx_sample_vndf(const float S[6], float3 wo, float U1, float U2) {
  float3 wk, wj;
  onb3(wo, wk, wj);
  const float Skk = sggx_form(S, wk, wk), Sjj = sggx_form(S, wj, wj), Sii = sggx_form(S, wo, wo);
  const float Skj = sggx_form(S, wk, wj), Ski = sggx_form(S, wk, wo), Sji = sggx_form(S, wj, wo);
  const float f = sqrtf(Sii);
  const float e = Sji / f, d = Ski / f;
  const float c = sqrtf(fmaxf(1e-30f, Sjj - e * e));
  const float b = (Skj - d * e) / c;
  const float a = sqrtf(fmaxf(0.f, Skk - b * b - d * d));
  const float r = sqrtf(U1);
  float sp, cp;
  sincospif(2.f * U2, &sp, &cp);
  const float u = r * cp, v = r * sp;
  const float w = sqrtf(fmaxf(0.f, 1.f - u * u - v * v));
  const float3 nl = f3(u * a + v * b + w * d, v * c + w * e, w * f);
  return normalize3(nl.x * wk + nl.y * wj + nl.z * wo);
}

// Roughened SGGX of App. B: eigenvalues (s1 + a^2 s3, s2 + a^2 s3, s3) with s1 <= s2 <= s3 and
// the same eigenvectors, i.e. S + a^2 s3 (I - v3 v3^T) with (s3, v3) the largest eigenpair.
// Cyclic Jacobi rotations give the eigen-decomposition.
__device__ inline void sggx_roughen(const float S[6], float alpha, float out[6]) {
  float A[3][3] = {{S[0], S[3], S[4]}, {S[3], S[1], S[5]}, {S[4], S[5], S[2]}};
  float V[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
  for (int sweep = 0; sweep < 8; ++sweep) {
    const float off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const float dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-14f * dia) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        const float apq = A[p][q];
        if (fabsf(apq) < 1e-30f) continue;
        const float th = (A[q][q] - A[p][p]) / (2.f * apq);
        const float t = copysignf(1.f, th) / (fabsf(th) + sqrtf(th * th + 1.f));
        const float cs = rsqrtf(t * t + 1.f), sn = t * cs;
        for (int k = 0; k < 3; ++k) {
          const float akp = A[k][p], akq = A[k][q];
          A[k][p] = cs * akp - sn * akq;
          A[k][q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < 3; ++k) {
          const float apk = A[p][k], aqk = A[q][k];
          A[p][k] = cs * apk - sn * aqk;
          A[q][k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const float vkp = V[k][p], vkq = V[k][q];
          V[k][p] = cs * vkp - sn * vkq;
          V[k][q] = sn * vkp + cs * vkq;
        }
      }
  }
  int m = 0;  // the largest eigenvalue; where it is shared, the last such axis
  if (A[1][1] >= A[m][m]) m = 1;
  if (A[2][2] >= A[m][m]) m = 2;
  const float s3 = A[m][m], add = alpha * alpha * s3;
  const float3 v = f3(V[0][m], V[1][m], V[2][m]);
  out[0] = S[0] + add * (1.f - v.x * v.x);
  out[1] = S[1] + add * (1.f - v.y * v.y);
  out[2] = S[2] + add * (1.f - v.z * v.z);
  out[3] = S[3] - add * v.x * v.y;
  out[4] = S[4] - add * v.x * v.z;
  out[5] = S[5] - add * v.y * v.z;
}

// ---------------------------------------------------------------------------- base BSDFs
__device__ __forceinline__ float3 lambert_f(float3 rho, float3 wi, float3 wo, float3 n) {
  const float ci = dot3(n, wi);
  if (ci <= 0.f || dot3(n, wo) <= 0.f) return f3(0.f, 0.f, 0.f);
  return (ci / kPiF) * rho;
}

__device__ __forceinline__ float ggx_D(float alpha, float ch) {
  if (ch <= 0.f) return 0.f;
  const float a2 = alpha * alpha;
  const float t = ch * ch * (a2 - 1.f) + 1.f;
  return a2 / (kPiF * t * t);
}
__device__ __forceinline__ float ggx_lambda(float alpha, float c) {
  const float c2 = c * c;
  const float tan2 = fmaxf(0.f, 1.f - c2) / c2;
  return 0.5f * (-1.f + sqrtf(1.f + alpha * alpha * tan2));
}
__device__ __forceinline__ float3 schlick(float3 F0, float c) {
  const float m1 = fmaxf(0.f, 1.f - c), m2 = m1 * m1, m = m2 * m2 * m1;
  return f3(F0.x + (1.f - F0.x) * m, F0.y + (1.f - F0.y) * m, F0.z + (1.f - F0.z) * m);
}
__device__ __forceinline__ float3 ggx_f(float3 F0, float alpha, float3 wi, float3 wo, float3 n) {
  const float ci = dot3(n, wi), co = dot3(n, wo);
  if (ci <= 0.f || co <= 0.f) return f3(0.f, 0.f, 0.f);
  const float3 h = normalize3(wi + wo);
  const float D = ggx_D(alpha, dot3(n, h));
  const float G2 = 1.f / (1.f + ggx_lambda(alpha, co) + ggx_lambda(alpha, ci));
  return (D * G2 / (4.f * co)) * schlick(F0, dot3(wo, h));
}

// GGX visible-normal sampling (Heitz, JCGT 2018) in the frame of n.
__device__ __forceinline__ float3 ggx_sample_vn(float alpha, float3 wo, float3 n, float U1, float U2) {
  float3 t1, t2;
  onb3(n, t1, t2);
  const float3 vl = f3(dot3(wo, t1), dot3(wo, t2), dot3(wo, n));
  const float3 vh = normalize3(f3(alpha * vl.x, alpha * vl.y, vl.z));
  const float l2 = vh.x * vh.x + vh.y * vh.y;
  const float3 T1 = l2 > 0.f ? rsqrtf(l2) * f3(-vh.y, vh.x, 0.f) : f3(1.f, 0.f, 0.f);
  const float3 T2 = cross3(vh, T1);
  const float r = sqrtf(U1);
  float sp, cp;
  sincospif(2.f * U2, &sp, &cp);
  const float p1 = r * cp;
  float p2 = r * sp;
  const float sb = 0.5f * (1.f + vh.z);
  p2 = (1.f - sb) * sqrtf(fmaxf(0.f, 1.f - p1 * p1)) + sb * p2;
  const float3 nh = p1 * T1 + p2 * T2 + sqrtf(fmaxf(0.f, 1.f - p1 * p1 - p2 * p2)) * vh;
  const float3 hl = normalize3(f3(alpha * nh.x, alpha * nh.y, fmaxf(1e-7f, nh.z)));
  return normalize3(hl.x * t1 + hl.y * t2 + hl.z * n);
}

// Normals drawn around a half vector with density D(n.h) <n.h> (the "reversed" sampling of Sec. 6).
__device__ __forceinline__ float micro_pdf(float alpha, float3 n, float3 h) {
  const float c = dot3(n, h);
  return c > 0.f ? ggx_D(alpha, c) * c : 0.f;
}
__device__ __forceinline__ float3 micro_sample(float alpha, float3 h, float U1, float U2) {
  const float a2 = alpha * alpha;
  const float c2 = (1.f - U1) / (1.f + (a2 - 1.f) * U1);
  const float c = sqrtf(fmaxf(0.f, c2)), s = sqrtf(fmaxf(0.f, 1.f - c2));
  float sp, cp;
  sincospif(2.f * U2, &sp, &cp);
  float3 t1, t2;
  onb3(h, t1, t2);
  return normalize3((s * cp) * t1 + (s * sp) * t2 + c * h);
}
__device__ __forceinline__ float3 cos_sample(float3 n, float U1, float U2) {
  const float r = sqrtf(U1);
  float sp, cp;
  sincospif(2.f * U2, &sp, &cp);
  float3 t1, t2;
  onb3(n, t1, t2);
  return normalize3((r * cp) * t1 + (r * sp) * t2 + sqrtf(fmaxf(0.f, 1.f - U1)) * n);
}

__device__ __forceinline__ float mis_w(float a, float b) { return a + b > 0.f ? a / (a + b) : 0.f; }

// ---------------------------------------------------------------------------- Disney base
// The isotropic principled BRDF (Burley 2012) as the base of Eq. 12, cosine-weighted like the
// others: a diffuse part (retro-reflective diffuse blended with the subsurface approximation,
// plus sheen, all scaled by 1 - metallic) and a glossy part (GGX specular with height-correlated
// Smith masking and Schlick Fresnel from the specular colour, plus a GTR1 clearcoat with
// separable Smith masking of roughness 1/4).
struct DisneyLobes {
  float3 spec0;    // specular colour at normal incidence
  float3 sheen_c;  // sheen colour
  float alpha, alpha_c;
  float p_diffuse, p_spec, p_coat;  // lobe choice of the sampler (also the App. B weights)
};

__device__ __forceinline__ float lum3(float3 c) { return 0.3f * c.x + 0.6f * c.y + 0.1f * c.z; }
__device__ __forceinline__ float schlick_w(float c) {
  const float m1 = fminf(1.f, fmaxf(0.f, 1.f - c)), m2 = m1 * m1;
  return m2 * m2 * m1;
}
__device__ __forceinline__ float3 lerp3(float3 a, float3 b, float t) {
  return f3(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y), fmaf(t, b.z - a.z, a.z));
}

__device__ __forceinline__ DisneyLobes disney_lobes(const Material& m) {
  DisneyLobes L;
  const float l = lum3(m.albedo);
  const float3 one = f3(1.f, 1.f, 1.f);
  const float3 tint = l > 0.f ? (1.f / l) * m.albedo : one;
  const float metallic = m.dis[0], clearcoat = m.dis[7];
  L.spec0 = lerp3((0.08f * m.dis[2]) * lerp3(one, tint, m.dis[3]), m.albedo, metallic);
  L.sheen_c = lerp3(one, tint, m.dis[6]);
  L.alpha = fmaxf(1e-3f, m.dis[4] * m.dis[4]);
  L.alpha_c = fmaf(m.dis[8], 0.001f - 0.1f, 0.1f);
  const float wd = (1.f - metallic) * l;
  const float ws = lum3(L.spec0) + 0.04f;
  const float wc = 0.01f * clearcoat + (clearcoat > 0.f ? 0.02f : 0.f);
  const float inv = 1.f / (wd + ws + wc);
  L.p_diffuse = wd * inv;
  L.p_spec = ws * inv;
  L.p_coat = wc * inv;
  return L;
}

// Clearcoat normal distribution (generalised Trowbridge-Reitz, exponent 1), normalised so that
// its projected integral over the hemisphere is 1.
__device__ __forceinline__ float gtr1_D(float a, float ch) {
  if (ch <= 0.f) return 0.f;
  if (a >= 1.f) return 1.f / kPiF;
  const float a2 = a * a;
  return (a2 - 1.f) / (kPiF * logf(a2) * fmaf(a2 - 1.f, ch * ch, 1.f));
}
__device__ __forceinline__ float smith_g1_sep(float c, float a) {
  const float c2 = c * c, a2 = a * a;
  return 2.f * c / (c + sqrtf(a2 + c2 - a2 * c2));
}

// Diffuse, subsurface and sheen (times <n.wi>).
__device__ inline float3 disney_f_diffuse(const Material& m, const DisneyLobes& L, float3 wi, float3 wo, float3 n) {
  const float cl = dot3(n, wi), cv = dot3(n, wo);
  if (cl <= 0.f || cv <= 0.f) return f3(0.f, 0.f, 0.f);
  const float3 h = normalize3(wi + wo);
  const float cd = dot3(wi, h);
  const float FL = schlick_w(cl), FV = schlick_w(cv), FH = schlick_w(cd);
  const float r = m.dis[4], cd2 = cd * cd;
  const float fd90 = fmaf(2.f * r, cd2, 0.5f);
  const float Fd = fmaf(fd90 - 1.f, FL, 1.f) * fmaf(fd90 - 1.f, FV, 1.f);
  const float fss90 = r * cd2;
  const float Fss = fmaf(fss90 - 1.f, FL, 1.f) * fmaf(fss90 - 1.f, FV, 1.f);
  const float ss = 1.25f * fmaf(Fss, 1.f / (cl + cv) - 0.5f, 0.5f);
  const float diff = fmaf(m.dis[1], ss - Fd, Fd) * (1.f / kPiF);
  const float k = (1.f - m.dis[0]) * cl;
  const float sh = FH * m.dis[5];
  return f3(k * fmaf(diff, m.albedo.x, sh * L.sheen_c.x), k * fmaf(diff, m.albedo.y, sh * L.sheen_c.y),
            k * fmaf(diff, m.albedo.z, sh * L.sheen_c.z));
}

// Specular and clearcoat (times <n.wi>).
__device__ inline float3 disney_f_glossy(const Material& m, const DisneyLobes& L, float3 wi, float3 wo, float3 n) {
  const float cl = dot3(n, wi), cv = dot3(n, wo);
  if (cl <= 0.f || cv <= 0.f) return f3(0.f, 0.f, 0.f);
  float3 f = ggx_f(L.spec0, L.alpha, wi, wo, n);
  if (m.dis[7] > 0.f) {
    const float3 h = normalize3(wi + wo);
    const float Fr = fmaf(0.96f, schlick_w(dot3(wi, h)), 0.04f);
    const float G = smith_g1_sep(cl, 0.25f) * smith_g1_sep(cv, 0.25f);
    const float c = 0.25f * m.dis[7] * Fr * gtr1_D(L.alpha_c, dot3(n, h)) * G / (4.f * cv);
    f = f + f3(c, c, c);
  }
  return f;
}

// Density of the lobe-mixture sampler below (cosine, GGX visible normals, GTR1 half vectors).
__device__ inline float disney_pdf(const DisneyLobes& L, float3 wi, float3 wo, float3 n) {
  const float cl = dot3(n, wi), cv = dot3(n, wo);
  if (cl <= 0.f || cv <= 0.f) return 0.f;
  const float3 h = normalize3(wi + wo);
  const float ch = dot3(n, h), oh = dot3(wo, h);
  float p = L.p_diffuse * cl / kPiF;
  p += L.p_spec * ggx_D(L.alpha, ch) / ((1.f + ggx_lambda(L.alpha, cv)) * 4.f * cv);
  if (L.p_coat > 0.f && oh > 0.f) p += L.p_coat * gtr1_D(L.alpha_c, ch) * ch / (4.f * oh);
  return p;
}

// One sample about the micro-normal n: U[0] picks the lobe and, rescaled within the lobe's share,
// drives its sampler with U[1]. The weight is f <n.wi> over the mixture's density.
__device__ inline bool disney_sample(const Material& m, float3 wo, float3 n, const float U[2], float3& wi,
                                     float3& weight) {
  const DisneyLobes L = disney_lobes(m);
  weight = f3(0.f, 0.f, 0.f);
  if (dot3(n, wo) <= 0.f) return false;
  const float u = U[0];
  if (u < L.p_diffuse) {
    wi = cos_sample(n, u / L.p_diffuse, U[1]);
  } else if (u < L.p_diffuse + L.p_spec || L.p_coat <= 0.f) {
    const float u1 = fminf(0.99999994f, (u - L.p_diffuse) / L.p_spec);
    const float3 h = ggx_sample_vn(L.alpha, wo, n, u1, U[1]);
    wi = normalize3((2.f * dot3(wo, h)) * h - wo);
  } else {
    const float u1 = fminf(0.99999994f, (u - L.p_diffuse - L.p_spec) / L.p_coat);
    const float a2 = L.alpha_c * L.alpha_c;
    const float c2 = (1.f - powf(a2, 1.f - u1)) / (1.f - a2);
    const float c = sqrtf(fmaxf(0.f, fminf(1.f, c2))), sn = sqrtf(fmaxf(0.f, 1.f - c * c));
    float sp, cp;
    sincospif(2.f * U[1], &sp, &cp);
    float3 t1, t2;
    onb3(n, t1, t2);
    const float3 h = normalize3((sn * cp) * t1 + (sn * sp) * t2 + c * n);
    wi = normalize3((2.f * dot3(wo, h)) * h - wo);
  }
  const float p = disney_pdf(L, wi, wo, n);
  if (!(p > 0.f)) return false;
  weight = (1.f / p) * (disney_f_diffuse(m, L, wi, wo, n) + disney_f_glossy(m, L, wi, wo, n));
  return true;
}

// Whether a material's base is glossier than `min_rough` (GGX alpha, or the Disney specular's
// alpha = max(1e-3, roughness^2), below it).
__device__ __forceinline__ bool guide_smooth(const Material& m, float min_rough) {
  if (m.type == kMatGGX) return m.alpha < min_rough;
  if (m.type == kMatDisney) return fmaxf(1e-3f, m.dis[4] * m.dis[4]) < min_rough;
  return false;
}

__device__ __forceinline__ float3 base_f(const Material& m, float3 wi, float3 wo, float3 n) {
  return m.type == kMatGGX ? ggx_f(m.albedo, m.alpha, wi, wo, n) : lambert_f(m.albedo, wi, wo, n);
}

__device__ __forceinline__ bool sggx_isotropic(const float S[6]) {
  return S[0] == S[1] && S[1] == S[2] && S[3] == 0.f && S[4] == 0.f && S[5] == 0.f && S[0] > 0.f;
}

// Improved stochastic evaluation of Eq. 12 (Sec. 6): one VNDF sample and one "reversed" base
// sample (around the half vector for GGX, the cosine lobe about wi for Lambertian), combined
// with the one-sample balance heuristic.  U holds six uniforms.
__device__ inline float3 phase_eval_stochastic(const Material& m, float3 wi, float3 wo, const float U[6]) {
  const float3 n1 = sggx_sample_vndf(m.S, wo, U[0], U[1]);
  const float p1 = sggx_dvis(m.S, wo, n1);
  if (m.type == kMatDisney) {
    // each part with its own pair of techniques: the glossy part with micro-normals about the half
    // vector, the diffuse part with normals from the cosine lobe about wi
    const DisneyLobes L = disney_lobes(m);
    const float3 h = normalize3(wi + wo);
    const float3 n2 = micro_sample(L.alpha, h, U[2], U[3]);
    const float q2 = micro_pdf(L.alpha, n2, h);
    float3 est = mis_w(p1, micro_pdf(L.alpha, n1, h)) * disney_f_glossy(m, L, wi, wo, n1);
    if (q2 > 0.f) {
      const float dv = sggx_dvis(m.S, wo, n2);
      est = est + (dv / q2 * mis_w(q2, dv)) * disney_f_glossy(m, L, wi, wo, n2);
    }
    const float3 n3 = cos_sample(wi, U[4], U[5]);
    const float q3 = fmaxf(0.f, dot3(n3, wi)) / kPiF;
    est = est + mis_w(p1, fmaxf(0.f, dot3(n1, wi)) / kPiF) * disney_f_diffuse(m, L, wi, wo, n1);
    if (q3 > 0.f) {
      const float dv = sggx_dvis(m.S, wo, n3);
      est = est + (dv / q3 * mis_w(q3, dv)) * disney_f_diffuse(m, L, wi, wo, n3);
    }
    return est;
  }
  if (m.type == kMatGGX) {
    const float3 h = normalize3(wi + wo);
    const float3 n2 = micro_sample(m.alpha, h, U[2], U[3]);
    const float q2 = micro_pdf(m.alpha, n2, h);
    float3 est = mis_w(p1, micro_pdf(m.alpha, n1, h)) * base_f(m, wi, wo, n1);
    if (q2 > 0.f) {
      const float dv = sggx_dvis(m.S, wo, n2);
      est = est + (dv / q2 * mis_w(q2, dv)) * base_f(m, wi, wo, n2);
    }
    return est;
  }
  const float3 n3 = cos_sample(wi, U[4], U[5]);
  const float q3 = fmaxf(0.f, dot3(n3, wi)) / kPiF;
  float3 est = mis_w(p1, fmaxf(0.f, dot3(n1, wi)) / kPiF) * base_f(m, wi, wo, n1);
  if (q3 > 0.f) {
    const float dv = sggx_dvis(m.S, wo, n3);
    est = est + (dv / q3 * mis_w(q3, dv)) * base_f(m, wi, wo, n3);
  }
  return est;
}

// Isotropic flakes with a Lambertian base: rho * 2 / (3 pi^2) [(pi - g) cos g + sin g].
__device__ __forceinline__ float3 phase_eval_lambert_sphere(float3 rho, float3 wi, float3 wo) {
  const float c = fminf(1.f, fmaxf(-1.f, dot3(wi, wo)));
  const float g = acosf(c);
  const float v = 2.f / (3.f * kPiF * kPiF) * ((kPiF - g) * c + sqrtf(fmaxf(0.f, 1.f - c * c)));
  return v * rho;
}

// The three entry points the shading kernels call (evaluation, sampling, App. B pdf) are not
// inlined: every kernel that shades (the renderer's and the batch server's) then runs the same
// compiled arithmetic, so a path gets the same value in both, bit for bit.
static __device__ __noinline__ float3 phase_eval(const Material& m, float3 wi, float3 wo, const float U[6]) {
  if (m.type == kMatDiffuse && sggx_isotropic(m.S)) return phase_eval_lambert_sphere(m.albedo, wi, wo);
  return phase_eval_stochastic(m, wi, wo, U);
}

// Importance sampling (Sec. 6): n from the VNDF, wi from the base BSDF about n; the weight is
// the base BSDF's own f / pdf.  Returns false if the sample carries no weight.
static __device__ __noinline__ bool phase_sample(const Material& m, float3 wo, const float U[4], float3& wi,
                                                 float3& weight) {
  const float3 n = sggx_sample_vndf(m.S, wo, U[0], U[1]);
  if (m.type == kMatDisney) return disney_sample(m, wo, n, U + 2, wi, weight);
  if (m.type == kMatGGX) {
    const float3 h = ggx_sample_vn(m.alpha, wo, n, U[2], U[3]);
    const float oh = dot3(wo, h);
    wi = normalize3((2.f * oh) * h - wo);
    const float ci = dot3(n, wi), co = dot3(n, wo);
    if (ci <= 0.f || co <= 0.f || oh <= 0.f) return false;
    const float Lo = ggx_lambda(m.alpha, co), Li = ggx_lambda(m.alpha, ci);
    weight = ((1.f + Lo) / (1.f + Lo + Li)) * schlick(m.albedo, oh);
    return true;
  }
  wi = cos_sample(n, U[2], U[3]);
  weight = m.albedo;
  return true;
}

// Approximate phase pdf of App. B, taken as written: D~_wo(w_h) with the roughened SGGX for a
// GGX base, <w_h.wo> / pi for a Lambertian base, w_h = normalize(wi + wo).
static __device__ __noinline__ float phase_pdf_approx(const Material& m, float3 wi, float3 wo) {
  const float3 s = wi + wo;
  const float l2 = dot3(s, s);
  if (l2 <= 1e-24f) return 0.f;
  const float3 h = rsqrtf(l2) * s;
  if (m.type == kMatGGX) {
    float r[6];
    sggx_roughen(m.S, m.alpha, r);
    return sggx_dvis(r, wo, h);
  }
  if (m.type == kMatDisney) {
    // the lobes weighted as the sampler picks them (by metallic and base-colour luminance)
    const DisneyLobes L = disney_lobes(m);
    float r[6];
    sggx_roughen(m.S, L.alpha, r);
    float p = fmaf(L.p_spec, sggx_dvis(r, wo, h), L.p_diffuse * fmaxf(0.f, dot3(h, wo)) / kPiF);
    if (L.p_coat > 0.f) {
      sggx_roughen(m.S, L.alpha_c, r);
      p = fmaf(L.p_coat, sggx_dvis(r, wo, h), p);
    }
    return p;
  }
  return fmaxf(0.f, dot3(h, wo)) / kPiF;
}

}  // namespace ugp
