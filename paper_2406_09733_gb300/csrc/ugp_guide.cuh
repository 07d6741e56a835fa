// Learned directional guide: input encoding and vMF-mixture arithmetic shared by the guide
// kernels and the renderer.
//
// The network maps a scattering vertex (position x, outgoing direction wo) to 8 von
// Mises-Fisher lobes over incident directions. The paper leaves the proposal open (Sec. 6: any
// sampling technique combined by MIS with the approximate phase pdf of App. B keeps the
// estimate unbiased); the readings of its unspecified details are:
//  * input: x normalised to [0,1]^3 over a box, sin/cos(2^l pi x) for l = 0..5 (36 features);
//    the polar angles (theta, phi) of wo in radians, sin/cos(2^l angle) for l = 0..3 (16);
//    the raw values (x, y, z, theta / pi, phi / (2 pi) + 1/2) (5); zeros up to 64;
//  * four 64 x 64 ReLU layers and a 64 -> 40 head, BF16 operands, FP32 accumulation;
//  * lobe j reads head outputs 5j..5j+4 = (m (3), s, a): mu = m / |m|,
//    kappa = min(kappa_max, kappa_min + softplus(s)), pi = softmax(a);
//  * vMF density kappa / (2 pi (1 - e^{-2 kappa})) e^{kappa (mu.w - 1)};
//  * sampling: lobe by the first cumulative pi above u_l, then 1 - mu.w =
//    -ln(v + (1 - v) e^{-2 kappa}) / kappa with v = 1 - u1, azimuth 2 pi u2 in the frame of mu;
//  * loss of a logged vertex: -(L / p) ln q(wi), L the incident-radiance estimate and p the
//    pdf the direction was sampled with.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "ugp_internal.cuh"
#include "ugp_phase.cuh"

namespace ugp {

constexpr int kGLobes = UGP_GUIDE_LOBES;
constexpr int kGWidth = UGP_GUIDE_WIDTH;
constexpr int kGOut = UGP_GUIDE_OUT;
constexpr int kGLayers = 4;

// Offsets of the flat FP32 parameter vector: for l = 0..3, W_l (64 x 64, [out][in]) then b_l;
// then the head W_4 (40 x 64) and b_4 (40).
__host__ __device__ constexpr int guide_w_off(int l) { return l * (kGWidth * kGWidth + kGWidth); }
__host__ __device__ constexpr int guide_out_dim(int l) { return l < kGLayers ? kGWidth : kGOut; }
__host__ __device__ constexpr int guide_b_off(int l) { return guide_w_off(l) + guide_out_dim(l) * kGWidth; }
static_assert(guide_b_off(kGLayers) + kGOut == UGP_GUIDE_NPARAMS, "guide parameter count");

// Shared-memory image of the network (the guide kernels bulk-copy it from the workspace):
//   [0, 40960)       W_l for l = 0..4, 64 x 64 tiles (rows = outputs, head padded with zero rows),
//                    the K-major B operand of X W_l^T and the MN-major B operand of dZ W_l
//   [40960, 42240)   biases, FP32, 64 per layer (head padded with zeros)
constexpr uint32_t kImgW = 0;
constexpr uint32_t kImgTile = kGWidth * kGWidth * 2;  // 8192
constexpr uint32_t kImgBias = 5 * kImgTile;           // 40960
constexpr uint32_t kImgBytes = kImgBias + 5 * kGWidth * 4;  // 42240

struct GuideCfgDev {
  float3 lo, inv_ext;  // position box: xn = (x - lo) * inv_ext
  float kappa_min, kappa_max;
};

__device__ __forceinline__ float clamp01(float v) { return fminf(1.f, fmaxf(0.f, v)); }

// The 64 input features of a vertex.
__device__ __forceinline__ void guide_encode(const GuideCfgDev& c, float3 x, float3 wo, float f[kGWidth]) {
  const float xn[3] = {clamp01((x.x - c.lo.x) * c.inv_ext.x), clamp01((x.y - c.lo.y) * c.inv_ext.y),
                       clamp01((x.z - c.lo.z) * c.inv_ext.z)};
  const float theta = acosf(fminf(1.f, fmaxf(-1.f, wo.z)));
  const float phi = atan2f(wo.y, wo.x);
  // the higher frequencies by double angles: sin 2a = 2 sin a cos a, cos 2a = (cos a - sin a)
  // (cos a + sin a); five doublings leave an error of a few 1e-6, far below the BF16 step the
  // layer input is rounded to
  int i = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float s, co;
    sincospif(xn[a], &s, &co);
#pragma unroll
    for (int l = 0; l < 6; ++l) {
      f[i++] = s;
      f[i++] = co;
      const float s2 = 2.f * s * co;
      co = (co - s) * (co + s);
      s = s2;
    }
  }
  const float ang[2] = {theta, phi};
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    float s, co;
    sincosf(ang[a], &s, &co);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      f[i++] = s;
      f[i++] = co;
      const float s2 = 2.f * s * co;
      co = (co - s) * (co + s);
      s = s2;
    }
  }
  f[i++] = xn[0];
  f[i++] = xn[1];
  f[i++] = xn[2];
  f[i++] = theta * 0.318309886183790672f;         // theta / pi
  f[i++] = phi * 0.159154943091895336f + 0.5f;    // phi / (2 pi) + 1/2
#pragma unroll
  for (; i < kGWidth;) f[i++] = 0.f;
}

__device__ __forceinline__ float softplusf(float s) { return fmaxf(s, 0.f) + log1pf(expf(-fabsf(s))); }

// log of the vMF normaliser kappa / (2 pi (1 - e^{-2 kappa})).
__device__ __forceinline__ float vmf_log_norm(float k) {
  return logf(k) - 1.83787706640934548f - logf(-expm1f(-2.f * k));
}

// Mixture (per lobe mu (3), kappa, pi) from the 40 head outputs.
__device__ __forceinline__ void mixture_from_head(const GuideCfgDev& c, const float Y[kGOut], float mix[kGOut]) {
  float amax = -3.4e38f;
#pragma unroll
  for (int j = 0; j < kGLobes; ++j) amax = fmaxf(amax, Y[5 * j + 4]);
  float z = 0.f;
#pragma unroll
  for (int j = 0; j < kGLobes; ++j) z += expf(Y[5 * j + 4] - amax);
  const float iz = 1.f / z;
#pragma unroll
  for (int j = 0; j < kGLobes; ++j) {
    const float mx = Y[5 * j], my = Y[5 * j + 1], mz = Y[5 * j + 2];
    const float n = sqrtf(mx * mx + my * my + mz * mz);
    const float in = n > 0.f ? 1.f / n : 0.f;
    mix[5 * j] = n > 0.f ? mx * in : 0.f;
    mix[5 * j + 1] = n > 0.f ? my * in : 0.f;
    mix[5 * j + 2] = n > 0.f ? mz * in : 1.f;
    mix[5 * j + 3] = fminf(c.kappa_max, c.kappa_min + softplusf(Y[5 * j + 3]));
    mix[5 * j + 4] = expf(Y[5 * j + 4] - amax) * iz;
  }
}

__device__ __forceinline__ float mixture_pdf(const float mix[kGOut], float3 w) {
  float q = 0.f;
#pragma unroll
  for (int j = 0; j < kGLobes; ++j) {
    const float k = mix[5 * j + 3];
    const float c = mix[5 * j] * w.x + mix[5 * j + 1] * w.y + mix[5 * j + 2] * w.z;
    q += mix[5 * j + 4] * expf(vmf_log_norm(k) + k * (c - 1.f));
  }
  return q;
}

__device__ __forceinline__ float3 mixture_sample(const float mix[kGOut], float ul, float u1, float u2) {
  // first lobe whose cumulative weight exceeds ul (the last one if rounding leaves none);
  // selected by predicated moves so the mixture stays in registers
  bool found = false;
  float cum = 0.f;
  float3 mu = f3(mix[5 * (kGLobes - 1)], mix[5 * (kGLobes - 1) + 1], mix[5 * (kGLobes - 1) + 2]);
  float k = mix[5 * (kGLobes - 1) + 3];
#pragma unroll
  for (int i = 0; i < kGLobes; ++i) {
    cum += mix[5 * i + 4];
    const bool take = !found && cum > ul;
    if (take) {
      mu = f3(mix[5 * i], mix[5 * i + 1], mix[5 * i + 2]);
      k = mix[5 * i + 3];
    }
    found = found || take;
  }
  const float v = 1.f - u1;
  const float omw = fminf(2.f, -logf(v + (1.f - v) * expf(-2.f * k)) / k);
  const float s = sqrtf(fmaxf(0.f, omw * (2.f - omw)));
  float sp, cp;
  sincospif(2.f * u2, &sp, &cp);
  float3 t, b;
  onb3(mu, t, b);
  return normalize3((1.f - omw) * mu + (s * cp) * t + (s * sp) * b);
}

// Loss -w ln q(wi) of one sample and its gradient with respect to the 40 head outputs.
__device__ __forceinline__ float mixture_loss_grad(const GuideCfgDev& c, const float Y[kGOut], float3 wi, float w,
                                                   float dY[kGOut]) {
  float amax = -3.4e38f;
#pragma unroll
  for (int j = 0; j < kGLobes; ++j) amax = fmaxf(amax, Y[5 * j + 4]);
  float z = 0.f;
#pragma unroll
  for (int j = 0; j < kGLobes; ++j) z += expf(Y[5 * j + 4] - amax);
  const float logz = amax + logf(z);
  float ell[kGLobes];
  float lmax = -3.4e38f;
#pragma unroll
  for (int j = 0; j < kGLobes; ++j) {
    const float mx = Y[5 * j], my = Y[5 * j + 1], mz = Y[5 * j + 2];
    const float n = sqrtf(mx * mx + my * my + mz * mz);
    const float in = n > 0.f ? 1.f / n : 0.f;
    const float cw = n > 0.f ? (mx * wi.x + my * wi.y + mz * wi.z) * in : wi.z;
    const float kr = c.kappa_min + softplusf(Y[5 * j + 3]);
    const float k = fminf(kr, c.kappa_max);
    ell[j] = (Y[5 * j + 4] - logz) + vmf_log_norm(k) + k * (cw - 1.f);
    lmax = fmaxf(lmax, ell[j]);
    // stash what the second pass needs in dY
    dY[5 * j] = cw;
    dY[5 * j + 1] = in;
    dY[5 * j + 2] = k;
    dY[5 * j + 3] = kr > c.kappa_max ? 0.f : 1.f;
  }
  float sq = 0.f;
#pragma unroll
  for (int j = 0; j < kGLobes; ++j) sq += expf(ell[j] - lmax);
  const float logq = lmax + logf(sq);
#pragma unroll
  for (int j = 0; j < kGLobes; ++j) {
    const float cw = dY[5 * j], in = dY[5 * j + 1], k = dY[5 * j + 2], free_k = dY[5 * j + 3];
    const float r = expf(ell[j] - logq);
    const float pi = expf(Y[5 * j + 4] - logz);
    dY[5 * j + 4] = w * (pi - r);
    const float dlk = 1.f / k - 2.f / expm1f(2.f * k) + (cw - 1.f);
    const float sig = 1.f / (1.f + expf(-Y[5 * j + 3]));
    dY[5 * j + 3] = free_k * (-w * r * dlk * sig);
    const float g = -w * r * k * in;
    const float mx = Y[5 * j] * in, my = Y[5 * j + 1] * in, mz = Y[5 * j + 2] * in;
    dY[5 * j] = g * (wi.x - cw * mx);
    dY[5 * j + 1] = g * (wi.y - cw * my);
    dY[5 * j + 2] = g * (wi.z - cw * mz);
  }
  return -w * logq;
}

}  // namespace ugp
