// The learned directional proposal ("guide") of the FP64 oracle: a small MLP that maps a
// scattering vertex (position, outgoing direction) to a mixture of von Mises-Fisher lobes,
// trained by the radiance-weighted log-likelihood and combined with phase sampling by
// one-sample MIS (Sec. 6 "Importance Sampling": any sampling technique combined with the
// approximate phase pdf of App. B stays unbiased).
//
// TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).
//
// The paper fixes none of the network's details; the readings used here are:
//  * input: position normalised to [0,1]^3 over a box (pos_lo, pos_hi), encoded by
//    sin/cos(2^l pi x) for l = 0..5 (36 features); the outgoing direction's polar angles
//    (theta, phi) in radians encoded by sin/cos(2^l angle) for l = 0..3 (16 features); then the
//    raw values (x, y, z, theta / pi, phi / (2 pi) + 1/2) (5 features); zero-padded to 64;
//  * four 64 x 64 layers with ReLU, then a 64 -> 40 head, biases everywhere;
//  * head: 8 lobes of (m (3), s, a): mu = m / |m|, kappa = min(kappa_max, kappa_min +
//    softplus(s)), mixture weight pi = softmax(a);
//  * the GPU computes the layers with BF16 operands and FP32 accumulation; the oracle mirrors
//    this by rounding every weight matrix and every layer input to BF16 (round to nearest
//    even) and accumulating in FP64 (round_bf16 = 0 turns the rounding off, for derivative
//    checks);
//  * loss of one logged vertex with incident-radiance estimate L and sampling pdf p:
//    -(L / p) log q(wi); the gradient is that of the batch mean; Adam updates the FP32
//    master weights.
#pragma once
#include "oracle_internal.h"

namespace orc {

constexpr int kGLobes = 8;
constexpr int kGWidth = 64;
constexpr int kGOut = 5 * kGLobes;  // 40
constexpr int kGLayers = 4;         // hidden 64 x 64 layers before the head
// Flat parameter vector: for l = 0..3, W_l (64 x 64, row-major [out][in]) then b_l (64);
// then the head W_4 (40 x 64) and b_4 (40).
constexpr int64_t kGNParams = kGLayers * (kGWidth * kGWidth + kGWidth) + kGOut * kGWidth + kGOut;

inline int64_t guide_w_offset(int l) { return int64_t(l) * (kGWidth * kGWidth + kGWidth); }
inline int64_t guide_b_offset(int l) {
  return guide_w_offset(l) + int64_t(l < kGLayers ? kGWidth : kGOut) * kGWidth;
}

struct GuideCfg {
  double pos_lo[3], pos_hi[3];
  double kappa_min, kappa_max;
  int32_t round_bf16;
};

double bf16_round(double x);

// The 64 input features of a vertex (before rounding).
void guide_encode(const GuideCfg& c, V3 x, V3 wo, double f[kGWidth]);

// Forward pass; fills Y (the 40 head outputs). When acts is not NULL it receives, per layer
// l = 0..4, the layer's input X_l (rounded as the forward used it) and, for l = 0..3, its
// pre-activation Z_l: acts[0 .. 5*64) = X_0..X_4, acts[5*64 .. 9*64) = Z_0..Z_3.
void guide_forward(const GuideCfg& c, const float* params, V3 x, V3 wo, double Y[kGOut], double* acts);

struct Mixture {
  V3 mu[kGLobes];
  double kappa[kGLobes];
  double pi[kGLobes];
};
Mixture guide_mixture(const GuideCfg& c, const double Y[kGOut]);

// vMF lobe density on the unit sphere: kappa / (2 pi (1 - e^{-2 kappa})) e^{kappa (mu.w - 1)}.
double vmf_pdf(V3 mu, double kappa, V3 w);
double mixture_pdf(const Mixture& m, V3 w);
// Direction from uniforms U = (lobe choice, u1, u2); inversion of the vMF's cosine CDF.
V3 mixture_sample(const Mixture& m, const double U[3]);

// Loss -(w) log q(wi) of one sample and its gradient with respect to the 40 head outputs.
double mixture_loss_grad(const GuideCfg& c, const double Y[kGOut], V3 wi, double w, double dY[kGOut]);

// Mean loss over n samples and the gradient of the mean (kGNParams entries, accumulated
// into grad after zeroing).
double guide_loss_grad(const GuideCfg& c, const float* params, int64_t n, const float* x3, const float* wo3,
                       const float* wi3, const float* weight, double* grad);

// One Adam step (t = step number after the update, starting at 1) on n parameters.
void adam_step(int64_t n, double* theta, double* m, double* v, const double* g, int64_t t, double lr, double b1,
               double b2, double eps);

}  // namespace orc
