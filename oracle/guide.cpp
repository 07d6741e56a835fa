// FP64 oracle: the learned vMF-mixture guide (forward, mixture density and sampling, analytic
// backward, Adam). The readings of the unspecified network details are listed in
// oracle_guide.h.
//
// TEST INFRASTRUCTURE ONLY.
#include <algorithm>
#include <cfenv>
#include <cmath>
#include <cstring>

#include "oracle_guide.h"
#include "oracle_phase.h"

namespace orc {

static const double kPi = 3.14159265358979323846;

// Round to the nearest bfloat16 (8 significant bits), ties to even. Zero, infinities and NaN
// pass through.
double bf16_round(double x) {
  if (x == 0.0 || !std::isfinite(x)) return x;
  int e = 0;
  const double m = std::frexp(x, &e);  // |m| in [0.5, 1)
  double s = std::ldexp(m, 8);         // 8 significant bits before the point
  const double fl = std::floor(s);
  const double rem = s - fl;
  if (rem > 0.5 || (rem == 0.5 && std::fmod(fl, 2.0) != 0.0)) s = fl + 1.0;
  else s = fl;
  return std::ldexp(s, e - 8);
}

void guide_encode(const GuideCfg& c, V3 x, V3 wo, double f[kGWidth]) {
  const double p[3] = {x.x, x.y, x.z};
  double xn[3];
  for (int a = 0; a < 3; ++a) {
    const double ext = c.pos_hi[a] - c.pos_lo[a];
    double t = ext > 0 ? (p[a] - c.pos_lo[a]) / ext : 0.0;
    xn[a] = std::min(1.0, std::max(0.0, t));
  }
  const double theta = std::acos(std::min(1.0, std::max(-1.0, wo.z)));
  const double phi = std::atan2(wo.y, wo.x);
  int i = 0;
  for (int a = 0; a < 3; ++a)
    for (int l = 0; l < 6; ++l) {
      const double arg = std::ldexp(kPi, l) * xn[a];
      f[i++] = std::sin(arg);
      f[i++] = std::cos(arg);
    }
  const double ang[2] = {theta, phi};
  for (int a = 0; a < 2; ++a)
    for (int l = 0; l < 4; ++l) {
      const double arg = std::ldexp(ang[a], l);
      f[i++] = std::sin(arg);
      f[i++] = std::cos(arg);
    }
  f[i++] = xn[0];
  f[i++] = xn[1];
  f[i++] = xn[2];
  f[i++] = theta / kPi;
  f[i++] = phi / (2 * kPi) + 0.5;
  while (i < kGWidth) f[i++] = 0.0;
}

static inline double rnd(const GuideCfg& c, double v) { return c.round_bf16 ? bf16_round(v) : v; }

void guide_forward(const GuideCfg& c, const float* params, V3 x, V3 wo, double Y[kGOut], double* acts) {
  double X[kGWidth], Z[kGWidth];
  guide_encode(c, x, wo, X);
  for (int j = 0; j < kGWidth; ++j) X[j] = rnd(c, X[j]);
  for (int l = 0; l <= kGLayers; ++l) {
    const int out = l < kGLayers ? kGWidth : kGOut;
    const float* W = params + guide_w_offset(l);
    const float* b = params + guide_b_offset(l);
    if (acts) std::memcpy(acts + l * kGWidth, X, sizeof(X));
    for (int o = 0; o < out; ++o) {
      double s = b[o];
      for (int i = 0; i < kGWidth; ++i) s += rnd(c, double(W[o * kGWidth + i])) * X[i];
      Z[o] = s;
    }
    if (l < kGLayers) {
      if (acts) std::memcpy(acts + (5 + l) * kGWidth, Z, sizeof(Z));
      for (int o = 0; o < kGWidth; ++o) X[o] = rnd(c, Z[o] > 0 ? Z[o] : 0.0);
    } else {
      for (int o = 0; o < kGOut; ++o) Y[o] = Z[o];
    }
  }
}

static double softplus(double s) { return std::max(s, 0.0) + std::log1p(std::exp(-std::fabs(s))); }

Mixture guide_mixture(const GuideCfg& c, const double Y[kGOut]) {
  Mixture m;
  double amax = -1e300;
  for (int j = 0; j < kGLobes; ++j) amax = std::max(amax, Y[5 * j + 4]);
  double z = 0;
  for (int j = 0; j < kGLobes; ++j) z += std::exp(Y[5 * j + 4] - amax);
  for (int j = 0; j < kGLobes; ++j) {
    const V3 v = v3(Y[5 * j], Y[5 * j + 1], Y[5 * j + 2]);
    const double n = length(v);
    m.mu[j] = n > 0 ? (1.0 / n) * v : v3(0, 0, 1);
    m.kappa[j] = std::min(c.kappa_max, c.kappa_min + softplus(Y[5 * j + 3]));
    m.pi[j] = std::exp(Y[5 * j + 4] - amax) / z;
  }
  return m;
}

// log of the vMF normaliser kappa / (2 pi (1 - e^{-2 kappa})).
static double vmf_log_norm(double kappa) { return std::log(kappa) - std::log(2 * kPi) - std::log(-std::expm1(-2 * kappa)); }

double vmf_pdf(V3 mu, double kappa, V3 w) { return std::exp(vmf_log_norm(kappa) + kappa * (dot(mu, w) - 1.0)); }

double mixture_pdf(const Mixture& m, V3 w) {
  double q = 0;
  for (int j = 0; j < kGLobes; ++j) q += m.pi[j] * vmf_pdf(m.mu[j], m.kappa[j], w);
  return q;
}

V3 mixture_sample(const Mixture& m, const double U[3]) {
  int j = kGLobes - 1;
  double cum = 0;
  for (int i = 0; i < kGLobes; ++i) {
    cum += m.pi[i];
    if (cum > U[0]) {
      j = i;
      break;
    }
  }
  const double k = m.kappa[j];
  // Cosine to the lobe axis: the CDF of w = mu.wi is (e^{k(w-1)} - e^{-2k}) / (1 - e^{-2k}); with
  // v = 1 - u1 in (0, 1], 1 - w = -ln(v + (1 - v) e^{-2k}) / k.
  const double v = 1.0 - U[1];
  const double omw = std::min(2.0, -std::log(v + (1.0 - v) * std::exp(-2 * k)) / k);
  const double w = 1.0 - omw;
  const double s = std::sqrt(std::max(0.0, omw * (2.0 - omw)));
  const double ph = 2 * kPi * U[2];
  V3 t, b;
  onb(m.mu[j], &t, &b);
  return normalize(w * m.mu[j] + (s * std::cos(ph)) * t + (s * std::sin(ph)) * b);
}

double mixture_loss_grad(const GuideCfg& c, const double Y[kGOut], V3 wi, double w, double dY[kGOut]) {
  double amax = -1e300;
  for (int j = 0; j < kGLobes; ++j) amax = std::max(amax, Y[5 * j + 4]);
  double z = 0;
  for (int j = 0; j < kGLobes; ++j) z += std::exp(Y[5 * j + 4] - amax);
  const double logz = amax + std::log(z);
  double ell[kGLobes], kap[kGLobes], dlk[kGLobes], nrm[kGLobes], cosw[kGLobes], pi[kGLobes];
  V3 mu[kGLobes];
  bool clamped[kGLobes];
  double lmax = -1e300;
  for (int j = 0; j < kGLobes; ++j) {
    const V3 mv = v3(Y[5 * j], Y[5 * j + 1], Y[5 * j + 2]);
    nrm[j] = length(mv);
    mu[j] = nrm[j] > 0 ? (1.0 / nrm[j]) * mv : v3(0, 0, 1);
    const double kr = c.kappa_min + softplus(Y[5 * j + 3]);
    clamped[j] = kr > c.kappa_max;
    kap[j] = clamped[j] ? c.kappa_max : kr;
    cosw[j] = dot(mu[j], wi);
    const double logpi = Y[5 * j + 4] - logz;
    pi[j] = std::exp(logpi);
    ell[j] = logpi + vmf_log_norm(kap[j]) + kap[j] * (cosw[j] - 1.0);
    // d log v / d kappa = 1/kappa - 2 / (e^{2 kappa} - 1) + (mu.wi - 1)
    dlk[j] = 1.0 / kap[j] - 2.0 / std::expm1(2 * kap[j]) + (cosw[j] - 1.0);
    lmax = std::max(lmax, ell[j]);
  }
  double sq = 0;
  for (int j = 0; j < kGLobes; ++j) sq += std::exp(ell[j] - lmax);
  const double logq = lmax + std::log(sq);
  for (int j = 0; j < kGLobes; ++j) {
    const double r = std::exp(ell[j] - logq);  // responsibility of lobe j
    dY[5 * j + 4] = w * (pi[j] - r);
    const double sig = 1.0 / (1.0 + std::exp(-Y[5 * j + 3]));
    dY[5 * j + 3] = clamped[j] ? 0.0 : -w * r * dlk[j] * sig;
    if (nrm[j] > 0) {
      const V3 g = (-w * r * kap[j] / nrm[j]) * (wi - cosw[j] * mu[j]);
      dY[5 * j] = g.x;
      dY[5 * j + 1] = g.y;
      dY[5 * j + 2] = g.z;
    } else {
      dY[5 * j] = dY[5 * j + 1] = dY[5 * j + 2] = 0.0;
    }
  }
  return -w * logq;
}

double guide_loss_grad(const GuideCfg& c, const float* params, int64_t n, const float* x3, const float* wo3,
                       const float* wi3, const float* weight, double* grad) {
  std::fill(grad, grad + kGNParams, 0.0);
  if (n <= 0) return 0.0;
  const double inv = 1.0 / double(n);
  double loss = 0;
  std::vector<double> acts(9 * kGWidth);
  for (int64_t s = 0; s < n; ++s) {
    double Y[kGOut], dY[kGOut];
    guide_forward(c, params, load3(x3 + 3 * s), load3(wo3 + 3 * s), Y, acts.data());
    loss += mixture_loss_grad(c, Y, load3(wi3 + 3 * s), double(weight[s]), dY);
    // Backward through the head and the hidden layers (chain rule, BF16 rounding treated as
    // the identity, as the GPU's straight-through use of rounded activations).
    double dZ[kGWidth], dX[kGWidth];
    int out = kGOut;
    for (int o = 0; o < kGOut; ++o) dZ[o] = dY[o] * inv;
    for (int l = kGLayers; l >= 0; --l) {
      const float* W = params + guide_w_offset(l);
      double* gW = grad + guide_w_offset(l);
      double* gb = grad + guide_b_offset(l);
      const double* X = acts.data() + l * kGWidth;
      for (int o = 0; o < out; ++o) {
        gb[o] += dZ[o];
        for (int i = 0; i < kGWidth; ++i) gW[o * kGWidth + i] += dZ[o] * X[i];
      }
      if (l == 0) break;
      for (int i = 0; i < kGWidth; ++i) {
        double s2 = 0;
        for (int o = 0; o < out; ++o) s2 += rnd(c, double(W[o * kGWidth + i])) * dZ[o];
        dX[i] = s2;
      }
      const double* Zp = acts.data() + (5 + l - 1) * kGWidth;  // pre-activation of layer l-1
      for (int i = 0; i < kGWidth; ++i) dZ[i] = Zp[i] > 0 ? dX[i] : 0.0;
      out = kGWidth;
    }
  }
  return loss * inv;
}

void adam_step(int64_t n, double* theta, double* m, double* v, const double* g, int64_t t, double lr, double b1,
               double b2, double eps) {
  const double c1 = 1.0 - std::pow(b1, double(t)), c2 = 1.0 - std::pow(b2, double(t));
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1 - b1) * g[i];
    v[i] = b2 * v[i] + (1 - b2) * g[i] * g[i];
    theta[i] -= lr * (m[i] / c1) / (std::sqrt(v[i] / c2) + eps);
  }
}

}  // namespace orc
