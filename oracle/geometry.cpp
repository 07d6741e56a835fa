// FP64 oracle: Gaussian primitives, the closed-form ray integral, transmittance
// and exact free-flight sampling, all by brute force over every primitive.
//
// TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline). Not linked into,
// and shares no code with, the CUDA library.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

#include "oracle_internal.h"

namespace orc {

static const double kPi = 3.14159265358979323846;

// Rotation matrix of a unit quaternion q = (w, x, y, z), row-major.
static void quat_to_R(const double q[4], double R[9]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// Eq. 1 and Eq. 2: Sigma = (RS)(RS)^T, so (RS)^-1 = S^-1 R^T and |Sigma|^{1/2} = s_x s_y s_z.
Prim make_prim(const float* mean3, const float* quat4, const float* scale3, float magnitude) {
  Prim p;
  p.mu = load3(mean3);
  double q[4] = {quat4[0], quat4[1], quat4[2], quat4[3]};
  const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (double& c : q) c /= qn;
  quat_to_R(q, p.R);
  for (int i = 0; i < 3; ++i) p.s[i] = scale3[i];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) p.W[3 * i + j] = p.R[3 * j + i] / p.s[i];  // (S^-1 R^T)_ij
  p.g0 = double(magnitude) / (std::pow(2 * kPi, 1.5) * p.s[0] * p.s[1] * p.s[2]);
  return p;
}

std::vector<Prim> make_prims(const SceneIn& s) {
  std::vector<Prim> out(size_t(s.n));
  for (int64_t i = 0; i < s.n; ++i)
    out[size_t(i)] = make_prim(s.mean3 + 3 * i, s.quat4 + 4 * i, s.scale3 + 3 * i, s.magnitude[i]);
  return out;
}

// Eq. 4: G / G(mu) = eps  <=>  ||(RS)^-1 (x - mu)|| = sqrt(-2 ln eps).
double cutoff_k(double eps) { return std::sqrt(-2.0 * std::log(eps)); }

static V3 mul(const double M[9], V3 v) {
  return {M[0] * v.x + M[1] * v.y + M[2] * v.z, M[3] * v.x + M[4] * v.y + M[5] * v.z,
          M[6] * v.x + M[7] * v.y + M[8] * v.z};
}

// App. A with the mean moved to the origin: (x_t)^T Sigma^-1 x_t = A t^2 + B t + C where
// A = w^T Sigma^-1 w, B = 2 w^T Sigma^-1 x, C = x^T Sigma^-1 x, and Sigma^-1 = W^T W.
// Completing the square (the form the appendix intends): A (t - t*)^2 + (C - B^2 / 4A).
void ray_prim_quadratic(const Prim& p, V3 o, V3 d, double* A, double* tstar, double* d2) {
  const V3 x = o - p.mu;
  const V3 wx = mul(p.W, x), wd = mul(p.W, d);
  const double a = dot(wd, wd), b = 2.0 * dot(wd, wx), c = dot(wx, wx);
  *A = a;
  *tstar = -b / (2.0 * a);
  *d2 = c - b * b / (4.0 * a);
}

bool ray_prim(const Prim& p, int32_t id, V3 o, V3 d, double t0, double t1, double k, Hit* h) {
  double A, tstar, d2;
  ray_prim_quadratic(p, o, d, &A, &tstar, &d2);
  const double k2 = k * k;
  if (!(d2 < k2)) return false;  // the line misses the bounding ellipsoid (Eq. 4)
  const double half = std::sqrt((k2 - d2) / A);
  const double a = std::max(t0, tstar - half), b = std::min(t1, tstar + half);
  if (!(a < b)) return false;
  h->id = id;
  h->a = a;
  h->b = b;
  h->A = A;
  h->tstar = tstar;
  h->d2 = d2;
  h->g0 = p.g0;
  return true;
}

// App. A: int_x^y G(x_t) dt = g0 exp(-d2/2) sqrt(pi / 2A) [erf(tau(y)) - erf(tau(x))],
// tau(t) = sqrt(A/2) t + B / (2 sqrt(2A)) = sqrt(A/2) (t - t*).
// When both arguments share a sign the difference is taken through erfc.
double ray_integral(const Hit& h, double x, double y) {
  const double s = std::sqrt(0.5 * h.A);
  const double ta = s * (x - h.tstar), tb = s * (y - h.tstar);
  double diff;
  if (ta >= 0.0)
    diff = std::erfc(ta) - std::erfc(tb);
  else if (tb <= 0.0)
    diff = std::erfc(-tb) - std::erfc(-ta);
  else
    diff = std::erf(tb) - std::erf(ta);
  return h.g0 * std::exp(-0.5 * h.d2) * std::sqrt(kPi / (2.0 * h.A)) * diff;
}

// Eq. 1 at x_t: (x_t - mu)^T Sigma^-1 (x_t - mu) = A (t - t*)^2 + d2.
double gauss_at(const Hit& h, double t) {
  const double dt = t - h.tstar;
  return h.g0 * std::exp(-0.5 * (h.d2 + h.A * dt * dt));
}

std::vector<Hit> all_hits(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1,
                          double k, int32_t exclude) {
  if (g_accel && g_accel->prims == &prims) return accel_hits(*g_accel, o, d, t0, t1, k, exclude);
  std::vector<Hit> hits;
  for (size_t i = 0; i < prims.size(); ++i) {
    if (int32_t(i) == exclude) continue;
    Hit h;
    if (ray_prim(prims[i], int32_t(i), o, d, t0, t1, k, &h)) hits.push_back(h);
  }
  return hits;
}

// Eq. 7: T(t0, t1) = max(0, 1 - 1/2 int sum_k G_k) with every contribution clipped to the
// primitive's bounding ellipsoid (Sec. 4.1). Order plays no role.
double transmittance(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1, double k,
                     int32_t exclude, double* tau_out) {
  double tau = 0.0;
  for (const Hit& h : all_hits(prims, o, d, t0, t1, k, exclude))
    tau += 0.5 * ray_integral(h, h.a, h.b);
  if (tau_out) *tau_out = tau;
  return std::max(0.0, 1.0 - tau);
}

// Exponential variate of primitive k in the race that picks the scattering primitive: Philox4x32-10
// with key (bits of u2, 0x2406C0DE) and counter (k, 0, 0, 0); U = (x0 >> 8 + 1) / 2^24 in (0, 1].
double race_exponential(double u2, int32_t k) {
  const float f = float(u2);
  uint32_t bits;
  std::memcpy(&bits, &f, 4);
  const uint32_t ctr[4] = {uint32_t(k), 0u, 0u, 0u};
  const uint32_t key[2] = {bits, 0x2406C0DEu};
  uint32_t x[4];
  philox4x32_10(ctr, key, x);
  const double U = double((x[0] >> 8) + 1u) * (1.0 / 16777216.0);
  return -std::log(U);
}

// erf^-1 by Newton's method on std::erf, started from a bisection bracket.
double erfinv(double y) {
  if (y <= -1.0) return -std::numeric_limits<double>::infinity();
  if (y >= 1.0) return std::numeric_limits<double>::infinity();
  double lo = -6.0, hi = 6.0, x = 0.0;
  for (int it = 0; it < 200; ++it) {
    const double f = std::erf(x) - y;
    if (f == 0.0) return x;
    if (f > 0) hi = x; else lo = x;
    const double fp = 2.0 / std::sqrt(kPi) * std::exp(-x * x);
    double xn = x - f / fp;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (std::fabs(xn - x) <= 1e-17 * std::max(1.0, std::fabs(x))) return xn;
    x = xn;
  }
  return x;
}

// Exact free-flight sampling (Sec. 5.2, Eq. 8, Eq. 10), in an order-free form:
//  1. The clipped intervals of all primitives cut [t0, t1] into segments on which the
//     set of active primitives is constant (the 1D form of the line sweep of Sec. 5.2).
//  2. F(t) = 1/2 sum_k I_k(a_k, min(t, b_k)) is accumulated segment by segment.
//  3. If F never exceeds u before t1 the ray escapes (probability max(0, 1 - F(t1)) = T).
//  4. Otherwise t_u with F(t_u) = u lies in the crossing segment and is found by a
//     bracketed Newton iteration with F' = 1/2 sum_active G_k (Eq. 9); with a single active
//     primitive the erf^-1 closed form is tried first.
//  5. The primitive is chosen among the primitives active at t_u with probability
//     G_k(x_{t_u}) / sum_active G_j(x_{t_u}) by an exponential race keyed by u2 (race_exponential).
//  Since u < 1, t_u lies before the saturating distance, so primitive k is returned with
//  probability 1/2 I_k(a_k, min(b_k, t_sat)).
FreeFlight sample_free_flight_hits(const std::vector<Hit>& hits, double t0, double t1, double u,
                                   double u2) {
  FreeFlight r{-1, 0.0, 0.0, 0.0, 0, std::numeric_limits<double>::infinity()};
  std::vector<double> ev;
  ev.reserve(2 * hits.size() + 2);
  for (const Hit& h : hits) {
    ev.push_back(h.a);
    ev.push_back(h.b);
  }
  std::sort(ev.begin(), ev.end());
  ev.erase(std::unique(ev.begin(), ev.end()), ev.end());

  double F = 0.0;
  for (const Hit& h : hits) r.F_end += 0.5 * ray_integral(h, h.a, h.b);
  std::vector<const Hit*> act;
  for (size_t j = 0; j + 1 < ev.size(); ++j) {
    const double s0 = ev[j], s1 = ev[j + 1];
    act.clear();
    for (const Hit& h : hits)
      if (h.a <= s0 && h.b >= s1) act.push_back(&h);
    if (act.empty()) continue;
    double dF = 0.0;
    for (const Hit* h : act) dF += 0.5 * ray_integral(*h, s0, s1);
    if (F + dF <= u) {
      F += dF;
      continue;
    }
    // Crossing segment: solve F(s0) + 1/2 sum I(s0, t) = u.
    auto Fm = [&](double t) {
      double v = F;
      for (const Hit* h : act) v += 0.5 * ray_integral(*h, s0, t);
      return v - u;
    };
    auto dFm = [&](double t) {
      double v = 0.0;
      for (const Hit* h : act) v += 0.5 * gauss_at(*h, t);
      return v;
    };
    double t = std::numeric_limits<double>::quiet_NaN();
    if (act.size() == 1) {
      // Single primitive: invert App. A with erf^-1 (Sec. 4.1, "Ray Sampling").
      const Hit& h = *act[0];
      const double s = std::sqrt(0.5 * h.A);
      const double amp = 0.5 * h.g0 * std::exp(-0.5 * h.d2) * std::sqrt(kPi / (2.0 * h.A));
      const double target = std::erf(s * (s0 - h.tstar)) + (u - F) / amp;
      const double tc = h.tstar + erfinv(target) / s;
      if (tc > s0 && tc < s1 && std::fabs(Fm(tc)) < 1e-12) t = tc;
    }
    if (!(t == t)) {
      double lo = s0, hi = s1;
      t = 0.5 * (lo + hi);
      for (int it = 0; it < 400; ++it) {
        const double f = Fm(t);
        if (f == 0.0) break;
        if (f < 0) lo = t; else hi = t;
        const double fp = dFm(t);
        double tn = (fp > 0) ? t - f / fp : 0.5 * (lo + hi);
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        if (std::fabs(tn - t) <= 1e-16 * std::max(1.0, std::fabs(t)) || hi - lo <= 1e-16 * std::max(1.0, std::fabs(t))) {
          t = tn;
          break;
        }
        t = tn;
      }
    }
    r.t_u = t;
    // Choose among the primitives active at t_u, proportionally to G_k(x_{t_u}), by an
    // exponential race: primitive k draws E_k = -ln U_k and the smallest E_k / G_k wins, which
    // happens with probability G_k / sum_j G_j whatever the order the candidates are seen in.
    const Hit* pick = nullptr;
    double best = std::numeric_limits<double>::infinity(), second = best;
    for (const Hit* h : act) {
      const double key = race_exponential(u2, h->id) / gauss_at(*h, t);
      if (key < best || (key == best && pick && h->id < pick->id)) {
        second = best;
        best = key;
        pick = h;
      } else if (key < second) {
        second = key;
      }
    }
    r.race_margin = act.size() > 1 ? (second - best) / best : std::numeric_limits<double>::infinity();
    r.prim = pick->id;
    r.t_spawn = 0.5 * (pick->a + pick->b);
    r.n_active = int32_t(act.size());
    return r;
  }
  r.prim = -1;
  r.t_u = t1;
  return r;
}

FreeFlight sample_free_flight(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1,
                              double k, int32_t exclude, double u, double u2) {
  return sample_free_flight_hits(all_hits(prims, o, d, t0, t1, k, exclude), t0, t1, u, u2);
}

// The paper's own disambiguation rule (Sec. 5.2, Eq. 10 and the free-flight listing), kept as a
// diagnostic of its bias; the sampler above is the parity target. Segments as above, primitives
// in ascending id within a segment (the traversal order of a leaf):
//  * a segment with one active primitive, or one that does not reach F = 1, accumulates
//    1/2 I_k over the whole segment primitive by primitive and returns the first primitive
//    whose running sum passes u;
//  * the segment in which F reaches 1 (the ambiguous one) solves F(t_u) = u and then picks
//    among its active primitives proportionally to I_k(s0, t_u), with the uniform
//    u_seg = F(s0) + u2 (u - F(s0)).
// Exact where the active primitives' densities keep constant ratios over that segment, biased
// otherwise (the pick should follow G_k at t_u).
int32_t sample_free_flight_paper_rule(const std::vector<Hit>& hits, double t0, double t1, double u, double u2) {
  (void)t0;
  (void)t1;
  std::vector<double> ev;
  for (const Hit& h : hits) {
    ev.push_back(h.a);
    ev.push_back(h.b);
  }
  std::sort(ev.begin(), ev.end());
  ev.erase(std::unique(ev.begin(), ev.end()), ev.end());
  double F = 0.0;
  std::vector<const Hit*> act;
  for (size_t j = 0; j + 1 < ev.size(); ++j) {
    const double s0 = ev[j], s1 = ev[j + 1];
    act.clear();
    for (const Hit& h : hits)
      if (h.a <= s0 && h.b >= s1) act.push_back(&h);
    if (act.empty()) continue;
    double dF = 0.0;
    for (const Hit* h : act) dF += 0.5 * ray_integral(*h, s0, s1);
    if (act.size() == 1 || F + dF < 1.0) {
      for (const Hit* h : act) {
        F += 0.5 * ray_integral(*h, s0, s1);
        if (u < F) return h->id;
      }
      continue;
    }
    // ambiguous segment: F reaches 1 inside it, so u < 1 <= F + dF
    double lo = s0, hi = s1, t = 0.5 * (s0 + s1);
    for (int it = 0; it < 400; ++it) {
      double f = F - u, fp = 0.0;
      for (const Hit* h : act) {
        f += 0.5 * ray_integral(*h, s0, t);
        fp += 0.5 * gauss_at(*h, t);
      }
      if (f == 0.0) break;
      if (f < 0) lo = t; else hi = t;
      double tn = fp > 0 ? t - f / fp : 0.5 * (lo + hi);
      if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
      if (std::fabs(tn - t) <= 1e-16 * std::max(1.0, std::fabs(t)) || hi - lo <= 1e-16 * std::max(1.0, std::fabs(t))) {
        t = tn;
        break;
      }
      t = tn;
    }
    const double u_seg = F + u2 * (u - F);
    for (const Hit* h : act) {
      F += 0.5 * ray_integral(*h, s0, t);
      if (u_seg < F) return h->id;
    }
    return act.back()->id;  // rounding: the running sum ends a hair below u
  }
  return -1;
}

// Sec. 7, Eq. rf. The saturating distance is where F reaches 1, i.e. the free-flight root for
// u = 1 (the paper's "u = 1" disambiguation); every primitive then counts with its probability
// mass up to t_sat, 1/2 I_k(a_k, min(b_k, t_sat)), which needs no disambiguation at all.
void radiance_field(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1, double k,
                    const float* emission3, const double* background3, double t_shift_ulps, double* rgb_out,
                    double* t_sat_out, double* F_end_out) {
  const std::vector<Hit> hits = all_hits(prims, o, d, t0, t1, k, -1);
  const FreeFlight f = sample_free_flight_hits(hits, t0, t1, 1.0, 0.0);
  const bool saturated = f.prim >= 0;
  double t_sat = saturated ? f.t_u : t1;
  if (saturated && t_shift_ulps != 0.0) {
    const float tf = float(t_sat);
    t_sat += t_shift_ulps * double(std::nextafter(tf, INFINITY) - tf);
  }
  double rgb[3] = {0.0, 0.0, 0.0}, mass = 0.0;
  for (const Hit& h : hits) {
    const double y = std::min(h.b, t_sat);
    if (!(h.a < y)) continue;
    const double w = 0.5 * ray_integral(h, h.a, y);
    mass += w;
    for (int c = 0; c < 3; ++c) rgb[c] += w * double(emission3[3 * size_t(h.id) + c]);
  }
  const double rest = saturated ? 0.0 : std::max(0.0, 1.0 - mass);
  for (int c = 0; c < 3; ++c) rgb_out[c] = rgb[c] + rest * (background3 ? background3[c] : 0.0);
  if (t_sat_out) *t_sat_out = t_sat;
  if (F_end_out) *F_end_out = f.F_end;
}

// Appendix "Sampling Exponential Transmittance Gaussians via Analog Decomposition Tracking".
// The same Gaussians read as an extinction coefficient sigma_t(x) = sum_k G_k(x) of the
// exponential model (Eq. exp_ff): T(t0, t) = exp(-sum_k I_k), every contribution clipped to the
// primitive's ellipsoid as in Sec. 4.1.

// Optical depth E_k at which component k collides: Philox4x32-10 with key (bits of u,
// 0x2406DEC0) and counter (k, 0, 0, 0), U = ((x0 >> 8) + 1) / 2^24 in (0, 1], E_k = -ln U (the
// appendix's -ln(1 - u') with u' = 1 - U).
double decomposition_exponential(double u, int32_t k) {
  const float f = float(u);
  uint32_t bits;
  std::memcpy(&bits, &f, 4);
  const uint32_t ctr[4] = {uint32_t(k), 0u, 0u, 0u};
  const uint32_t key[2] = {bits, 0x2406DEC0u};
  uint32_t x[4];
  philox4x32_10(ctr, key, x);
  return -std::log(double((x[0] >> 8) + 1u) * (1.0 / 16777216.0));
}

// The distance t in [a, b] of a hit with I(a, t) = E, for 0 < E < I(a, b): the erf^-1 closed
// form of App. A as the first guess, then Newton's method on I(a, t) - E with I' = G, kept
// inside a shrinking bracket.
double invert_integral(const Hit& h, double E) {
  const double s = std::sqrt(0.5 * h.A);
  const double amp = h.g0 * std::exp(-0.5 * h.d2) * std::sqrt(kPi / (2.0 * h.A));
  double lo = h.a, hi = h.b;
  double t = h.tstar + erfinv(std::erf(s * (h.a - h.tstar)) + E / amp) / s;
  if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
  for (int it = 0; it < 400; ++it) {
    const double f = ray_integral(h, h.a, t) - E;
    if (f == 0.0) return t;
    if (f < 0) lo = t; else hi = t;
    const double fp = gauss_at(h, t);
    double tn = fp > 0 ? t - f / fp : 0.5 * (lo + hi);
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    if (std::fabs(tn - t) <= 1e-16 * std::max(1.0, std::fabs(t)) || hi - lo <= 1e-16 * std::max(1.0, std::fabs(t)))
      return tn;
    t = tn;
  }
  return t;
}

// Analog decomposition tracking: every primitive on the ray samples its own exponential
// free flight by inverting 1 - exp(-I_k(a_k, t)) (a collision only when E_k < I_k(a_k, b_k)),
// and the nearest collision is the sample of the summed medium (equal distances: the lower id).
ExpFreeFlight sample_free_flight_exponential(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1,
                                             double k, int32_t exclude, double u) {
  const double inf = std::numeric_limits<double>::infinity();
  ExpFreeFlight r{-1, t1, inf, inf, 0.0, 0.0, 0.0};
  const std::vector<Hit> hits = all_hits(prims, o, d, t0, t1, k, exclude);
  const Hit* pick = nullptr;
  for (const Hit& h : hits) {
    const double E = decomposition_exponential(u, h.id);
    const double I = ray_integral(h, h.a, h.b);
    r.depth += I;
    r.margin = std::min(r.margin, std::fabs(E - I) / std::max(E, I));
    if (!(E < I)) continue;
    const double t = invert_integral(h, E);
    if (!pick || t < r.t) {
      if (pick) r.t_second = r.t;
      r.t = t;
      pick = &h;
    } else if (t < r.t_second) {
      r.t_second = t;
    }
  }
  if (pick) {
    r.prim = pick->id;
    r.amp = pick->g0 * std::exp(-0.5 * pick->d2) * std::sqrt(kPi / (2.0 * pick->A));
    r.G_t = gauss_at(*pick, r.t);
  }
  return r;
}

// Exponential transmittance over [t0, t1] (Eq. exp_ff with the ellipsoid cut-off).
double transmittance_exponential(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1, double k,
                                 int32_t exclude, double* depth_out) {
  double depth = 0.0;
  for (const Hit& h : all_hits(prims, o, d, t0, t1, k, exclude)) depth += ray_integral(h, h.a, h.b);
  if (depth_out) *depth_out = depth;
  return std::exp(-depth);
}

// Philox4x32-10: ten rounds of two 32x32->64 multiplications with the key bumped by the
// Weyl constants between rounds (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4).
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = uint64_t(0xD2511F53u) * c0;
    const uint64_t p1 = uint64_t(0xCD9E8D57u) * c2;
    const uint32_t n0 = uint32_t(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = uint32_t(p0 >> 32) ^ c3 ^ k1;
    c0 = n0;
    c1 = uint32_t(p1);
    c2 = n2;
    c3 = uint32_t(p0);
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

}  // namespace orc
