// Internal declarations of the FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY. The oracle is a plain, slow, brute-force statement
// of what the Gaussian-primitive path tracer computes. Only the tests, the
// smoke check and the benchmark's CPU-baseline leg may load it; the product
// path never does. It shares no code with the CUDA library.
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>

namespace orc {

struct V3 {
  double x, y, z;
};
inline V3 v3(double x, double y, double z) { return V3{x, y, z}; }
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator-(V3 a) { return {-a.x, -a.y, -a.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline V3 operator*(V3 a, V3 b) { return {a.x * b.x, a.y * b.y, a.z * b.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double length(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 normalize(V3 a) { return (1.0 / length(a)) * a; }
inline V3 load3(const float* p) { return {p[0], p[1], p[2]}; }

// One Gaussian primitive (Eq. 1, Eq. 2): mean mu, whitening W = (RS)^-1 = S^-1 R^T
// (row-major), normaliser g0 = c / ((2 pi)^{3/2} |Sigma|^{1/2}).
struct Prim {
  V3 mu;
  double W[9];
  double R[9];
  double s[3];
  double g0;
};

// The scene as passed through the oracle's C entry points (same SoA layout as
// the CUDA library's inputs, float32).
struct SceneIn {
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
  const float* disney9;  // n x 9, read for type-3 (Disney) primitives; NULL: published defaults
};

Prim make_prim(const float* mean3, const float* quat4, const float* scale3, float magnitude);
std::vector<Prim> make_prims(const SceneIn& s);

// k of the bounding ellipsoid (Eq. 4): ||(RS)^-1 (x - mu)|| = sqrt(-2 ln eps).
double cutoff_k(double eps);

// A primitive's clipped interval along a ray and the quantities of App. A.
struct Hit {
  int32_t id;
  double a, b;   // clipped interval [max(t0, t-), min(t1, t+)]
  double A;      // w^T Sigma^-1 w
  double tstar;  // -B / (2A): parameter of the closest approach in the whitened metric
  double d2;     // C - B^2 / (4A): squared whitened distance of the closest approach
  double g0;
};

// Ray x_t = o + t d. Returns true and fills h if the ray's k-ellipsoid interval
// intersected with [t0, t1] is non-empty.
bool ray_prim(const Prim& p, int32_t id, V3 o, V3 d, double t0, double t1, double k, Hit* h);
// App. A quantities without clipping (for the unclipped integral).
void ray_prim_quadratic(const Prim& p, V3 o, V3 d, double* A, double* tstar, double* d2);
// I(x, y) of Eq. 6 for a hit, by the closed form of App. A (x <= y).
double ray_integral(const Hit& h, double x, double y);
// G(x_t) of Eq. 1 for a hit.
double gauss_at(const Hit& h, double t);
// All hits of a ray, brute force over every primitive; sorted by id.
std::vector<Hit> all_hits(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1,
                          double k, int32_t exclude);

// Transmittance of Eq. 7 over [t0, t1]: max(0, 1 - tau), tau = 1/2 sum_k I_k(clip).
double transmittance(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1, double k,
                     int32_t exclude, double* tau_out);

struct FreeFlight {
  int32_t prim;   // -1: escape
  double t_u;     // root of F(t_u) = u
  double t_spawn; // centre of the chosen primitive's clipped interval
  double F_end;   // F(t1) = 1/2 sum_k I_k(clip) (unclamped optical depth)
  int32_t n_active;
  double race_margin;  // relative gap between the two smallest race keys (inf if one candidate)
};
FreeFlight sample_free_flight(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1,
                              double k, int32_t exclude, double u, double u2);
FreeFlight sample_free_flight_hits(const std::vector<Hit>& hits, double t0, double t1, double u,
                                   double u2);

// The paper's disambiguation rule (pick proportional to I_k(s0, t_u) in the segment where F
// reaches 1), kept to measure its bias. Returns the primitive id, or -1 for escape.
int32_t sample_free_flight_paper_rule(const std::vector<Hit>& hits, double t0, double t1, double u, double u2);

// Radiance-field render of Sec. 7 (Eq. rf): L = sum_k 1/2 I_k(a_k, min(b_k, t_sat)) L_e,k, with
// t_sat the root of F(t_sat) = 1 (free flight at u = 1); when F(t1) <= 1 the ray is not
// saturated, t_sat = t1 and the remaining 1 - F(t1) sees the background. emission3 is indexed
// by primitive id. Returns F(t1) in *F_end (unclamped).
// t_shift_ulps moves the saturating distance by that many float32 ulps of itself (0: none), so a
// test can bound how much the float32 resolution of t changes the result.
void radiance_field(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1, double k,
                    const float* emission3, const double* background3, double t_shift_ulps, double* rgb_out,
                    double* t_sat_out, double* F_end_out);

// Exponential-transmittance variant (appendix on analog decomposition tracking): sigma_t(x) =
// sum_k G_k(x) and T = exp(-sum_k I_k) with the ellipsoid cut-off.
struct ExpFreeFlight {
  int32_t prim;     // nearest colliding primitive, -1: escape
  double t;         // its collision distance (t1 on escape)
  double t_second;  // second-nearest collision distance (inf if none)
  double margin;    // min over the ray's primitives of |E_k - I_k(a_k, b_k)| / max(E_k, I_k)
  double amp;       // g0 e^{-d2/2} sqrt(pi / 2A) of the chosen primitive: I = amp [erf(tau_t) - erf(tau_a)]
  double G_t;       // G of the chosen primitive at t
  double depth;     // sum_k I_k(a_k, b_k): optical depth of [t0, t1]
};
double decomposition_exponential(double u, int32_t k);
double invert_integral(const Hit& h, double E);
ExpFreeFlight sample_free_flight_exponential(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1,
                                             double k, int32_t exclude, double u);
double transmittance_exponential(const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1, double k,
                                 int32_t exclude, double* depth_out);

// The paper's own sampler over an SAH kd-tree (kdtree.cpp): a diagnostic of the paper-faithful
// variant, not a parity target.
struct KdNode {
  int axis = -1;     // -1: leaf
  double pos = 0.0;  // split plane
  int child[2] = {-1, -1};
  int32_t first = 0, count = 0;  // leaf: range in KdTree::leaf_ids
};
struct KdTree {
  std::vector<KdNode> nodes;  // nodes[0] is the root
  std::vector<int32_t> leaf_ids;
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
};
struct KdStats {
  int64_t nodes_visited = 0, prims_tested = 0;
  double F_end = 0.0;            // the CDF reached (1/2 sum I when the ray escapes)
  double ambiguous_start = 0.0;  // start of the ambiguous segment used (NaN if none)
};
KdTree kd_build(const std::vector<Prim>& prims, double k);

// A plain BVH that finds the same intervals as the brute-force loop (accel.cpp). While g_accel
// points at one built over a primitive list, all_hits over that list uses it.
struct AccelNode {
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  int left = -1, right = -1;
  int32_t first = 0, count = 0;
};
struct Accel {
  const std::vector<Prim>* prims = nullptr;
  std::vector<AccelNode> nodes;
  std::vector<int32_t> ids;
};
Accel accel_build(const std::vector<Prim>& prims, double k);
std::vector<Hit> accel_hits(const Accel& A, V3 o, V3 d, double t0, double t1, double k, int32_t exclude);
extern const Accel* g_accel;
// nbins = 0: exact line-sweep segments in a leaf where the CDF reaches 1 (the paper's CPU
// partition); nbins > 0: that many equal bins of the ray-node interval (its GPU partition).
int32_t kd_sample_free_flight(const KdTree& T, const std::vector<Prim>& prims, V3 o, V3 d, double t0, double t1,
                              double k, double u, double u2, KdStats* stats, int nbins = 0);

double erfinv(double y);
double race_exponential(double u2, int32_t k);

// Philox4x32-10 (Salmon et al., SC'11).
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
inline double u24(uint32_t x) { return double(x >> 8) * (1.0 / 16777216.0); }

}  // namespace orc
