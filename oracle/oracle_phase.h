// Appearance and path-tracing declarations of the FP64 oracle.
//
// TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).
#pragma once
#include "oracle_guide.h"
#include "oracle_internal.h"

namespace orc {

constexpr int kMatDiffuse = 0;
constexpr int kMatGGX = 1;
constexpr int kMatEmissive = 2;
constexpr int kMatDisney = 3;

struct Material {
  int type;
  V3 albedo;     // Lambertian rho, GGX F0, or the Disney base colour
  double alpha;  // GGX roughness
  V3 emission;   // emissive primitives
  double S[6];   // SGGX matrix (Sxx, Syy, Szz, Sxy, Sxz, Syz)
  // Disney base: metallic, subsurface, specular, specular tint, roughness, sheen, sheen tint,
  // clearcoat, clearcoat gloss
  double dis[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};

// Disney principled base BSDF (disney.cpp): derived constants and the sampler's lobe choice.
struct DisneyLobes {
  V3 spec0, sheen;
  double alpha, alpha_c;
  double p_diffuse, p_spec, p_coat;
};
DisneyLobes disney_lobes(const Material& m);
double gtr1_D(double a, double cos_h);
V3 disney_f_diffuse(const Material& m, V3 wi, V3 wo, V3 n);
V3 disney_f_glossy(const Material& m, V3 wi, V3 wo, V3 n);
V3 disney_f(const Material& m, V3 wi, V3 wo, V3 n);
double disney_pdf(const Material& m, V3 wi, V3 wo, V3 n);
bool disney_sample(const Material& m, V3 wo, V3 n, const double U[2], V3* wi, V3* weight);

Material material_of(const SceneIn& s, int64_t i);

void onb(V3 n, V3* b1, V3* b2);
double sggx_sigma(const double s6[6], V3 w);
double sggx_D(const double s6[6], V3 n);
double sggx_Dvis(const double s6[6], V3 wo, V3 n);
V3 sggx_sample_vndf(const double s6[6], V3 wo, double U1, double U2);
void sggx_roughen(const double s6[6], double alpha, double out6[6]);
bool sggx_isotropic(const double s6[6]);

V3 lambert_f(V3 rho, V3 wi, V3 wo, V3 n);
double ggx_D(double alpha, double cos_h);
double ggx_Lambda(double alpha, double cos_t);
V3 ggx_f(V3 F0, double alpha, V3 wi, V3 wo, V3 n);
V3 ggx_sample_vn(double alpha, V3 wo, V3 n, double U1, double U2);
double micro_pdf(double alpha, V3 n, V3 h);
V3 micro_sample(double alpha, V3 h, double U1, double U2);
V3 cos_sample(V3 n, double U1, double U2);

V3 phase_eval_stochastic(const Material& m, V3 wi, V3 wo, const double U[6]);
V3 phase_eval_lambert_sphere(V3 rho, V3 wi, V3 wo);
V3 phase_eval(const Material& m, V3 wi, V3 wo, const double U[6]);
bool phase_sample(const Material& m, V3 wo, const double U[4], V3* wi, V3* weight);
double phase_pdf_approx(const Material& m, V3 wi, V3 wo);

// Camera, lights and render parameters (same meaning as the CUDA library's structs).
struct Camera {
  V3 eye, look, up;
  double vfov_deg;
  int width, height;
};
struct Lights {
  bool has_quad;
  V3 corner, e1, e2, Le;
  V3 bg;
};
struct RenderParams {
  int spp, spp_begin, max_depth;
  uint64_t seed;
  double cutoff_eps;
  int nee;         // 1: light sampling + MIS, 0: lights found by phase sampling only
  int spawn_mode;  // 0: centre of the primitive's clipped interval, 1: x_{t_u}
  // Learned guide (NULL: plain phase sampling). With a guide, each scattering vertex picks the
  // guide with probability guide_alpha, else phase sampling, and weights the sample by the
  // balance heuristic over both (one-sample MIS); the same mixture pdf enters the MIS with
  // light sampling.
  const float* guide = nullptr;
  GuideCfg guide_cfg{};
  double guide_alpha = 0.5;
  int nee_emitters = 0;  // 1: also next-event estimation toward emissive primitives, with MIS
  int accel = 0;         // 1: find intervals with a BVH (same intervals, for timing large scenes)
  // Vertices whose base is glossier than this (GGX alpha, or the Disney specular's
  // max(1e-3, roughness^2), below it) scatter by phase sampling alone even with a guide.
  double guide_min_roughness = 0.0;
  // Columns [crop_x0, crop_x1) of the pixel range only (crop_x1 <= crop_x0: every column), so
  // that a rectangle of rows and columns can be rendered in one call.
  int crop_x0 = 0, crop_x1 = 0;
};

// Next-event estimation toward emissive primitives (not specified by the paper): emitter j is
// chosen with probability pi_j proportional to c_j mean(L_e,j), and a point of it from its
// Gaussian restricted to the k-ellipsoid.
struct EmitterTable {
  std::vector<int32_t> ids;
  std::vector<double> cdf;  // running sums of c_j mean(L_e,j)
  double total = 0.0;
  double mass = 0.0;        // P(|z| <= k), z ~ N(0, I_3): the Gaussian mass inside the ellipsoid
};
EmitterTable emitter_table(const SceneIn& s, double k);
// CDF of the chi distribution with 3 degrees of freedom (radius of a standard 3D normal).
double chi3_cdf(double r);
// A point of primitive p from its Gaussian restricted to the k-ellipsoid (three uniforms).
V3 sample_in_ellipsoid(const Prim& p, double k, const double U[3]);
// One light sample from vertex x (material m, outgoing wo, the vertex's primitive excluded).
// Returns false when it adds nothing; else *contrib = f_p * L_e * c_j m / (2 r^2 pi_j) (the
// estimate without beta and MIS weight), *dir the direction, and the two balance-heuristic terms
// in a common scale: *p_light = 2 r_c^2 pi_j with r_c the distance from x to the emitter's mean,
// *p_scatter_scale = c_j m (times the scattering pdf).
bool emitter_nee(const SceneIn& s, const std::vector<Prim>& prims, const EmitterTable& E, double k,
                 const Material& m, V3 x, V3 wo, int32_t exclude, const double U4[4], const double Uf[6],
                 V3* contrib, V3* dir, double* p_light, double* p_scatter_scale, int64_t* shadow_rays);

// Sum and sum of squares of n one-sample light estimates of emitter_nee (no MIS weight) at the
// vertex x; uniforms from Philox with key seed and counters (0, sample, 8 | 9 | 10, 0).
void emitter_nee_sums(const SceneIn& s, double cutoff_eps, const Material& m, V3 x, V3 wo, int32_t exclude,
                      int64_t n, uint64_t seed, double sum[3], double sq[3]);

// Renders pixels [p_begin, p_end) of the image (row-major), adding per-channel sums of the
// sample values and of their squares; also counts queries.
void render_pixels(const SceneIn& s, const Camera& cam, const Lights& L, const RenderParams& P,
                   int64_t p_begin, int64_t p_end, double* accum, double* accum_sq, int64_t* n_extend,
                   int64_t* n_shadow);

}  // namespace orc
