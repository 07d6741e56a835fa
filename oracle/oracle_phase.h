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

struct Material {
  int type;
  V3 albedo;     // Lambertian rho, or GGX F0
  double alpha;  // GGX roughness
  V3 emission;   // emissive primitives
  double S[6];   // SGGX matrix (Sxx, Syy, Szz, Sxy, Sxz, Syz)
};

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
};

// Renders pixels [p_begin, p_end) of the image (row-major), adding per-channel sums of the
// sample values and of their squares; also counts queries.
void render_pixels(const SceneIn& s, const Camera& cam, const Lights& L, const RenderParams& P,
                   int64_t p_begin, int64_t p_end, double* accum, double* accum_sq, int64_t* n_extend,
                   int64_t* n_shadow);

}  // namespace orc
