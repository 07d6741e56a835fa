// Phase-function queries (Sec. 6, Eq. 11-12, App. B) on independent (material, direction)
// records: the same device functions the renderer's shading kernels call, one thread per record,
// so that each can be checked element by element against a reference.
#include "ugp_internal.cuh"
#include "ugp_phase.cuh"

namespace ugp {
namespace {

constexpr int kPqBlock = 128;

__global__ void __launch_bounds__(kPqBlock)
k_phase_query(int64_t n, const uint8_t* __restrict__ type, const float* __restrict__ albedo3,
              const float* __restrict__ roughness, const float* __restrict__ sggx6, const float* __restrict__ disney9,
              const float* __restrict__ wo3, const float* __restrict__ wi3, const float* __restrict__ ue6,
              const float* __restrict__ us4, float* __restrict__ eval3, float* __restrict__ pdf,
              float* __restrict__ swi3, float* __restrict__ sw3, uint8_t* __restrict__ sok) {
  const int64_t i = int64_t(blockIdx.x) * kPqBlock + threadIdx.x;
  if (i >= n) return;
  Material m;
  m.type = type[i];
  m.albedo = f3(albedo3[3 * i], albedo3[3 * i + 1], albedo3[3 * i + 2]);
  m.alpha = roughness[i];
  for (int j = 0; j < 6; ++j) m.S[j] = sggx6[6 * i + j];
  for (int j = 0; j < 9; ++j) m.dis[j] = disney9 ? disney9[9 * i + j] : 0.f;
  const float3 wo = f3(wo3[3 * i], wo3[3 * i + 1], wo3[3 * i + 2]);
  const float3 wi = f3(wi3[3 * i], wi3[3 * i + 1], wi3[3 * i + 2]);
  float U[6];
  for (int j = 0; j < 6; ++j) U[j] = ue6[6 * i + j];
  const float3 f = phase_eval(m, wi, wo, U);
  eval3[3 * i] = f.x;
  eval3[3 * i + 1] = f.y;
  eval3[3 * i + 2] = f.z;
  pdf[i] = phase_pdf_approx(m, wi, wo);
  float V[4];
  for (int j = 0; j < 4; ++j) V[j] = us4[4 * i + j];
  float3 swi = f3(0.f, 0.f, 0.f), sw = f3(0.f, 0.f, 0.f);
  const bool ok = phase_sample(m, wo, V, swi, sw);
  if (!ok) sw = f3(0.f, 0.f, 0.f);
  swi3[3 * i] = swi.x;
  swi3[3 * i + 1] = swi.y;
  swi3[3 * i + 2] = swi.z;
  sw3[3 * i] = sw.x;
  sw3[3 * i + 1] = sw.y;
  sw3[3 * i + 2] = sw.z;
  sok[i] = ok ? 1 : 0;
}

}  // namespace
}  // namespace ugp

using namespace ugp;

extern "C" ugp_status ugp_phase_query(int64_t n, const uint8_t* type, const float* albedo3, const float* roughness,
                                      const float* sggx6, const float* disney9, const float* wo3, const float* wi3,
                                      const float* u_eval6, const float* u_sample4, float* eval3_out,
                                      float* pdf_out, float* sample_wi3_out, float* sample_weight3_out,
                                      uint8_t* sample_ok_out, void* stream) {
  clear_error();
  if (n < 0) return fail(UGP_ERR_INVALID_ARG, "ugp_phase_query: n < 0");
  if (n == 0) return UGP_OK;
  if (!type || !albedo3 || !roughness || !sggx6 || !wo3 || !wi3 || !u_eval6 || !u_sample4 || !eval3_out ||
      !pdf_out || !sample_wi3_out || !sample_weight3_out || !sample_ok_out)
    return fail(UGP_ERR_INVALID_ARG, "ugp_phase_query: NULL array (only disney9 may be NULL)");
  if (n > (int64_t(1) << 31) * kPqBlock) return fail(UGP_ERR_INVALID_ARG, "ugp_phase_query: n too large");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_begin(kStQuery, st);
  k_phase_query<<<unsigned((n + kPqBlock - 1) / kPqBlock), kPqBlock, 0, st>>>(
      n, type, albedo3, roughness, sggx6, disney9, wo3, wi3, u_eval6, u_sample4, eval3_out, pdf_out, sample_wi3_out,
      sample_weight3_out, sample_ok_out);
  prof_end(kStQuery, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}
