// Exponential-transmittance variant of the primitives (appendix "Sampling Exponential
// Transmittance Gaussians via Analog Decomposition Tracking"): the same Gaussians read as the
// extinction coefficient sigma_t(x) = sum_k G_k(x) of the classical model (Eq. exp_ff), so that
// T(t0, t) = exp(-sum_k I_k(a_k, min(b_k, t))) with each contribution clipped to its ellipsoid
// (Sec. 4.1).
//
// Free flight by analog decomposition tracking: every primitive on the ray draws its own
// collision depth E_k = -ln U_k and, when E_k < I_k(a_k, b_k), collides where I_k(a_k, t_k) = E_k
// (closed form through erfc^-1, App. A); the nearest collision is the sample of the summed
// medium. One thread per ray, nearest-first traversal whose far bound shrinks to the nearest
// collision found so far: a primitive that starts beyond it cannot be the answer.
#include "ugp_gauss.cuh"
#include "ugp_philox.cuh"
#include "ugp_trace.cuh"

namespace ugp {
namespace {

// Collision depth of primitive k: Philox4x32-10 with key (bits of the ray's uniform u,
// 0x2406DEC0) and counter (k, 0, 0, 0), U = ((x0 >> 8) + 1) / 2^24 in (0, 1], E = -ln U.
__device__ __forceinline__ float decomposition_exponential(float u, int k) {
  const uint4 x = philox4x32_10(make_uint4(uint32_t(k), 0u, 0u, 0u), make_uint2(__float_as_uint(u), 0x2406DEC0u));
  return -logf(float((x.x >> 8) + 1u) * (1.0f / 16777216.0f));
}

// erf argument tau_t with erf(tau_t) = erf(ta) + D, D in (0, erf(ty) - erf(ta)].  The sum is
// formed in the tail that holds the start (erfc(ta) - D for ta >= 0, erfc(-ta) + D otherwise)
// so a thin tail keeps its relative precision, then inverted with erfc^-1; the result is
// kept inside [ta, ty].
__device__ __forceinline__ float invert_erf_step(float ta, float ty, float D) {
  float tt;
  if (ta >= 0.f) {
    const float c = erfcf(ta) - D;  // erfc(tau_t)
    tt = c > 0.f ? erfcinvf(c) : ty;
  } else {
    const float y = erfcf(-ta) + D;  // 1 + erf(tau_t)
    if (y <= 1.f) {
      tt = -erfcinvf(y);
    } else {
      const float c = 2.f - y;  // erfc(tau_t)
      tt = c > 0.f ? erfcinvf(c) : ty;
    }
  }
  return fminf(fmaxf(tt, ta), ty);
}

// Per-ray traversal shared by the two queries: visits every primitive whose clipped interval
// [a, b] meets [t0, t_far()] in nearest-first order and calls visit(h) on it; t_far may shrink
// between calls.  Returns the ray status.
template <class Far, class Visit>
__device__ __forceinline__ uint8_t traverse(const TraceScene& sc, const Ray& ray, float t0, float t1, int excl,
                                            int* stk, Far t_far, Visit visit) {
  const int tid = threadIdx.x;
  int sp = 0, node = 0;
  while (true) {
    if (unsigned(node) >= unsigned(sc.n_nodes)) return UGP_RAY_BAD_NODE;
    const float4* nd = sc.nodes + 4 * node;
    const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
    const int4 n3 = __ldg(reinterpret_cast<const int4*>(nd) + 3);
    const float tf = t_far();
    float en[2];
    bool hc[2];
    hc[0] = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, ray, t0, tf, en[0]);
    hc[1] = n3.y != kEmptyChild && slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, ray, t0, tf, en[1]);
    const int ch[2] = {n3.x, n3.y};
    if ((ch[0] < 0 && ~ch[0] >= sc.n_prims) || (ch[1] < 0 && ch[1] != kEmptyChild && ~ch[1] >= sc.n_prims))
      return UGP_RAY_BAD_NODE;
    for (int c = 0; c < 2; ++c) {
      if (!hc[c] || ch[c] >= 0) continue;
      hc[c] = false;
      PrimHit h;
      if (prim_test(sc.prims, sc.wlo, ~ch[c], ray, t0, t1, sc.k2, excl, h)) visit(h);
    }
    if (hc[0] && hc[1]) {
      if (sp == kTrStack) return UGP_RAY_STACK_OVERFLOW;
      const bool first0 = en[0] <= en[1];
      stk[sp * kTrBlock + tid] = first0 ? ch[1] : ch[0];
      ++sp;
      node = first0 ? ch[0] : ch[1];
    } else if (hc[0]) {
      node = ch[0];
    } else if (hc[1]) {
      node = ch[1];
    } else {
      if (sp == 0) return UGP_RAY_OK;
      --sp;
      node = stk[sp * kTrBlock + tid];
    }
  }
}

__global__ void __launch_bounds__(kTrBlock, kTrBlocksPerSM)
k_exp_free_flight(TraceScene sc, int64_t n_rays, const float* __restrict__ o3, const float* __restrict__ d3,
                  const float* __restrict__ t0a, const float* __restrict__ t1a, const float* __restrict__ ua,
                  const int32_t* __restrict__ excl, int32_t* __restrict__ prim_out, float* __restrict__ t_out,
                  uint8_t* __restrict__ st_out) {
  __shared__ int stk[kTrStack * kTrBlock];
  const int64_t r = int64_t(blockIdx.x) * kTrBlock + threadIdx.x;
  if (r >= n_rays) return;
  const Ray ray = make_ray(ld3(o3, r), ld3(d3, r));
  const float t0 = __ldg(t0a + r), t1 = __ldg(t1a + r);
  const float u = __ldg(ua + r);
  const int ex = excl ? __ldg(excl + r) : -1;
  float t_best = t1;
  int best = -1;
  uint8_t st = UGP_RAY_OK;
  if (sc.n_prims > 0 && t0 < t1) {
    st = traverse(sc, ray, t0, t1, ex, stk, [&]() { return t_best; }, [&](const PrimHit& h) {
      // only the part of the interval before the nearest collision so far can win
      const float y = fminf(h.b, t_best);
      if (!(h.a < y)) return;
      const float ta = h.a_end ? -h.th : tau_at(h.a, h.tn, h.ts, h.s);
      const float ty = (h.b_end && y == h.b) ? h.th : tau_at(y, h.tn, h.ts, h.s);
      const float E = decomposition_exponential(u, h.id);
      if (!(E < 2.f * half_integral_tau(ta, ty, h.s, h.e0))) return;
      // I(a, t) = e0 sqrt(pi) / (2 s) [erf(tau_t) - erf(tau_a)] = E
      const float D = E * (2.f * h.s) / (h.e0 * kSqrtPi);
      const float tt = invert_erf_step(ta, ty, D);
      const float t = fminf(fmaxf(h.tn + (h.ts + tt / h.s), h.a), y);
      if (best < 0 || t < t_best || (t == t_best && h.id < best)) {
        t_best = t;
        best = h.id;
      }
    });
  }
  prim_out[r] = best;
  t_out[r] = best >= 0 ? t_best : t1;
  if (st_out) st_out[r] = st;
}

__global__ void __launch_bounds__(kTrBlock, kTrBlocksPerSM)
k_exp_transmittance(TraceScene sc, int64_t n_rays, const float* __restrict__ o3, const float* __restrict__ d3,
                    const float* __restrict__ t0a, const float* __restrict__ t1a, const int32_t* __restrict__ excl,
                    float* __restrict__ T_out, uint8_t* __restrict__ st_out) {
  // exp(-x) is 0 in float32 for x above about 104; the traversal stops once the depth passes this
  constexpr float kOpaqueDepth = 112.f;
  __shared__ int stk[kTrStack * kTrBlock];
  const int64_t r = int64_t(blockIdx.x) * kTrBlock + threadIdx.x;
  if (r >= n_rays) return;
  const Ray ray = make_ray(ld3(o3, r), ld3(d3, r));
  const float t0 = __ldg(t0a + r), t1 = __ldg(t1a + r);
  const int ex = excl ? __ldg(excl + r) : -1;
  float depth = 0.f, far = t1;
  uint8_t st = UGP_RAY_OK;
  if (sc.n_prims > 0 && t0 < t1) {
    st = traverse(sc, ray, t0, t1, ex, stk, [&]() { return far; }, [&](const PrimHit& h) {
      depth += 2.f * hit_half_integral(h);
      if (depth > kOpaqueDepth) far = t0;  // the remaining nodes fail the slab test
    });
  }
  T_out[r] = expf(-depth);
  if (st_out) st_out[r] = st;
}

}  // namespace
}  // namespace ugp

using namespace ugp;

// one thread per ray: the grid's x extent bounds the ray count
static constexpr int64_t kMaxRays = int64_t(0x7fffffff) * kTrBlock;

extern "C" ugp_status ugp_sample_free_flight_exponential(const ugp_bvh* bvh, int64_t n_rays, const float* o3,
                                                         const float* d3, const float* t0, const float* t1,
                                                         const float* u, const int32_t* exclude_prim,
                                                         int32_t* prim_out, float* t_out, uint8_t* status_out,
                                                         void* stream) {
  clear_error();
  ugp_status s = check_rays("ugp_sample_free_flight_exponential", bvh, n_rays, o3, d3, t0, t1);
  if (s != UGP_OK) return s;
  if (n_rays > 0 && (!u || !prim_out || !t_out))
    return fail(UGP_ERR_INVALID_ARG, "ugp_sample_free_flight_exponential: NULL uniform or output array");
  if (n_rays == 0) return UGP_OK;
  if (n_rays > kMaxRays) return fail(UGP_ERR_INVALID_ARG, "%s: n_rays above %lld", __func__, (long long)kMaxRays);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_begin(kStQuery, st);
  k_exp_free_flight<<<unsigned((n_rays + kTrBlock - 1) / kTrBlock), kTrBlock, 0, st>>>(
      trace_scene(bvh), n_rays, o3, d3, t0, t1, u, exclude_prim, prim_out, t_out, status_out);
  prof_end(kStQuery, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

extern "C" ugp_status ugp_trace_transmittance_exponential(const ugp_bvh* bvh, int64_t n_rays, const float* o3,
                                                          const float* d3, const float* t0, const float* t1,
                                                          const int32_t* exclude_prim, float* T_out,
                                                          uint8_t* status_out, void* stream) {
  clear_error();
  ugp_status s = check_rays("ugp_trace_transmittance_exponential", bvh, n_rays, o3, d3, t0, t1);
  if (s != UGP_OK) return s;
  if (n_rays > 0 && !T_out) return fail(UGP_ERR_INVALID_ARG, "ugp_trace_transmittance_exponential: NULL T_out");
  if (n_rays == 0) return UGP_OK;
  if (n_rays > kMaxRays) return fail(UGP_ERR_INVALID_ARG, "%s: n_rays above %lld", __func__, (long long)kMaxRays);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_begin(kStQuery, st);
  k_exp_transmittance<<<unsigned((n_rays + kTrBlock - 1) / kTrBlock), kTrBlock, 0, st>>>(
      trace_scene(bvh), n_rays, o3, d3, t0, t1, exclude_prim, T_out, status_out);
  prof_end(kStQuery, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}
