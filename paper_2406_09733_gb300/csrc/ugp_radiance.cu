// Radiance-field forward render (Sec. 7, Eq. rf): an emitting, non-scattering medium of the
// primitives, rendered without Monte Carlo.
//
//   L = sum_k 1/2 I_k(a_k, min(b_k, t_sat)) L_e,k  +  max(0, 1 - F(t1)) L_bg  (when F(t1) <= 1)
//
// t_sat is where F (the free-flight CDF, Eq. 8) reaches 1: the free-flight root for u = 1, which
// is also how the paper settles which primitives straddle the saturating boundary. Each
// primitive then counts with its probability mass up to t_sat, which needs no choice among
// them. Two passes per ray: free-flight sampling at u = 1 (scan and finish, as for the path
// tracer), then one thread per ray sums the clipped integrals weighted by the emissions.
#include "ugp_dense.cuh"
#include "ugp_gauss.cuh"
#include "ugp_trace.cuh"

namespace ugp {
namespace {

__global__ void k_fill(int64_t n, float* __restrict__ p, float v) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = v;
}

// One ray per thread: traversal over [t0, t_end] (t_end = t_sat when the free-flight pass found
// one, else t1), every clipped interval cut at t_end, its 1/2 I times the primitive's emission.
__global__ void __launch_bounds__(kTrBlock, kTrBlocksPerSM)
k_radiance(TraceScene sc, int64_t n_rays, const float* __restrict__ o3, const float* __restrict__ d3,
           const float* __restrict__ t0a, const float* __restrict__ t1a, const int32_t* __restrict__ prim_ff,
           const float* __restrict__ tu_ff, const uint8_t* __restrict__ st_ff, const float* __restrict__ em3,
           float3 bg, float* __restrict__ rgb_out, uint8_t* __restrict__ st_out) {
  __shared__ int stk[kTrStack * kTrBlock];
  const int tid = threadIdx.x;
  const int64_t r = int64_t(blockIdx.x) * kTrBlock + tid;
  if (r >= n_rays) return;
  const Ray ray = make_ray(ld3(o3, r), ld3(d3, r));
  const float t0 = __ldg(t0a + r), t1 = __ldg(t1a + r);
  const bool sat = __ldg(prim_ff + r) >= 0;
  const float t_end = sat ? __ldg(tu_ff + r) : t1;
  uint8_t st = st_ff ? __ldg(st_ff + r) : UGP_RAY_OK;
  float cr = 0.f, cg = 0.f, cb = 0.f, mass = 0.f;
  if (sc.n_prims > 0 && t0 < t_end && st == UGP_RAY_OK) {
    int sp = 0, node = 0;
    while (true) {
      if (unsigned(node) >= unsigned(sc.n_nodes)) {
        st = UGP_RAY_BAD_NODE;
        break;
      }
      const float4* nd = sc.nodes + 4 * node;
      const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
      const int4 n3 = __ldg(reinterpret_cast<const int4*>(nd) + 3);
      float en[2];
      bool hc[2];
      hc[0] = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, ray, t0, t_end, en[0]);
      hc[1] = n3.y != kEmptyChild && slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, ray, t0, t_end, en[1]);
      const int ch[2] = {n3.x, n3.y};
      if ((ch[0] < 0 && ~ch[0] >= sc.n_prims) || (ch[1] < 0 && ch[1] != kEmptyChild && ~ch[1] >= sc.n_prims)) {
        st = UGP_RAY_BAD_NODE;
        break;
      }
      for (int c = 0; c < 2; ++c) {
        if (!hc[c] || ch[c] >= 0) continue;
        hc[c] = false;
        PrimHit h;
        if (!prim_test(sc.prims, sc.wlo, ~ch[c], ray, t0, t1, sc.k2, -1, h)) continue;
        const float y = fminf(h.b, t_end);
        if (!(h.a < y)) continue;
        const float v = seg_half_integral(h.a, y, h.a, h.b, h.a_end, h.b_end, h.tn, h.ts, h.s, h.e0, h.th);
        mass += v;
        cr = fmaf(v, __ldg(em3 + 3 * int64_t(h.id)), cr);
        cg = fmaf(v, __ldg(em3 + 3 * int64_t(h.id) + 1), cg);
        cb = fmaf(v, __ldg(em3 + 3 * int64_t(h.id) + 2), cb);
      }
      if (hc[0] && hc[1]) {
        if (sp == kTrStack) {
          st = UGP_RAY_STACK_OVERFLOW;
          break;
        }
        const bool first0 = en[0] <= en[1];
        stk[sp * kTrBlock + tid] = first0 ? ch[1] : ch[0];
        ++sp;
        node = first0 ? ch[0] : ch[1];
      } else if (hc[0]) {
        node = ch[0];
      } else if (hc[1]) {
        node = ch[1];
      } else {
        if (sp == 0) break;
        --sp;
        node = stk[sp * kTrBlock + tid];
      }
    }
  }
  const float rest = sat ? 0.f : fmaxf(0.f, 1.f - mass);
  rgb_out[3 * r] = fmaf(rest, bg.x, cr);
  rgb_out[3 * r + 1] = fmaf(rest, bg.y, cg);
  rgb_out[3 * r + 2] = fmaf(rest, bg.z, cb);
  if (st_out) st_out[r] = st;
}

// Workspace: the free-flight pass's, then u, u2, prim, t_u, t_spawn and the status per ray.
struct RfLayout {
  size_t ff, u, u2, prim, tu, tsp, st, total;
};
RfLayout rf_layout(int64_t n) {
  RfLayout L;
  size_t off = 0;
  L.ff = off;   off += dense_queue_bytes(n) + slot_list_bytes(n);
  L.u = off;    off += align256(size_t(n) * 4);
  L.u2 = off;   off += align256(size_t(n) * 4);
  L.prim = off; off += align256(size_t(n) * 4);
  L.tu = off;   off += align256(size_t(n) * 4);
  L.tsp = off;  off += align256(size_t(n) * 4);
  L.st = off;   off += align256(size_t(n));
  L.total = off;
  return L;
}

}  // namespace
}  // namespace ugp

using namespace ugp;

extern "C" size_t ugp_render_radiance_field_workspace_size(int64_t n_rays) {
  if (n_rays < 0 || n_rays > (int64_t(1) << 31) - 1) return 0;
  return rf_layout(n_rays).total;
}

extern "C" ugp_status ugp_render_radiance_field(const ugp_bvh* bvh, int64_t n_rays, const float* o3,
                                                const float* d3, const float* t0, const float* t1,
                                                const float* emission3, const float* background3, float* rgb_out,
                                                uint8_t* status_out, void* workspace, size_t workspace_bytes,
                                                void* stream) {
  clear_error();
  ugp_status s = check_rays("ugp_render_radiance_field", bvh, n_rays, o3, d3, t0, t1);
  if (s != UGP_OK) return s;
  if (n_rays > 0 && (!emission3 || !rgb_out))
    return fail(UGP_ERR_INVALID_ARG, "ugp_render_radiance_field: NULL emission or output array");
  if (n_rays == 0) return UGP_OK;
  if (n_rays > (int64_t(1) << 31) - 1)
    return fail(UGP_ERR_INVALID_ARG, "ugp_render_radiance_field: at most 2^31 - 1 rays per call");
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(UGP_ERR_INVALID_ARG, "ugp_render_radiance_field: workspace must be non-NULL and 256-byte aligned");
  const RfLayout L = rf_layout(n_rays);
  if (workspace_bytes < L.total)
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_render_radiance_field: need %zu bytes, got %zu", L.total,
                workspace_bytes);
  const float3 bg = background3 ? make_float3(background3[0], background3[1], background3[2])
                                : make_float3(0.f, 0.f, 0.f);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  float* u = reinterpret_cast<float*>(ws + L.u);
  float* u2 = reinterpret_cast<float*>(ws + L.u2);
  int32_t* prim = reinterpret_cast<int32_t*>(ws + L.prim);
  float* tu = reinterpret_cast<float*>(ws + L.tu);
  float* tsp = reinterpret_cast<float*>(ws + L.tsp);
  uint8_t* sf = reinterpret_cast<uint8_t*>(ws + L.st);
  const TraceScene sc = trace_scene(bvh);
  const int fill_grid = int((n_rays + 255) / 256 < 4096 ? (n_rays + 255) / 256 : 4096);
  prof_begin(kStQuery, st);
  k_fill<<<fill_grid, 256, 0, st>>>(n_rays, u, 1.f);  // u = 1: the root is the saturating distance
  prof_end(kStQuery, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  UGP_CUDA_CHECK(cudaMemsetAsync(u2, 0, size_t(n_rays) * 4, st));
  if ((s = launch_free_flight(sc, n_rays, o3, d3, t0, t1, u, u2, nullptr, prim, tu, tsp, sf, ws + L.ff, true, st)) !=
      UGP_OK)
    return s;
  prof_begin(kStQuery, st);
  k_radiance<<<unsigned((n_rays + kTrBlock - 1) / kTrBlock), kTrBlock, 0, st>>>(
      sc, n_rays, o3, d3, t0, t1, prim, tu, sf, emission3, bg, rgb_out, status_out);
  prof_end(kStQuery, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}
