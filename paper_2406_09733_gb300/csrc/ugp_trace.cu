// Transmittance evaluation (Sec. 5.3, Eq. 7) over the BVH, and hit collection for diagnostics.
//
// One thread per ray.  Traversal stacks live in shared memory, one column per thread
// (stack[level][thread]) so neighbouring threads hit neighbouring banks.
#include "ugp_gauss.cuh"
#include "ugp_trace.cuh"
#include "ugp_transmit.cuh"

namespace ugp {

// ----------------------------------------------------------------------------------------
// Transmittance: T = max(0, 1 - 1/2 sum_k I_k(clip_k)).  Any traversal order gives the same
// sum; nearest-child-first only makes the early exit at sum >= 1 come sooner.
template <bool STATS>
__global__ void __launch_bounds__(kTrBlock, kTrBlocksPerSM)
k_transmittance(TraceScene sc, int64_t n_rays, const float* __restrict__ o3, const float* __restrict__ d3,
                const float* __restrict__ t0a, const float* __restrict__ t1a,
                const int32_t* __restrict__ excl, float* __restrict__ T_out, uint8_t* __restrict__ st_out,
                unsigned long long* __restrict__ ctr) {
  __shared__ int stk[kTrStack * kTrBlock];
  __shared__ unsigned long long tr_acc[kTrBlock];
  __shared__ int tr_owner[kTrBlock];
  const int64_t r = int64_t(blockIdx.x) * kTrBlock + threadIdx.x;
  if (r >= n_rays) return;
  TrStats ts{0u, 0u, UGP_RAY_OK};
  const float acc = tr_optical_depth(sc, make_ray(ld3(o3, r), ld3(d3, r)), __ldg(t0a + r), __ldg(t1a + r),
                                     excl ? __ldg(excl + r) : -1, stk + threadIdx.x, kTrBlock, tr_acc + threadIdx.x,
                                     tr_owner + threadIdx.x, ts);
  T_out[r] = fmaxf(0.f, 1.f - acc);
  if (st_out) st_out[r] = ts.st;
  if (STATS) add_counters(ctr, ts.n_nodes, ts.n_prims, 1u, 1u, 0u);
}

// All hits along each ray, for hit-set diagnostics (no early exit).
__global__ void __launch_bounds__(kTrBlock)
k_collect_hits(TraceScene sc, int64_t n_rays, const float* __restrict__ o3, const float* __restrict__ d3,
               const float* __restrict__ t0a, const float* __restrict__ t1a,
               const int32_t* __restrict__ excl, int cap, int32_t* __restrict__ ids, float* __restrict__ aa,
               float* __restrict__ bb, int32_t* __restrict__ cnt, uint8_t* __restrict__ st_out) {
  __shared__ int stk[kTrStack * kTrBlock];
  const int tid = threadIdx.x;
  const int64_t r = int64_t(blockIdx.x) * kTrBlock + tid;
  if (r >= n_rays) return;
  const Ray ray = make_ray(ld3(o3, r), ld3(d3, r));
  const float t0 = __ldg(t0a + r), t1 = __ldg(t1a + r);
  const int ex = excl ? __ldg(excl + r) : -1;
  int count = 0;
  uint8_t st = UGP_RAY_OK;
  if (sc.n_prims > 0 && t0 < t1) {
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
      hc[0] = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, ray, t0, t1, en[0]);
      hc[1] = n3.y != kEmptyChild && slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, ray, t0, t1, en[1]);
      const int ch[2] = {n3.x, n3.y};
      if ((ch[0] < 0 && ~ch[0] >= sc.n_prims) || (ch[1] < 0 && ch[1] != kEmptyChild && ~ch[1] >= sc.n_prims)) {
        st = UGP_RAY_BAD_NODE;
        break;
      }
      for (int c = 0; c < 2; ++c) {
        if (!hc[c] || ch[c] >= 0) continue;
        hc[c] = false;
        PrimHit h;
        if (!prim_test(sc.prims, sc.wlo, ~ch[c], ray, t0, t1, sc.k2, ex, h)) continue;
        if (count < cap) {
          ids[r * cap + count] = h.id;
          aa[r * cap + count] = h.a;
          bb[r * cap + count] = h.b;
        }
        ++count;
      }
      if (hc[0] && hc[1]) {
        if (sp == kTrStack) {
          st = UGP_RAY_STACK_OVERFLOW;
          break;
        }
        stk[sp * kTrBlock + tid] = ch[1];
        ++sp;
        node = ch[0];
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
  cnt[r] = count;
  if (st_out) st_out[r] = st;
}

TraceScene trace_scene(const ugp_bvh* b) {
  TraceScene s;
  s.nodes = b->nodes;
  s.nodes4 = b->nodes4;
  s.prims = b->prims;
  s.wlo = b->wlo;
  s.n_prims = b->n_prims;
  s.n_nodes = b->n_nodes;
  s.k2 = b->k2;
  return s;
}

}  // namespace ugp

using namespace ugp;

ugp_status ugp::check_rays(const char* fn, const ugp_bvh* bvh, int64_t n, const void* o3, const void* d3,
                           const void* t0, const void* t1) {
  if (!valid_bvh(bvh)) return fail(UGP_ERR_NOT_BUILT, "%s: invalid BVH handle", fn);
  if (n < 0 || n > (int64_t(1) << 40)) return fail(UGP_ERR_INVALID_ARG, "%s: n_rays %lld out of range", fn, (long long)n);
  if (n > 0 && (!o3 || !d3 || !t0 || !t1)) return fail(UGP_ERR_INVALID_ARG, "%s: NULL ray array", fn);
  return UGP_OK;
}

extern "C" ugp_status ugp_trace_transmittance(const ugp_bvh* bvh, int64_t n_rays, const float* o3,
                                              const float* d3, const float* t0, const float* t1,
                                              const int32_t* exclude_prim, float* T_out,
                                              uint8_t* status_out, void* stream) {
  clear_error();
  ugp_status s = check_rays("ugp_trace_transmittance", bvh, n_rays, o3, d3, t0, t1);
  if (s != UGP_OK) return s;
  if (n_rays > 0 && !T_out) return fail(UGP_ERR_INVALID_ARG, "ugp_trace_transmittance: NULL T_out");
  if (n_rays == 0) return UGP_OK;
  return launch_transmittance(trace_scene(bvh), n_rays, o3, d3, t0, t1, exclude_prim, T_out, status_out,
                              static_cast<cudaStream_t>(stream));
}

extern "C" ugp_status ugp_collect_hits(const ugp_bvh* bvh, int64_t n_rays, const float* o3, const float* d3,
                                       const float* t0, const float* t1, const int32_t* exclude_prim,
                                       int32_t cap, int32_t* ids_out, float* a_out, float* b_out,
                                       int32_t* count_out, uint8_t* status_out, void* stream) {
  clear_error();
  ugp_status s = check_rays("ugp_collect_hits", bvh, n_rays, o3, d3, t0, t1);
  if (s != UGP_OK) return s;
  if (cap < 0) return fail(UGP_ERR_INVALID_ARG, "ugp_collect_hits: cap < 0");
  if (n_rays > 0 && (!count_out || (cap > 0 && (!ids_out || !a_out || !b_out))))
    return fail(UGP_ERR_INVALID_ARG, "ugp_collect_hits: NULL output array");
  if (n_rays == 0) return UGP_OK;
  const unsigned grid = unsigned((n_rays + kTrBlock - 1) / kTrBlock);
  prof_begin(kStQuery, static_cast<cudaStream_t>(stream));
  k_collect_hits<<<grid, kTrBlock, 0, static_cast<cudaStream_t>(stream)>>>(
      trace_scene(bvh), n_rays, o3, d3, t0, t1, exclude_prim, cap, ids_out, a_out, b_out, count_out, status_out);
  prof_end(kStQuery, static_cast<cudaStream_t>(stream));
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

namespace ugp {

ugp_status launch_transmittance(const TraceScene& sc, int64_t n, const float* o3, const float* d3,
                                const float* t0, const float* t1, const int32_t* excl, float* T,
                                uint8_t* st, cudaStream_t stream) {
  const unsigned grid = unsigned((n + kTrBlock - 1) / kTrBlock);
  unsigned long long* ctr = trace_counters();
  prof_begin(kStQuery, stream);
  if (ctr)
    k_transmittance<true><<<grid, kTrBlock, 0, stream>>>(sc, n, o3, d3, t0, t1, excl, T, st, ctr);
  else
    k_transmittance<false><<<grid, kTrBlock, 0, stream>>>(sc, n, o3, d3, t0, t1, excl, T, st, ctr);
  prof_end(kStQuery, stream);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

}  // namespace ugp
