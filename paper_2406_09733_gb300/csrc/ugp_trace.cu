// Scene queries of Sec. 5: transmittance evaluation (Sec. 5.3, Eq. 7) and exact
// free-flight distribution sampling (Sec. 5.2, Eq. 8-10) over the BVH.
//
// One thread per ray.  Traversal stacks live in shared memory, one column per thread
// (stack[level][thread]) so neighbouring threads hit neighbouring banks.
#include "ugp_gauss.cuh"
#include "ugp_trace.cuh"

namespace ugp {

// ----------------------------------------------------------------------------------------
// Transmittance: T = max(0, 1 - 1/2 sum_k I_k(clip_k)).  Any traversal order gives the same
// sum; nearest-child-first only makes the early exit at sum >= 1 come sooner.
template <bool STATS>
__global__ void __launch_bounds__(kTrBlock)
k_transmittance(TraceScene sc, int64_t n_rays, const float* __restrict__ o3, const float* __restrict__ d3,
                const float* __restrict__ t0a, const float* __restrict__ t1a,
                const int32_t* __restrict__ excl, float* __restrict__ T_out, uint8_t* __restrict__ st_out,
                unsigned long long* __restrict__ ctr) {
  __shared__ int stk[kTrStack * kTrBlock];
  const int tid = threadIdx.x;
  const int64_t r = int64_t(blockIdx.x) * kTrBlock + tid;
  if (r >= n_rays) return;
  const Ray ray = make_ray(ld3(o3, r), ld3(d3, r));
  const float t0 = __ldg(t0a + r), t1 = __ldg(t1a + r);
  const int ex = excl ? __ldg(excl + r) : -1;
  unsigned n_nodes = 0, n_prims = 0;
  float acc = 0.f;
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
      ++n_nodes;
      float e0, e1;
      bool h0 = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, ray, t0, t1, e0);
      bool h1 = n3.y != kEmptyChild && slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, ray, t0, t1, e1);
      PrimHit h;
      if ((n3.x < 0 && ~n3.x >= sc.n_prims) || (n3.y < 0 && n3.y != kEmptyChild && ~n3.y >= sc.n_prims)) {
        st = UGP_RAY_BAD_NODE;
        break;
      }
      if (h0 && n3.x < 0) {
        ++n_prims;
        if (prim_test(sc.prims, ~n3.x, ray, t0, t1, sc.k2, ex, h))
          acc += half_integral(h.a, h.b, h.tn, h.ts, h.s, h.e0);
        h0 = false;
      }
      if (h1 && n3.y < 0) {
        ++n_prims;
        if (prim_test(sc.prims, ~n3.y, ray, t0, t1, sc.k2, ex, h))
          acc += half_integral(h.a, h.b, h.tn, h.ts, h.s, h.e0);
        h1 = false;
      }
      if (acc >= 1.f) break;  // saturated: T = 0 whatever follows
      if (h0 && h1) {
        const bool first0 = e0 <= e1;
        if (sp == kTrStack) {
          st = UGP_RAY_STACK_OVERFLOW;
          break;
        }
        stk[sp * kTrBlock + tid] = first0 ? n3.y : n3.x;
        ++sp;
        node = first0 ? n3.x : n3.y;
      } else if (h0) {
        node = n3.x;
      } else if (h1) {
        node = n3.y;
      } else {
        if (sp == 0) break;
        --sp;
        node = stk[sp * kTrBlock + tid];
      }
    }
  }
  T_out[r] = fmaxf(0.f, 1.f - acc);
  if (st_out) st_out[r] = st;
  if (STATS) add_counters(ctr, n_nodes, n_prims, 1u, 1u);
}

// ----------------------------------------------------------------------------------------
// Free-flight sampling.
//
// The exact, order-free definition: with the clipped intervals [a_k, b_k] and
// F(t) = 1/2 sum_k I_k(a_k, min(t, b_k)), escape if F(t1) <= u, else solve F(t_u) = u and
// pick k among the intervals containing t_u with probability G_k(x_{t_u}) / sum G.
//
// A BVH gives no front-to-back order (the paper's reason for a kd-tree, Sec. 5.1), so the
// kernel works in rounds over a window [t_c, t_w]:
//   * a traversal collects the kK - nC new intervals with the smallest (a, index) keys after
//     a cursor, keeping them sorted in a per-thread shared-memory buffer; nC intervals
//     that were already active at t_c are carried from the previous round;
//   * every interval not kept starts at or after t_w (the smallest start that was dropped,
//     or the entry of a pruned subtree), so F on [t_c, t_w] is known exactly from the buffer;
//   * if F crosses u inside the window, a safeguarded Newton iteration (F' = 1/2 sum G, Eq. 9)
//     finds t_u and the primitive is chosen; otherwise F and t_c advance to t_w.
// Each round keeps at least one new interval, so the number of rounds is bounded by the number
// of intervals along the ray; kFFMaxRounds caps it.
struct FFSmem {
  float a[kK][kFFBlock];
  float b[kK][kFFBlock];
  float tn[kK][kFFBlock];
  float ts[kK][kFFBlock];
  float s[kK][kFFBlock];
  float e0[kK][kFFBlock];
  int id[kK][kFFBlock];
  int stk[kFFStack][kFFBlock];
};

__device__ __forceinline__ bool key_less(float a0, int i0, float a1, int i1) {
  return a0 < a1 || (a0 == a1 && i0 < i1);
}

#define FB(arr, i) sm.arr[(i)][tid]

template <bool STATS>
__global__ void __launch_bounds__(kFFBlock)
k_free_flight(TraceScene sc, int64_t n_rays, const float* __restrict__ o3, const float* __restrict__ d3,
              const float* __restrict__ t0a, const float* __restrict__ t1a, const float* __restrict__ ua,
              const float* __restrict__ u2a, const int32_t* __restrict__ excl,
              int32_t* __restrict__ prim_out, float* __restrict__ tu_out, float* __restrict__ tsp_out,
              uint8_t* __restrict__ st_out, unsigned long long* __restrict__ ctr) {
  __shared__ FFSmem sm;
  const int tid = threadIdx.x;
  const int64_t r = int64_t(blockIdx.x) * kFFBlock + tid;
  if (r >= n_rays) return;
  const Ray ray = make_ray(ld3(o3, r), ld3(d3, r));
  const float t0 = __ldg(t0a + r), t1 = __ldg(t1a + r);
  const float u = __ldg(ua + r), u2 = __ldg(u2a + r);
  const int ex = excl ? __ldg(excl + r) : -1;
  unsigned n_nodes = 0, n_prims = 0, n_rounds = 0;
  uint8_t st = UGP_RAY_OK;
  int out_prim = -1;
  float out_tu = t1, out_tsp = t1;

  float t_c = t0, F_c = 0.f;
  float cur_a = -INFINITY;
  int cur_id = -1;
  int nC = 0;
  bool done = !(sc.n_prims > 0 && t0 < t1);
  while (!done) {
    if (n_rounds >= kFFMaxRounds) {
      st = UGP_RAY_ITER_LIMIT;
      break;
    }
    ++n_rounds;
    const int cap = kK - nC;
    if (cap == 0) {
      st = UGP_RAY_BUFFER_OVERFLOW;
      break;
    }
    // ---- collection traversal over [t_c, t1] ----
    int nNew = 0;
    float limit = t1;    // prune subtrees starting after this once the buffer is full
    float t_next = t1;   // smallest start of anything not kept
    int sp = 0, node = 0;
    while (true) {
      if (unsigned(node) >= unsigned(sc.n_nodes)) {
        st = UGP_RAY_BAD_NODE;
        break;
      }
      const float4* nd = sc.nodes + 4 * node;
      const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
      const int4 n3 = __ldg(reinterpret_cast<const int4*>(nd) + 3);
      ++n_nodes;
      float en[2];
      bool hc[2];
      hc[0] = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, ray, t_c, t1, en[0]);
      hc[1] = n3.y != kEmptyChild && slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, ray, t_c, t1, en[1]);
      const int ch[2] = {n3.x, n3.y};
      if ((ch[0] < 0 && ~ch[0] >= sc.n_prims) || (ch[1] < 0 && ch[1] != kEmptyChild && ~ch[1] >= sc.n_prims)) {
        st = UGP_RAY_BAD_NODE;
        break;
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!hc[c]) continue;
        if (en[c] > limit) {  // everything below starts after the kept set
          t_next = fminf(t_next, en[c]);
          hc[c] = false;
          continue;
        }
        if (ch[c] >= 0) continue;
        hc[c] = false;
        ++n_prims;
        PrimHit h;
        if (!prim_test(sc.prims, ~ch[c], ray, t0, t1, sc.k2, ex, h)) continue;
        if (h.b <= t_c) continue;                                // finished before the window
        if (!key_less(cur_a, cur_id, h.a, h.id)) continue;       // kept in an earlier round
        int pos;
        if (nNew < cap) {
          pos = nC + nNew;
          ++nNew;
        } else {
          const int last = nC + nNew - 1;
          if (!key_less(h.a, h.id, FB(a, last), FB(id, last))) {
            t_next = fminf(t_next, h.a);
            continue;
          }
          t_next = fminf(t_next, FB(a, last));  // the evicted interval starts here
          pos = last;
        }
        // insertion into the sorted new-interval range [nC, pos]
        while (pos > nC && key_less(h.a, h.id, FB(a, pos - 1), FB(id, pos - 1))) {
          FB(a, pos) = FB(a, pos - 1);
          FB(b, pos) = FB(b, pos - 1);
          FB(tn, pos) = FB(tn, pos - 1);
          FB(ts, pos) = FB(ts, pos - 1);
          FB(s, pos) = FB(s, pos - 1);
          FB(e0, pos) = FB(e0, pos - 1);
          FB(id, pos) = FB(id, pos - 1);
          --pos;
        }
        FB(a, pos) = h.a;
        FB(b, pos) = h.b;
        FB(tn, pos) = h.tn;
        FB(ts, pos) = h.ts;
        FB(s, pos) = h.s;
        FB(e0, pos) = h.e0;
        FB(id, pos) = h.id;
        if (nNew == cap) limit = FB(a, nC + nNew - 1);
      }
      if (hc[0] && hc[1]) {
        const bool first0 = en[0] <= en[1];
        if (sp == kFFStack) {
          st = UGP_RAY_STACK_OVERFLOW;
          break;
        }
        FB(stk, sp) = first0 ? ch[1] : ch[0];
        ++sp;
        node = first0 ? ch[0] : ch[1];
      } else if (hc[0]) {
        node = ch[0];
      } else if (hc[1]) {
        node = ch[1];
      } else {
        if (sp == 0) break;
        --sp;
        node = FB(stk, sp);
      }
    }
    if (st != UGP_RAY_OK) break;
    const int nE = nC + nNew;
    const float t_w = fmaxf(t_next, t_c);
    // ---- F over the window [t_c, t_w] ----
    float dF = 0.f;
    for (int e = 0; e < nE; ++e) {
      const float lo = fmaxf(FB(a, e), t_c), hi = fminf(FB(b, e), t_w);
      if (lo < hi) dF += half_integral(lo, hi, FB(tn, e), FB(ts, e), FB(s, e), FB(e0, e));
    }
    if (F_c + dF > u) {
      // ---- root of F(t) = u in [t_c, t_w], bracketed Newton ----
      // Safeguarded Newton: a Newton step is taken only if it stays inside the bracket and
      // the previous-but-one step shows it converges at least as fast as bisection.
      float lo = t_c, hi = t_w, t = 0.5f * (t_c + t_w);
      float dx_old = hi - lo, dx = dx_old;
      bool conv = false;
      for (int it = 0; it < kFFNewtonIters; ++it) {
        float f = F_c - u, fp = 0.f;
        for (int e = 0; e < nE; ++e) {
          const float x0 = fmaxf(FB(a, e), t_c), x1 = fminf(FB(b, e), t);
          if (x0 < x1) f += half_integral(x0, x1, FB(tn, e), FB(ts, e), FB(s, e), FB(e0, e));
          if (FB(a, e) <= t && t <= FB(b, e))
            fp += 0.5f * gauss_at(t, FB(tn, e), FB(ts, e), FB(s, e), FB(e0, e));
        }
        if (f == 0.f) { conv = true; break; }
        if (f < 0.f) lo = t; else hi = t;
        if (!(nextafterf(lo, INFINITY) < hi)) { conv = true; break; }  // bracket is one ulp wide
        const float tn_ = fp > 0.f ? t - f / fp : lo;
        float tnew;
        if (fp > 0.f && tn_ > lo && tn_ < hi && fabsf(2.f * f) <= fabsf(dx_old * fp)) {
          dx_old = dx;
          dx = f / fp;
          tnew = tn_;
        } else {
          dx_old = dx;
          dx = 0.5f * (hi - lo);
          tnew = lo + dx;
        }
        if (tnew == t) { conv = true; break; }
        t = tnew;
      }
      if (!conv) st = UGP_RAY_SOLVE_LIMIT;
      // ---- choose among the intervals containing t, proportional to G, ascending index ----
      float tot = 0.f;
      for (int e = 0; e < nE; ++e)
        if (FB(a, e) <= t && t <= FB(b, e)) tot += gauss_at(t, FB(tn, e), FB(ts, e), FB(s, e), FB(e0, e));
      const float target = u2 * tot;
      float cum = 0.f;
      int last_id = -1, pick = -1, pick_any = -1;
      while (true) {
        int best = -1, best_id = INT32_MAX;
        for (int e = 0; e < nE; ++e) {
          const int idv = FB(id, e);
          if (FB(a, e) <= t && t <= FB(b, e) && idv > last_id && idv < best_id) {
            best = e;
            best_id = idv;
          }
        }
        if (best < 0) break;
        pick_any = best;
        cum += gauss_at(t, FB(tn, best), FB(ts, best), FB(s, best), FB(e0, best));
        last_id = best_id;
        if (cum > target) {
          pick = best;
          break;
        }
      }
      if (pick < 0) pick = pick_any;  // rounding left the sum just short of u2 * total
      if (pick >= 0) {
        out_prim = FB(id, pick);
        out_tu = t;
        out_tsp = 0.5f * (FB(a, pick) + FB(b, pick));
      }
      done = true;
    } else {
      F_c += dF;
      t_c = t_w;
      if (t_w >= t1) {
        done = true;  // escape
      } else {
        if (nNew > 0) {
          cur_a = FB(a, nE - 1);
          cur_id = FB(id, nE - 1);
        }
        // carry the intervals still active after t_w
        int m = 0;
        for (int e = 0; e < nE; ++e) {
          if (FB(b, e) > t_w) {
            if (m != e) {
              FB(a, m) = FB(a, e);
              FB(b, m) = FB(b, e);
              FB(tn, m) = FB(tn, e);
              FB(ts, m) = FB(ts, e);
              FB(s, m) = FB(s, e);
              FB(e0, m) = FB(e0, e);
              FB(id, m) = FB(id, e);
            }
            ++m;
          }
        }
        nC = m;
      }
    }
  }
  prim_out[r] = out_prim;
  tu_out[r] = out_tu;
  tsp_out[r] = out_tsp;
  if (st_out) st_out[r] = st;
  if (STATS) add_counters(ctr, n_nodes, n_prims, 1u, n_rounds);
}

#undef FB

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
        if (!prim_test(sc.prims, ~ch[c], ray, t0, t1, sc.k2, ex, h)) continue;
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
  s.prims = b->prims;
  s.n_prims = b->n_prims;
  s.n_nodes = b->n_nodes;
  s.k2 = b->k2;
  return s;
}

}  // namespace ugp

using namespace ugp;

static ugp_status check_rays(const char* fn, const ugp_bvh* bvh, int64_t n, const void* o3, const void* d3,
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

extern "C" ugp_status ugp_sample_free_flight(const ugp_bvh* bvh, int64_t n_rays, const float* o3,
                                             const float* d3, const float* t0, const float* t1,
                                             const float* u, const float* u2, const int32_t* exclude_prim,
                                             int32_t* prim_out, float* t_u_out, float* t_spawn_out,
                                             uint8_t* status_out, void* stream) {
  clear_error();
  ugp_status s = check_rays("ugp_sample_free_flight", bvh, n_rays, o3, d3, t0, t1);
  if (s != UGP_OK) return s;
  if (n_rays > 0 && (!u || !u2 || !prim_out || !t_u_out || !t_spawn_out))
    return fail(UGP_ERR_INVALID_ARG, "ugp_sample_free_flight: NULL uniform or output array");
  if (n_rays == 0) return UGP_OK;
  return launch_free_flight(trace_scene(bvh), n_rays, o3, d3, t0, t1, u, u2, exclude_prim, prim_out, t_u_out,
                            t_spawn_out, status_out, static_cast<cudaStream_t>(stream));
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
  k_collect_hits<<<grid, kTrBlock, 0, static_cast<cudaStream_t>(stream)>>>(
      trace_scene(bvh), n_rays, o3, d3, t0, t1, exclude_prim, cap, ids_out, a_out, b_out, count_out, status_out);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

namespace ugp {

ugp_status launch_transmittance(const TraceScene& sc, int64_t n, const float* o3, const float* d3,
                                const float* t0, const float* t1, const int32_t* excl, float* T,
                                uint8_t* st, cudaStream_t stream) {
  const unsigned grid = unsigned((n + kTrBlock - 1) / kTrBlock);
  unsigned long long* ctr = trace_counters();
  if (ctr)
    k_transmittance<true><<<grid, kTrBlock, 0, stream>>>(sc, n, o3, d3, t0, t1, excl, T, st, ctr);
  else
    k_transmittance<false><<<grid, kTrBlock, 0, stream>>>(sc, n, o3, d3, t0, t1, excl, T, st, ctr);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

ugp_status launch_free_flight(const TraceScene& sc, int64_t n, const float* o3, const float* d3,
                              const float* t0, const float* t1, const float* u, const float* u2,
                              const int32_t* excl, int32_t* prim, float* tu, float* tsp, uint8_t* st,
                              cudaStream_t stream) {
  const unsigned grid = unsigned((n + kFFBlock - 1) / kFFBlock);
  unsigned long long* ctr = trace_counters();
  if (ctr)
    k_free_flight<true><<<grid, kFFBlock, 0, stream>>>(sc, n, o3, d3, t0, t1, u, u2, excl, prim, tu, tsp, st, ctr);
  else
    k_free_flight<false><<<grid, kFFBlock, 0, stream>>>(sc, n, o3, d3, t0, t1, u, u2, excl, prim, tu, tsp, st, ctr);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

}  // namespace ugp
