// Warp-per-ray finish of free-flight sampling: every ray whose root the scan has bracketed in
// [lo, hi] (with F(lo) = Flo) is finished here.
//
// For each queued ray one warp
//   1. collects every clipped interval meeting [lo, hi] into a per-warp shared-memory list: from
//      the primitive slots the per-thread scan recorded for the ray when that list is complete
//      (32 re-tests per step), else by a warp-parallel traversal that pops up to 32 nodes from a
//      shared stack per step, one per lane, pushing the hit internal children and appending hit
//      leaves with ballot-ranked slots;
//   2. if the list fits, solves F(t_u) = u (Eq. 10) on the bracket by Newton's method, kept in a
//      shrinking bracket by false-position steps (Illinois rule) and finally by bisection, with
//      F and F' = 1/2 sum G (Eq. 9) summed across lanes, and draws the primitive with the
//      exponential race (smallest E_k / G_k(x_{t_u})) as a warp argmin;
//   3. otherwise hands the ray to a second kernel in which one warp per block holds up to 1024
//      intervals (rays through the cores of dense clusters, where hundreds of ellipsoids contain
//      the root itself, so no narrower bracket would hold fewer); beyond that, it adds every
//      interval's contribution to 32 sub-bins of the bracket (shared-memory atomics), moves the
//      bracket to the crossing sub-bin and repeats.
// The result is the same function of (u, u2) as the per-thread paths: the same F, root and race.
// It is also bit-for-bit independent of the order in which the intervals were collected (the
// scan's slot list follows its warp's schedule): the solve sums the intervals in primitive-id
// order, and the sub-bins are fixed-point integers.
#include "ugp_dense.cuh"
#include "ugp_gauss.cuh"
#include "ugp_philox.cuh"

namespace ugp {
namespace {

constexpr int kDWarps = 4;     // rays in flight per block
constexpr int kDCap = 256;     // intervals one warp holds
constexpr int kDCapH = 1024;   // intervals the warp of the heavy-ray kernel holds
constexpr int kDLevels = 8;    // bracket refinements when the intervals do not fit
constexpr int kDNewton = 64;
constexpr int kDBisectAfter = 24;  // Newton / false-position steps before plain bisection
constexpr float kNewtonStep = 1e-6f;   // relative Newton step that ends the iteration
constexpr float kNewtonFloor = 1e-3f;  // distance scale below which the step is taken absolute
constexpr unsigned kFull = 0xffffffffu;

template <int kCapacity>
struct WarpSmemT {
  static constexpr int kCap = kCapacity;
  static constexpr int kStack = 2 * kCap > 512 ? 2 * kCap : 512;  // shared traversal stack
  float a[kCap], b[kCap], tn[kCap], ts[kCap], s[kCap], e0[kCap], th[kCap];
  int id[kCap];  // index with the end-point flags (pack_id)
  int stk[kStack];  // traversal stack; after a collection, keys and the id order (stk + kCap)
  unsigned long long bin[32];  // sub-bins of step 3, units of 2^-40
};
using WarpSmem = WarpSmemT<kDCap>;
using WarpSmemH = WarpSmemT<kDCapH>;
static_assert(kDCap >= kListCap, "a ray with more intervals than the main pass holds has overflowed its list");
constexpr float kSubScale = 1099511627776.f;           // 2^40
constexpr float kSubUnit = 9.094947017729282e-13f;     // 2^-40

// Orders the n <= kDCap collected intervals by primitive id (ids along one ray are distinct):
// each interval's rank is the number of smaller ids, counted with shuffles when the intervals
// fit one or two per lane and with broadcast shared-memory reads otherwise. On return ord[r]
// (the second half of the traversal stack) is the interval of rank r.
template <class WS>
__device__ void order_by_id(WS& W, int n, int lane) {
  int* key = W.stk;
  int* ord = W.stk + WS::kCap;
  if (n <= 32) {
    const int k = lane < n ? unpack_id(W.id[lane]) : INT32_MAX;
    int r = 0;
#pragma unroll 4
    for (int m = 0; m < n; ++m) r += __shfl_sync(kFull, k, m) < k ? 1 : 0;
    if (lane < n) ord[r] = lane;
  } else if (n <= 64) {
    const int k0 = unpack_id(W.id[lane]);
    const int k1 = lane + 32 < n ? unpack_id(W.id[lane + 32]) : INT32_MAX;
    int r0 = 0, r1 = 0;
#pragma unroll 4
    for (int m = 0; m < 32; ++m) {
      const int a = __shfl_sync(kFull, k0, m), b = __shfl_sync(kFull, k1, m);
      r0 += (a < k0 ? 1 : 0) + (b < k0 ? 1 : 0);
      r1 += (a < k1 ? 1 : 0) + (b < k1 ? 1 : 0);
    }
    ord[r0] = lane;
    if (lane + 32 < n) ord[r1] = lane + 32;
  } else {
    for (int i = lane; i < n; i += 32) key[i] = unpack_id(W.id[i]);
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const int k = key[i];
      int r = 0;
#pragma unroll 4
      for (int m = 0; m < n; ++m) r += key[m] < k ? 1 : 0;
      ord[r] = i;
    }
  }
  __syncwarp();
}

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return __shfl_sync(kFull, v, 0);  // lane 0's sum, identical on every lane
}

// Warp-parallel traversal of the leaves whose boxes meet [lo, hi]; `leaf(slot)` is called by all
// lanes together (slot < 0 for lanes without a leaf), twice per step.
template <class WS, class LeafFn>
__device__ void warp_traverse(WS& W, const TraceScene& sc, const Ray& ray, float lo, float hi, int lane,
                              uint8_t& st, unsigned& nn, LeafFn&& leaf) {
  int size = 1;
  if (lane == 0) W.stk[0] = 0;
  __syncwarp();
  while (size > 0) {
    const int m = min(size, 32);
    const int node = lane < m ? W.stk[size - 1 - lane] : -1;
    size -= m;
    __syncwarp();
    int ch[2] = {-1, -1};
    bool h[2] = {false, false};
    bool bad = false;
    if (node >= 0) {
      if (node >= sc.n_nodes) {
        bad = true;
      } else {
        const float4* nd = sc.nodes + 4 * node;
        const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
        const int4 n3 = __ldg(reinterpret_cast<const int4*>(nd) + 3);
        ++nn;
        ch[0] = n3.x;
        ch[1] = n3.y;
        bad = (ch[0] < 0 && ~ch[0] >= sc.n_prims) || (ch[1] < 0 && ch[1] != kEmptyChild && ~ch[1] >= sc.n_prims);
        float en;
        h[0] = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, ray, lo, hi, en);
        h[1] = ch[1] != kEmptyChild && slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, ray, lo, hi, en);
      }
    }
    if (__any_sync(kFull, bad)) {
      st = UGP_RAY_BAD_NODE;
      return;
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const bool push = h[c] && ch[c] >= 0;
      const unsigned mask = __ballot_sync(kFull, push);
      if (push) {
        const int off = size + __popc(mask & ((1u << lane) - 1u));
        if (off < WS::kStack) W.stk[off] = ch[c];
      }
      size += __popc(mask);
    }
    if (size > WS::kStack) {
      st = UGP_RAY_STACK_OVERFLOW;
      return;
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 2; ++c) leaf((h[c] && ch[c] < 0) ? ~ch[c] : -1);
    __syncwarp();
  }
}

// Calls `leaf(slot)` on all lanes for every candidate primitive of [lo, hi]: from the ray's
// recorded slot list when it is complete (32 slots per step), else by a warp traversal.
template <class WS, class LeafFn>
__device__ void for_each_candidate(WS& W, const TraceScene& sc, const Ray& ray, float lo, float hi, int lane,
                                   uint8_t& st, unsigned& nn, const int* list, int nlist, LeafFn&& leaf) {
  if (list) {
    for (int base = 0; base < nlist; base += 32) {
      const int e = base + lane;
      leaf(e < nlist ? __ldg(list + e) : -1);
    }
    __syncwarp();
    return;
  }
  warp_traverse(W, sc, ray, lo, hi, lane, st, nn, leaf);
}

// Finishes the ray in slot j of the table with the warp's interval buffer W. In the main pass
// (kHeavy false) a ray with more intervals than W holds is appended to the heavy-ray list (when
// the queue has one) and left to the heavy-ray kernel, which writes its results.
template <bool kHeavy, class WS>
__device__ void finish_ray(WS& W, const TraceScene& sc0, const DenseQueue& q, int j, int lane, int* __restrict__ prim_out,
                           float* __restrict__ tu_out, float* __restrict__ tsp_out, uint8_t* __restrict__ st_out,
                           int spawn_mode, unsigned long long* stats, unsigned long long* rays_err) {
  constexpr int kCap = WS::kCap;
  {
    const TraceScene sc = q.scenes ? q.scenes[q.scene[j]] : sc0;
    const int idx = q.idx[j];
    float lo = q.lo[j], hi = q.hi[j], Flo = q.Flo[j];
    const float u = q.u[j], u2 = q.u2[j], t0 = q.t0[j], t1 = q.t1[j];
    const int excl = q.excl[j];
    const int nlist = q.nlist[j];
    const int* list = (q.list && nlist <= kListCap) ? q.list + size_t(idx) * kListCap : nullptr;
    const Ray ray = make_ray(make_float3(q.ox[j], q.oy[j], q.oz[j]), make_float3(q.dx[j], q.dy[j], q.dz[j]));
    uint8_t st = UGP_RAY_OK;
    unsigned nn = 0, np = 0;
    int out_prim = -1;
    float out_tu = t1, out_tsp = t1;
    bool done = false, deferred = false;
    for (int level = 0; level < kDLevels && !done && st == UGP_RAY_OK; ++level) {
      // ---- 1. collect the intervals meeting [lo, hi]
      int n = 0;
      for_each_candidate(W, sc, ray, lo, hi, lane, st, nn, list, nlist, [&](int slot) {
        PrimHit hh;
        bool ok = false;
        if (slot >= 0) {
          ++np;
          ok = prim_test(sc.prims, sc.wlo, slot, ray, t0, t1, sc.k2, excl, hh) && fmaxf(hh.a, lo) < fminf(hh.b, hi);
        }
        const unsigned mask = __ballot_sync(kFull, ok);
        if (ok) {
          const int i = n + __popc(mask & ((1u << lane) - 1u));
          if (i < kCap) {
            W.a[i] = hh.a; W.b[i] = hh.b; W.tn[i] = hh.tn; W.ts[i] = hh.ts;
            W.s[i] = hh.s; W.e0[i] = hh.e0; W.th[i] = hh.th; W.id[i] = pack_id(hh);
          }
        }
        n += __popc(mask);
      });
      __syncwarp();
      if (st != UGP_RAY_OK) break;
      if (n <= kCap) {
        // ---- 2. root of F = u on [lo, min(hi, last interval end)], then the race at t_u
        // The main pass orders the intervals by id: whether a ray's list overflowed (list or
        // traversal) follows its warp's schedule. A heavy ray always overflowed its list (it
        // has more intervals than the list holds), so its traversal order is already a
        // function of the ray alone.
        int* ord = W.stk + kCap;
        if (kHeavy) {
          for (int i = lane; i < n; i += 32) ord[i] = i;
          __syncwarp();
        } else {
          order_by_id(W, n, lane);
        }
        float bmax = lo;
        for (int e = lane; e < n; e += 32) bmax = fmaxf(bmax, W.b[e]);
        for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(kFull, bmax, o));
        float hi_e = fminf(hi, bmax);
        const float w_lo = lo;
        // full[r]: the term of the interval of rank r at t = hi_e, which for an interval ending at
        // or before hi_e is its whole contribution; later evaluations reuse it for every interval
        // that ends before t, so only the intervals containing t need the erf.
        float* full = reinterpret_cast<float*>(W.stk);
        auto term = [&](int e, float t) {
          const float x0 = fmaxf(W.a[e], w_lo), x1 = fminf(W.b[e], t);
          const int p = W.id[e];
          return x0 < x1 ? seg_half_integral(x0, x1, W.a[e], W.b[e], packed_a_end(p), packed_b_end(p), W.tn[e],
                                             W.ts[e], W.s[e], W.e0[e], W.th[e])
                         : 0.f;
        };
        auto evalF = [&](float t, float& f, float& fp) {
          float fl = 0.f, fpl = 0.f;
          for (int r = lane; r < n; r += 32) {
            const int e = ord[r];
            const float a = W.a[e], b = W.b[e];
            fl += b <= t ? full[r] : term(e, t);
            if (a <= t && t <= b) fpl += 0.5f * gauss_at(t, W.tn[e], W.ts[e], W.s[e], W.e0[e]);
          }
          f = Flo - u + warp_sum(fl);
          fp = warp_sum(fpl);
        };
        float fh;
        {
          float fl = 0.f;
          for (int r = lane; r < n; r += 32) {
            const float v = term(ord[r], hi_e);
            full[r] = v;
            fl += v;
          }
          fh = Flo - u + warp_sum(fl);
          __syncwarp();
        }
        float t;
        if (!(fh > 0.f)) {
          t = hi_e;  // rounding placed the crossing at the end of the bracket
        } else {
          // Newton's method safeguarded by a bracket [a0, b0] with f(a0) < 0 < f(b0); a step that
          // leaves the bracket or does not shrink fast enough is replaced by a false-position step
          // with the Illinois rule (F is monotone and S-shaped across thin primitives, where plain
          // Newton overshoots and bisection would crawl)
          float a0 = lo, b0 = hi_e, fa = Flo - u, fb = fh;
          int moved = 0;  // -1: a0 moved last, +1: b0 moved last
          t = a0 - fa * (b0 - a0) / (fb - fa);
          if (!(t > a0 && t < b0)) t = 0.5f * (a0 + b0);
          float dx_old = b0 - a0, dx = dx_old;
          bool conv = false;
          for (int it = 0; it < kDNewton; ++it) {
            float f, fp;
            evalF(t, f, fp);
            if (f == 0.f) { conv = true; break; }
            if (f < 0.f) {
              a0 = t;
              fa = f;
              if (moved < 0) fb *= 0.5f;
              moved = -1;
            } else {
              b0 = t;
              fb = f;
              if (moved > 0) fa *= 0.5f;
              moved = 1;
            }
            if (!(nextafterf(a0, INFINITY) < b0)) { conv = true; break; }
            // a Newton correction below 1e-6 of the distance scale ends the iteration: its own
            // error is of the order of its square (or of itself across a kink of F'), far below
            // the 1e-5 accuracy asked (taken even where the shrink safeguard below would refuse
            // the step, which near the root only reflects the rounding noise of f)
            if (fp > 0.f && fabsf(f) <= kNewtonStep * fmaxf(fabsf(t), kNewtonFloor) * fp) {
              const float tn = t - f / fp;
              if (tn > a0 && tn < b0) t = tn;
              conv = true;
              break;
            }
            const float tn = fp > 0.f ? t - f / fp : a0;
            float tnew;
            // past kDBisectAfter steps only bisection: the bracket then collapses to adjacent
            // floats within the iteration bound, whatever F looks like
            const bool bisect = it >= kDBisectAfter;
            if (!bisect && fp > 0.f && tn > a0 && tn < b0 && fabsf(2.f * f) <= fabsf(dx_old * fp)) {
              dx_old = dx;
              dx = f / fp;
              tnew = tn;
            } else {
              tnew = bisect ? 0.5f * (a0 + b0) : a0 - fa * (b0 - a0) / (fb - fa);
              if (!(tnew > a0 && tnew < b0)) tnew = 0.5f * (a0 + b0);
              dx_old = dx;
              dx = tnew - t;
            }
            if (tnew == t) { conv = true; break; }
            t = tnew;
          }
          if (!conv) st = UGP_RAY_SOLVE_LIMIT;
        }
        // race: smallest E_k / G_k(x_t) among the intervals containing t (ties: smaller index)
        float best = INFINITY;
        int best_id = INT32_MAX, best_e = -1;
        for (int e = lane; e < n; e += 32) {
          if (!(W.a[e] <= t && t <= W.b[e])) continue;
          const int idv = unpack_id(W.id[e]);
          const float key = race_exponential(u2, idv) / gauss_at(t, W.tn[e], W.ts[e], W.s[e], W.e0[e]);
          if (best_e < 0 || key < best || (key == best && idv < best_id)) {
            best = key;
            best_id = idv;
            best_e = e;
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const float ok = __shfl_xor_sync(kFull, best, o);
          const int oi = __shfl_xor_sync(kFull, best_id, o);
          const int oe = __shfl_xor_sync(kFull, best_e, o);
          if (oe >= 0 && (best_e < 0 || ok < best || (ok == best && oi < best_id))) {
            best = ok;
            best_id = oi;
            best_e = oe;
          }
        }
        if (best_e >= 0) {
          out_prim = best_id;
          out_tu = t;
          out_tsp = spawn_mode == 1 ? t : 0.5f * (W.a[best_e] + W.b[best_e]);
        }
        done = true;
      } else if (!kHeavy && q.heavy) {
        deferred = true;  // the heavy-ray kernel holds more intervals
        break;
      } else {
        // ---- 3. too many intervals: shrink the bracket to the crossing sub-bin
        W.bin[lane] = 0ull;
        __syncwarp();
        const float w = (hi - lo) / 32.f;
        auto edge = [&](int k) { return k >= 32 ? hi : lo + w * float(k); };
        for_each_candidate(W, sc, ray, lo, hi, lane, st, nn, list, nlist, [&](int slot) {
          if (slot < 0) return;
          ++np;
          PrimHit hh;
          if (!prim_test(sc.prims, sc.wlo, slot, ray, t0, t1, sc.k2, excl, hh)) return;
          const float x = fmaxf(hh.a, lo), y = fminf(hh.b, hi);
          if (!(x < y)) return;
          int k = min(31, max(0, int((x - lo) / w)));
          while (k > 0 && x < edge(k)) --k;
          while (k < 31 && x >= edge(k + 1)) ++k;
          for (; k < 32 && edge(k) < y; ++k) {
            const float xa = fmaxf(x, edge(k)), ya = fminf(y, edge(k + 1));
            if (xa < ya) {
              const float v = seg_half_integral(xa, ya, hh.a, hh.b, hh.a_end, hh.b_end, hh.tn, hh.ts, hh.s, hh.e0,
                                                hh.th);
              atomicAdd(&W.bin[k], (unsigned long long)__float2ll_rn(fminf(fmaxf(v, 0.f), 4.f) * kSubScale));
            }
          }
        });
        __syncwarp();
        if (st != UGP_RAY_OK) break;
        unsigned long long acc = 0ull;
        int jx = 31;
        for (int k = 0; k < 32; ++k) {
          const unsigned long long nxt = acc + W.bin[k];
          if (float(nxt) * kSubUnit > u - Flo) {
            jx = k;
            break;
          }
          if (k < 31) acc = nxt;
        }
        const float nlo = edge(jx), nhi = edge(jx + 1);
        Flo += float(acc) * kSubUnit;
        lo = nlo;
        hi = nhi;
        __syncwarp();
      }
    }
    const unsigned tn_nodes = __reduce_add_sync(kFull, nn), tn_prims = __reduce_add_sync(kFull, np);
    if (deferred) {
      if (lane == 0) {
        q.heavy[atomicAdd(q.count + 2, 1)] = j;
        if (stats) {
          atomicAdd(stats + 0, (unsigned long long)tn_nodes);
          atomicAdd(stats + 1, (unsigned long long)tn_prims);
        }
      }
      __syncwarp();
      return;
    }
    if (!done && st == UGP_RAY_OK) st = UGP_RAY_ITER_LIMIT;
    if (lane == 0) {
      prim_out[idx] = out_prim;
      tsp_out[idx] = out_tsp;
      if (tu_out) tu_out[idx] = out_tu;
      if (st_out) st_out[idx] = st;
      if (st != UGP_RAY_OK && rays_err) atomicAdd(rays_err, 1ull);
      if (stats) {
        atomicAdd(stats + 0, (unsigned long long)tn_nodes);
        atomicAdd(stats + 1, (unsigned long long)tn_prims);
      }
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(32 * kDWarps) k_dense(TraceScene sc0, DenseQueue q, int64_t n_host,
                                                        const int* n_dev, int* __restrict__ prim_out,
                                                        float* __restrict__ tu_out, float* __restrict__ tsp_out,
                                                        uint8_t* __restrict__ st_out, int spawn_mode,
                                                        unsigned long long* stats, unsigned long long* rays_err) {
  extern __shared__ __align__(16) unsigned char dsm[];
  WarpSmem& W = reinterpret_cast<WarpSmem*>(dsm)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int count = n_dev ? *reinterpret_cast<const volatile int*>(n_dev) : int(n_host);
  const int nwarps = gridDim.x * kDWarps;
  // slot j to warp j mod (warps), so the rays in flight together are neighbours in the table;
  // empty slots are skipped by the whole warp
  for (int j = blockIdx.x * kDWarps + (threadIdx.x >> 5); j < count; j += nwarps) {
    if (__ldg(q.idx + j) < 0) continue;
    finish_ray<false>(W, sc0, q, j, lane, prim_out, tu_out, tsp_out, st_out, spawn_mode, stats, rays_err);
  }
}

// The rays the main pass handed on, one warp per block; q.count[2] of them, in q.heavy.
__global__ void __launch_bounds__(32) k_dense_heavy(TraceScene sc0, DenseQueue q, int* __restrict__ prim_out,
                                                    float* __restrict__ tu_out, float* __restrict__ tsp_out,
                                                    uint8_t* __restrict__ st_out, int spawn_mode,
                                                    unsigned long long* stats, unsigned long long* rays_err) {
  extern __shared__ __align__(16) unsigned char dsm[];
  WarpSmemH& W = *reinterpret_cast<WarpSmemH*>(dsm);
  const int lane = threadIdx.x & 31;
  const int count = *reinterpret_cast<const volatile int*>(q.count + 2);
  for (int h = blockIdx.x; h < count; h += gridDim.x)
    finish_ray<true>(W, sc0, q, q.heavy[h], lane, prim_out, tu_out, tsp_out, st_out, spawn_mode, stats, rays_err);
}

}  // namespace

static int g_dense_grid = 0, g_heavy_grid = 0;

ugp_status dense_prepare() {
  if (g_dense_grid != 0) return UGP_OK;
  const size_t smem = sizeof(WarpSmem) * kDWarps, smem_h = sizeof(WarpSmemH);
  UGP_CUDA_CHECK(cudaFuncSetAttribute(k_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  UGP_CUDA_CHECK(cudaFuncSetAttribute(k_dense_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_h)));
  int dev = 0, sms = 0, per_sm = 0, per_sm_h = 0;
  UGP_CUDA_CHECK(cudaGetDevice(&dev));
  UGP_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  UGP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense, 32 * kDWarps, smem));
  UGP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_h, k_dense_heavy, 32, smem_h));
  if (sms <= 0) sms = 1;
  g_heavy_grid = sms * (per_sm_h > 0 ? per_sm_h : 1);
  g_dense_grid = sms * (per_sm > 0 ? per_sm : 1);
  return UGP_OK;
}

ugp_status launch_dense(const TraceScene& sc, const DenseQueue& q, int64_t n_host, const int* n_dev,
                        int64_t max_slots, int* prim_out, float* t_u_out, float* t_spawn_out, uint8_t* status_out,
                        int spawn_mode, unsigned long long* stats, unsigned long long* rays_err, cudaStream_t stream) {
  const ugp_status ps = dense_prepare();
  if (ps != UGP_OK) return ps;
  const int64_t need = (max_slots + 32 * kDWarps - 1) / (32 * kDWarps);
  const int grid = int(need < g_dense_grid ? (need > 0 ? need : 1) : g_dense_grid);
  const size_t smem = sizeof(WarpSmem) * kDWarps;
  const int64_t need_h = max_slots < g_heavy_grid ? (max_slots > 0 ? max_slots : 1) : g_heavy_grid;
  UGP_CUDA_CHECK(cudaMemsetAsync(q.count + 2, 0, sizeof(int), stream));
  prof_begin(kStDense, stream);
  k_dense<<<grid, 32 * kDWarps, smem, stream>>>(sc, q, n_host, n_dev, prim_out, t_u_out, t_spawn_out, status_out,
                                               spawn_mode, stats, rays_err);
  k_dense_heavy<<<unsigned(need_h), 32, sizeof(WarpSmemH), stream>>>(sc, q, prim_out, t_u_out, t_spawn_out,
                                                                     status_out, spawn_mode, stats, rays_err);
  prof_end(kStDense, stream, 2);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

}  // namespace ugp
