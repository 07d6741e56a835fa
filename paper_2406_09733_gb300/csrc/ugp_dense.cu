// Finish of free-flight sampling: every ray whose root the scan has bracketed in [lo, hi] (with
// F(lo) = Flo) is finished here, in two kernels that differ only in how many intervals they
// hold per ray. Both keep, per interval collected, its whole term on the bracket and erfc(|tau|)
// at its clipped start (with tau's sign), so each Newton evaluation takes one erfc per interval
// that contains t.
//
// Main pass (k_dense): each half-warp (16 lanes) finishes one ray, so a warp works on two rays
// at a time (most brackets hold a few dozen intervals, which would leave lanes of a whole warp
// idle). The half-warp
//   1. rebuilds every clipped interval meeting [lo, hi] from the primitive slots the scan
//      recorded for the ray (16 re-tests per step) into its slice of the warp's shared memory;
//   2. solves F(t_u) = u (Eq. 10) on the bracket by Newton's method, kept in a shrinking bracket
//      by false-position steps (Illinois rule) and finally by bisection, with F and
//      F' = 1/2 sum G (Eq. 9) summed across its lanes, and draws the primitive with the
//      exponential race (smallest E_k / G_k(x_{t_u})) as an argmin across its lanes.
// A ray whose slot list overflowed, or that has more intervals than a half-warp holds (128), goes
// to k_dense_big: one warp per ray rebuilds the intervals from the list or by a warp-parallel
// traversal (up to 32 nodes per step from a shared stack) and solves with 32 lanes. Its intervals
// (up to kBigCap = 2048) live in a slot of global memory that the warp owns, so the pass is not
// held to a few warps per SM by shared memory; rays through the cores of dense clusters need the
// room: there hundreds of ellipsoids contain the root itself, so no narrower bracket would hold
// fewer. Beyond kBigCap every interval's contribution goes to 32 sub-bins of the bracket
// (fixed-point shared-memory atomics), the bracket moves to the crossing sub-bin, and the rebuild
// repeats.
//
// The result is the same function of (u, u2) as the per-thread paths: the same F, root and race.
// It is also bit-for-bit independent of the order in which the intervals were collected and of
// the kernel and lane count that finished the ray (the scan's slot list, and whether it
// overflowed, follow its warp's schedule): F and F' are summed in 64-bit fixed point (F in units
// of 2^-40; F' in a power-of-two unit set by the ray's largest peak density), which no order of
// addition changes, and the race is an argmin.
#include "ugp_dense.cuh"
#include "ugp_gauss.cuh"
#include "ugp_philox.cuh"

namespace ugp {
namespace {

constexpr int kDWarps = 4;           // warps per block of the main pass (two rays each)
constexpr int kHalf = 16;            // lanes of the main pass that finish one ray
constexpr int kDCap = 128;           // intervals a half-warp of the main pass holds
constexpr int kDStack = 1024;        // traversal stack of a big-pass warp
constexpr int kDLevels = 8;          // bracket refinements when the intervals do not fit
constexpr int kDNewton = 64;
constexpr int kDBisectAfter = 24;    // Newton / false-position steps before plain bisection
constexpr float kNewtonStep = 1e-6f;   // relative Newton correction that ends the iteration
constexpr float kNewtonFloor = 1e-3f;  // distance scale below which the step is taken absolute
constexpr unsigned kFull = 0xffffffffu;
constexpr float kSubScale = 1099511627776.f;        // 2^40
constexpr float kSubUnit = 9.094947017729282e-13f;  // 2^-40

// Lanes that work on one ray: G = 16 (half a warp) or 32.
template <int G>
struct Grp {
  unsigned mask;  // the group's lanes in the warp
  int lane;       // lane within the group
  int base;       // warp lane of the group's lane 0
  __device__ unsigned ballot(bool p) const { return __ballot_sync(mask, p) >> base; }
  __device__ unsigned below() const { return (1u << lane) - 1u; }
  __device__ float sum(float v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_down_sync(mask, v, o, G);
    return __shfl_sync(mask, v, 0, G);  // group lane 0's sum, identical on every lane
  }
  __device__ long long sum(long long v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_down_sync(mask, v, o, G);
    return __shfl_sync(mask, v, 0, G);
  }
  __device__ float max(float v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o, G));
    return v;
  }
  template <class T>
  __device__ T shfl(T v, int src) const { return __shfl_sync(mask, v, src, G); }
  template <class T>
  __device__ T shfl_xor(T v, int o) const { return __shfl_xor_sync(mask, v, o, G); }
  __device__ void sync() const { __syncwarp(mask); }
  __device__ unsigned total(unsigned v) const { return __reduce_add_sync(mask, v); }
};

// Interval columns of one ray (cap entries each). For the interval clipped to the bracket,
// [x0, y0] = [max(a, lo), min(b, hi)]: `ex0` is erfc(|tau(x0)|) carrying the sign of tau(x0)
// (tau(x0) >= 0: positive), and `full` is 1/2 I over [x0, y0], both taken when the interval is
// collected, so that a later term over [x0, t] costs one erfc.
struct Iv {
  float *a, *b, *tn, *ts, *s, *e0, *ex0, *full;
  int* id;  // index with the end-point flags (pack_id)
  int cap;
};

template <int kCap>
struct Intervals {
  float a[kCap], b[kCap], tn[kCap], ts[kCap], s[kCap], e0[kCap], ex0[kCap], full[kCap];
  int id[kCap];
  __device__ Iv view(int off, int cap) {
    return Iv{a + off, b + off, tn + off, ts + off, s + off, e0 + off, ex0 + off, full + off, id + off, cap};
  }
};

// 1/2 I between two cut points of an interval (App. A) from erfc(|tau|) at each, signed as in
// Iv::ex0: a difference of erf values without cancellation for same-sign pairs.
__device__ __forceinline__ float cut_diff(float ep_signed, float eq, float tq) {
  const float ep = fabsf(ep_signed);
  return !signbit(ep_signed) ? ep - eq : (tq <= 0.f ? eq - ep : 2.f - ep - eq);
}
struct WarpSmem {  // main pass: the two half-warps' slices
  Intervals<2 * kDCap> iv;
};
struct WarpSmemBig {  // big pass: one ray per warp, its intervals in global memory
  static constexpr int kStack = kDStack;
  int stk[kStack];             // traversal stack
  unsigned long long bin[32];  // sub-bins, units of 2^-40
};
static_assert(kDCap >= kHalf && kBigCap >= kListCap, "capacities");

constexpr float kFScale = 1099511627776.f;  // 2^40: unit of the fixed-point F sums
constexpr float kFUnit = 9.094947017729282e-13f;

// Outcome of one ray's solve.
struct Finish {
  int prim;
  float tu, tsp;
  uint8_t st;
};

// Root of F = u on [lo, min(hi, last interval end)] over the n collected intervals, then the
// race at t_u. The sums are fixed-point integers, so the result does not depend on G or on the
// order of the intervals.
template <int G>
__device__ Finish solve(const Grp<G>& g, const Iv& iv, int n, float lo, float hi, float Flo, float u, float u2,
                        float t1, int spawn_mode) {
  const int lane = g.lane;
  Finish out{-1, t1, t1, UGP_RAY_OK};
  float bmax = lo, emax = 0.f;
  for (int e = lane; e < n; e += G) {
    bmax = fmaxf(bmax, iv.b[e]);
    emax = fmaxf(emax, iv.e0[e]);
  }
  bmax = g.max(bmax);
  emax = g.max(emax);
  const float hi_e = fminf(hi, bmax);
  // F' is a sum of n terms 1/2 G_k(t) <= emax / 2: a unit of 2^-x with 2^(62 - x) > n emax / 2
  int ex = 0;
  frexpf(fmaxf(emax, 1e-30f) * float(n > 0 ? n : 1), &ex);
  ex = max(ex, -60);  // below 2^-60 every term rounds to zero, which changes no decision
  const float dscale = ldexpf(1.f, 61 - ex), dunit = ldexpf(1.f, ex - 61);
  auto fxF = [](float v) { return __float2ll_rn(fminf(fmaxf(v, 0.f), 64.f) * kFScale); };
  // full[e] is interval e's whole term on the bracket, which is its term at t = hi_e (every
  // interval ends by bmax); later evaluations reuse it for every interval that ends before t,
  // so only the intervals containing t need an erfc, one each (its start's is in ex0).
  const float* full = iv.full;
  auto term = [&](int e, float t) {
    if (!(fmaxf(iv.a[e], lo) < t)) return 0.f;
    const float tq = tau_at(t, iv.tn[e], iv.ts[e], iv.s[e]);
    return iv.e0[e] * (0.25f * kSqrtPi) / iv.s[e] * cut_diff(iv.ex0[e], erfcf(fabsf(tq)), tq);
  };
  auto evalF = [&](float t, float& f, float& fp) {
    long long fl = 0, fpl = 0;
    for (int e = lane; e < n; e += G) {
      const float a = iv.a[e], b = iv.b[e];
      fl += fxF(b <= t ? full[e] : term(e, t));
      if (a <= t && t <= b) fpl += __float2ll_rn(0.5f * gauss_at(t, iv.tn[e], iv.ts[e], iv.s[e], iv.e0[e]) * dscale);
    }
    f = Flo - u + float(g.sum(fl)) * kFUnit;
    fp = float(g.sum(fpl)) * dunit;
  };
  float fh;
  {
    long long fl = 0;
    for (int e = lane; e < n; e += G) fl += fxF(full[e]);
    fh = Flo - u + float(g.sum(fl)) * kFUnit;
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
      // a Newton correction below 1e-6 of the distance scale ends the iteration: its own error
      // is of the order of its square (or of itself across a kink of F'), far below the 1e-5
      // accuracy asked (taken even where the shrink safeguard below would refuse the step,
      // which near the root only reflects the rounding noise of f)
      if (fp > 0.f && fabsf(f) <= kNewtonStep * fmaxf(fabsf(t), kNewtonFloor) * fp) {
        const float tn = t - f / fp;
        if (tn > a0 && tn < b0) t = tn;
        conv = true;
        break;
      }
      const float tn = fp > 0.f ? t - f / fp : a0;
      float tnew;
      // past kDBisectAfter steps only bisection: the bracket then collapses to adjacent floats
      // within the iteration bound, whatever F looks like
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
    if (!conv) out.st = UGP_RAY_SOLVE_LIMIT;
  }
  // race: smallest E_k / G_k(x_t) among the intervals containing t (ties: smaller index)
  float best = INFINITY;
  int best_id = INT32_MAX, best_e = -1;
  for (int e = lane; e < n; e += G) {
    if (!(iv.a[e] <= t && t <= iv.b[e])) continue;
    const int idv = unpack_id(iv.id[e]);
    const float key = race_exponential(u2, idv) / gauss_at(t, iv.tn[e], iv.ts[e], iv.s[e], iv.e0[e]);
    if (best_e < 0 || key < best || (key == best && idv < best_id)) {
      best = key;
      best_id = idv;
      best_e = e;
    }
  }
  for (int o = G / 2; o > 0; o >>= 1) {
    const float ok = g.shfl_xor(best, o);
    const int oi = g.shfl_xor(best_id, o);
    const int oe = g.shfl_xor(best_e, o);
    if (oe >= 0 && (best_e < 0 || ok < best || (ok == best && oi < best_id))) {
      best = ok;
      best_id = oi;
      best_e = oe;
    }
  }
  if (best_e >= 0) {
    out.prim = best_id;
    out.tu = t;
    out.tsp = spawn_mode == 1 ? t : 0.5f * (iv.a[best_e] + iv.b[best_e]);
  }
  return out;
}

// Tests candidate `slot` (< 0: none) on every lane of the group and appends the hits meeting
// [lo, hi] to iv (at most iv.cap are stored); n counts all of them.
template <int G>
__device__ __forceinline__ void collect_one(const Grp<G>& g, const Iv& iv, const TraceScene& sc, const Ray& ray,
                                            float lo, float hi, float t0, float t1, int excl, int slot, int& n,
                                            unsigned& np) {
  PrimHit hh;
  bool ok = false;
  if (slot >= 0) {
    ++np;
    ok = prim_test(sc.prims, sc.wlo, slot, ray, t0, t1, sc.k2, excl, hh) && fmaxf(hh.a, lo) < fminf(hh.b, hi);
  }
  const unsigned m = g.ballot(ok);
  if (ok) {
    const int i = n + __popc(m & g.below());
    if (i < iv.cap) {
      const float x0 = fmaxf(hh.a, lo), y0 = fminf(hh.b, hi);
      const float tp = (hh.a_end && x0 == hh.a) ? -hh.th : tau_at(x0, hh.tn, hh.ts, hh.s);
      const float tq = (hh.b_end && y0 == hh.b) ? hh.th : tau_at(y0, hh.tn, hh.ts, hh.s);
      const float ep = erfcf(fabsf(tp));
      const float ex0 = tp >= 0.f ? ep : -ep;
      iv.a[i] = hh.a; iv.b[i] = hh.b; iv.tn[i] = hh.tn; iv.ts[i] = hh.ts;
      iv.s[i] = hh.s; iv.e0[i] = hh.e0; iv.ex0[i] = ex0; iv.id[i] = pack_id(hh);
      iv.full[i] = hh.e0 * (0.25f * kSqrtPi) / hh.s * cut_diff(ex0, erfcf(fabsf(tq)), tq);
    }
  }
  n += __popc(m);
}

// Warp-parallel traversal of the leaves whose boxes meet [lo, hi]; `leaf(slot)` is called by all
// lanes together (slot < 0 for lanes without a leaf), twice per step.
template <int kStack, class LeafFn>
__device__ void warp_traverse(int* stk, const TraceScene& sc, const Ray& ray, float lo, float hi, int lane,
                              uint8_t& st, unsigned& nn, LeafFn&& leaf) {
  int size = 1;
  if (lane == 0) stk[0] = 0;
  __syncwarp();
  while (size > 0) {
    const int m = min(size, 32);
    const int node = lane < m ? stk[size - 1 - lane] : -1;
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
        if (off < kStack) stk[off] = ch[c];
      }
      size += __popc(mask);
    }
    if (size > kStack) {
      st = UGP_RAY_STACK_OVERFLOW;
      return;
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 2; ++c) leaf((h[c] && ch[c] < 0) ? ~ch[c] : -1);
    __syncwarp();
  }
}

// Per-ray inputs from slot j of the table.
struct RayIn {
  TraceScene sc;
  int idx, excl, nlist;
  float lo, hi, Flo, u, u2, t0, t1;
  const int* list;  // complete slot list, or NULL
  Ray ray;
};
__device__ __forceinline__ RayIn ray_in(const TraceScene& sc0, const DenseQueue& q, int j) {
  RayIn R;
  R.sc = q.scenes ? q.scenes[q.scene[j]] : sc0;
  R.idx = q.idx[j];
  R.lo = q.lo[j];
  R.hi = q.hi[j];
  R.Flo = q.Flo[j];
  R.u = q.u[j];
  R.u2 = q.u2[j];
  R.t0 = q.t0[j];
  R.t1 = q.t1[j];
  R.excl = q.excl[j];
  R.nlist = q.nlist[j];
  R.list = (q.list && R.nlist <= kListCap) ? q.list + size_t(R.idx) * kListCap : nullptr;
  R.ray = make_ray(make_float3(q.ox[j], q.oy[j], q.oz[j]), make_float3(q.dx[j], q.dy[j], q.dz[j]));
  return R;
}

struct Outputs {
  int* prim;
  float *tu, *tsp;
  uint8_t* st;
  int spawn_mode;
  unsigned long long *stats, *rays_err;
};

// Written by one lane.
__device__ __forceinline__ void write_out(const Outputs& O, int idx, const Finish& f, unsigned nn, unsigned np) {
  O.prim[idx] = f.prim;
  O.tsp[idx] = f.tsp;
  if (O.tu) O.tu[idx] = f.tu;
  if (O.st) O.st[idx] = f.st;
  if (f.st != UGP_RAY_OK && O.rays_err) atomicAdd(O.rays_err, 1ull);
  if (O.stats) {
    atomicAdd(O.stats + 0, (unsigned long long)nn);
    atomicAdd(O.stats + 1, (unsigned long long)np);
  }
}

// Appends slot j of the table to the list of a bigger pass (counter `count`, array `list`).
__device__ __forceinline__ void hand_on(int* count, int* list, int j) { list[atomicAdd(count, 1)] = j; }

__global__ void __launch_bounds__(32 * kDWarps) k_dense(TraceScene sc0, DenseQueue q, int64_t n_host,
                                                        const int* n_dev, Outputs O) {
  extern __shared__ __align__(16) unsigned char dsm[];
  WarpSmem& W = reinterpret_cast<WarpSmem*>(dsm)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31, half = lane >> 4;
  const Grp<kHalf> g{0xffffu << (16 * half), lane & 15, 16 * half};
  const Iv iv = W.iv.view(half * kDCap, kDCap);
  const int count = n_dev ? *reinterpret_cast<const volatile int*>(n_dev) : int(n_host);
  const int nwarps = gridDim.x * kDWarps;
  // slots 2p and 2p + 1 to warp p mod (warps), one per half-warp; neighbouring rays in the
  // table are in flight together
  for (int p = blockIdx.x * kDWarps + (threadIdx.x >> 5); 2 * p < count; p += nwarps) {
    const int j = 2 * p + half;
    if (j >= count || __ldg(q.idx + j) < 0) continue;
    const RayIn R = ray_in(sc0, q, j);
    bool big = R.list == nullptr;
    int n = 0;
    unsigned np = 0;
    if (!big) {
      for (int base = 0; base < R.nlist; base += kHalf) {
        const int e = base + g.lane;
        collect_one(g, iv, R.sc, R.ray, R.lo, R.hi, R.t0, R.t1, R.excl, e < R.nlist ? __ldg(R.list + e) : -1, n, np);
      }
      g.sync();
      big = n > kDCap;
    }
    const unsigned tp = g.total(np);
    if (big) {  // k_dense_big rebuilds and finishes the ray
      if (g.lane == 0) {
        hand_on(q.count + 2, q.wide, j);
        if (O.stats) {
          atomicAdd(O.stats + 1, (unsigned long long)tp);
          atomicAdd(O.stats + 5, 1ull);
        }
      }
      g.sync();
      continue;
    }
    const Finish f = solve(g, iv, n, R.lo, R.hi, R.Flo, R.u, R.u2, R.t1, O.spawn_mode);
    if (g.lane == 0) write_out(O, R.idx, f, 0u, tp);
    g.sync();
  }
}

// The rays the first pass handed on (count of them in `list`), one warp each, kWarps warps per
// block, up to kCap intervals per ray in the warp's slot of q.big_iv; a ray with more has its
// bracket narrowed by sub-bins (or is handed on to a next pass when `next_count` is given).
template <int kCap, int kWarps>
__global__ void __launch_bounds__(32 * kWarps) k_dense_big(TraceScene sc0, DenseQueue q, const int* count_p,
                                                           const int* __restrict__ list, int* next_count,
                                                           int* __restrict__ next_list, Outputs O) {
  extern __shared__ __align__(16) unsigned char dsm[];
  WarpSmemBig& W = reinterpret_cast<WarpSmemBig*>(dsm)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const Grp<32> gw{kFull, lane, 0};
  // this warp's interval slot (the grid has at most q.big_slots warps)
  float* slot = q.big_iv + size_t(blockIdx.x * kWarps + (threadIdx.x >> 5)) * (size_t(kCap) * 9);
  const Iv iv{slot, slot + kCap, slot + 2 * kCap, slot + 3 * kCap, slot + 4 * kCap, slot + 5 * kCap,
              slot + 6 * kCap, slot + 7 * kCap, reinterpret_cast<int*>(slot + 8 * kCap), kCap};
  const int count = *reinterpret_cast<const volatile int*>(count_p);
  for (int h = blockIdx.x * kWarps + (threadIdx.x >> 5); h < count; h += gridDim.x * kWarps) {
    const int j = list[h];
    const RayIn R = ray_in(sc0, q, j);
    float lo = R.lo, hi = R.hi, Flo = R.Flo;
    uint8_t st = UGP_RAY_OK;
    unsigned nn = 0, np = 0;
    Finish f{-1, R.t1, R.t1, UGP_RAY_OK};
    bool done = false, handed = false;
    for (int level = 0; level < kDLevels && !done && st == UGP_RAY_OK; ++level) {
      // ---- 1. collect the intervals meeting [lo, hi]
      int n = 0;
      if (R.list) {
        for (int base = 0; base < R.nlist; base += 32) {
          const int e = base + lane;
          collect_one(gw, iv, R.sc, R.ray, lo, hi, R.t0, R.t1, R.excl, e < R.nlist ? __ldg(R.list + e) : -1, n, np);
        }
      } else {
        warp_traverse<WarpSmemBig::kStack>(W.stk, R.sc, R.ray, lo, hi, lane, st, nn, [&](int s) {
          collect_one(gw, iv, R.sc, R.ray, lo, hi, R.t0, R.t1, R.excl, s, n, np);
        });
      }
      __syncwarp();
      if (st != UGP_RAY_OK) break;
      if (n <= kCap) {
        // ---- 2. the solve
        f = solve(gw, iv, n, lo, hi, Flo, R.u, R.u2, R.t1, O.spawn_mode);
        done = true;
      } else if (next_count && level == 0) {
        handed = true;  // the next pass holds more intervals
        break;
      } else {
        // ---- 3. too many intervals: shrink the bracket to the crossing sub-bin
        W.bin[lane] = 0ull;
        __syncwarp();
        const float w = (hi - lo) / 32.f;
        auto edge = [&](int k) { return k >= 32 ? hi : lo + w * float(k); };
        auto bin_one = [&](int slot) {
          if (slot < 0) return;
          ++np;
          PrimHit hh;
          if (!prim_test(R.sc.prims, R.sc.wlo, slot, R.ray, R.t0, R.t1, R.sc.k2, R.excl, hh)) return;
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
        };
        if (R.list) {
          for (int base = 0; base < R.nlist; base += 32) {
            const int e = base + lane;
            bin_one(e < R.nlist ? __ldg(R.list + e) : -1);
          }
        } else {
          warp_traverse<WarpSmemBig::kStack>(W.stk, R.sc, R.ray, lo, hi, lane, st, nn, bin_one);
        }
        __syncwarp();
        if (st != UGP_RAY_OK) break;
        unsigned long long acc = 0ull;
        int jx = 31;
        for (int k = 0; k < 32; ++k) {
          const unsigned long long nxt = acc + W.bin[k];
          if (float(nxt) * kSubUnit > R.u - Flo) {
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
    const unsigned tn = gw.total(nn), tp = gw.total(np);
    if (handed) {
      if (lane == 0) {
        hand_on(next_count, next_list, j);
        if (O.stats) {
          atomicAdd(O.stats + 0, (unsigned long long)tn);
          atomicAdd(O.stats + 1, (unsigned long long)tp);
        }
      }
      __syncwarp();
      continue;
    }
    if (st != UGP_RAY_OK) f.st = st;
    else if (!done) f.st = UGP_RAY_ITER_LIMIT;
    if (lane == 0) {
      if (f.st != UGP_RAY_OK && f.st != UGP_RAY_SOLVE_LIMIT) f = Finish{-1, R.t1, R.t1, f.st};
      write_out(O, R.idx, f, tn, tp);
    }
    __syncwarp();
  }
}

}  // namespace

// Resident-block grid of each pass (set once, before any capture).
static int g_dense_grid = 0, g_wide_grid = 0;
constexpr int kWideWarps = 4;

template <class K>
static ugp_status big_grid(K kern, int block, size_t smem, int sms, int* grid) {
  int per_sm = 0;
  UGP_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  UGP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem));
  *grid = sms * (per_sm > 0 ? per_sm : 1);
  return UGP_OK;
}

ugp_status dense_prepare() {
  if (g_dense_grid != 0) return UGP_OK;
  int dev = 0, sms = 0;
  UGP_CUDA_CHECK(cudaGetDevice(&dev));
  UGP_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (sms <= 0) sms = 1;
  ugp_status s = big_grid(k_dense_big<kBigCap, kWideWarps>, 32 * kWideWarps, sizeof(WarpSmemBig) * kWideWarps, sms,
                          &g_wide_grid);
  if (s != UGP_OK) return s;
  int grid = 0;
  if ((s = big_grid(k_dense, 32 * kDWarps, sizeof(WarpSmem) * kDWarps, sms, &grid)) != UGP_OK) return s;
  g_dense_grid = grid;
  return UGP_OK;
}

ugp_status launch_dense(const TraceScene& sc, const DenseQueue& q, int64_t n_host, const int* n_dev,
                        int64_t max_slots, int* prim_out, float* t_u_out, float* t_spawn_out, uint8_t* status_out,
                        int spawn_mode, unsigned long long* stats, unsigned long long* rays_err, cudaStream_t stream) {
  const ugp_status ps = dense_prepare();
  if (ps != UGP_OK) return ps;
  auto cap_grid = [](int64_t need, int cap) { return unsigned(need < cap ? (need > 0 ? need : 1) : cap); };
  const Outputs O{prim_out, t_u_out, t_spawn_out, status_out, spawn_mode, stats, rays_err};
  UGP_CUDA_CHECK(cudaMemsetAsync(q.count + 2, 0, 2 * sizeof(int), stream));
  prof_begin(kStDense, stream);
  k_dense<<<cap_grid((max_slots + 64 * kDWarps - 1) / (64 * kDWarps), g_dense_grid), 32 * kDWarps,
            sizeof(WarpSmem) * kDWarps, stream>>>(sc, q, n_host, n_dev, O);
  // at most one warp per interval slot
  const int slot_blocks = q.big_slots / kWideWarps;
  k_dense_big<kBigCap, kWideWarps><<<cap_grid((max_slots + kWideWarps - 1) / kWideWarps,
                                              g_wide_grid < slot_blocks ? g_wide_grid : slot_blocks),
                                     32 * kWideWarps, sizeof(WarpSmemBig) * kWideWarps, stream>>>(
      sc, q, q.count + 2, q.wide, nullptr, nullptr, O);
  prof_end(kStDense, stream, 2);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

}  // namespace ugp
