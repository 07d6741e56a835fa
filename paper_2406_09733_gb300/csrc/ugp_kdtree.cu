// The paper's own free-flight sampler (Sec. 5.1-5.2) on the GPU: an SAH kd-tree over the
// primitives' k-ellipsoid boxes, front-to-back traversal, per-leaf accumulation of the CDF in the
// leaf's order, and in a leaf where the CDF reaches 1 the paper's GPU partition of the ray-node
// interval into a fixed number of bins, each bin classified again, and the disambiguation of
// Eq. 10 in the bin where it reaches 1 (t_u solved there, the primitive drawn proportionally to
// I_k(bin start, t_u) among the primitives overlapping the bin).
//
// The kd-tree is a comparison variant: its sampled primitive follows the paper's rule, which
// depends on the tree and is biased where the rule's assumption fails (the library's own
// free-flight sampler is exact and order-free). It reuses the BVH's primitive records.
//
// Build (on the device, one level of nodes per round, the host reading two counts per level):
//   1. every reference (node, primitive) bins its box, clipped to the node, into kKdBins bins per
//      axis (starts and ends);
//   2. every node takes the cheapest bin plane by the surface-area heuristic (traversal 1,
//      intersection 1.5), or becomes a leaf when no plane beats the leaf;
//   3. references go left if their box starts before the plane and right if it ends after it
//      (both when it straddles); the children's reference lists follow in a new level.
// Leaves keep their references in ascending slot order (the leaf's order of the rule).
#include <math.h>
#include <string.h>

#include <vector>

#include "ugp_gauss.cuh"
#include "ugp_trace.cuh"

struct ugp_kdtree {
  uint32_t magic;
  const ugp_bvh* bvh;
  const int4* nodes;   // interior (axis, pos bits, left, right); leaf (3, count, first, 0)
  const int* refs;     // leaf references (BVH slots)
  int64_t n_nodes, n_refs;
  int depth;
  float box[6];        // root box
};

namespace ugp {
namespace {

constexpr uint32_t kKdMagic = 0x5547504Bu;  // "UGPK"
constexpr int kKdBins = 8;
constexpr int kKdMaxDepth = 28;
constexpr int kKdSegBins = 8;    // bins of an ambiguous leaf's ray interval (the paper's GPU partition)
constexpr int kKdStack = 48;
constexpr float kKdTrav = 1.f, kKdIsect = 1.5f;
constexpr int kKdLeafType = 3;

struct KdLayout {
  size_t nodes, refs, persistent;
  size_t aabb, refA, refB, nodeA, nodeB, lvA, lvB, bins, cnt, cur, ctl, total;
  int64_t cap_refs, cap_nodes;
};

// Per level node: box, its reference range, final node id, depth.
struct LvNode {
  float lo[3], hi[3];
  int first, count, gid, depth;
};

// Control words written by the scan of a level.
struct KdCtl {
  int next_m, next_r, leaf_refs, splits, leaves_total, refs_total;
};

KdLayout kd_layout(int64_t n) {
  KdLayout L;
  L.cap_refs = 4 * n + 1024;
  L.cap_nodes = 2 * L.cap_refs;
  size_t off = 0;
  L.nodes = off;  off = align256(off + size_t(L.cap_nodes) * 16);
  L.refs = off;   off = align256(off + size_t(L.cap_refs) * 4);
  L.persistent = off;
  L.aabb = off;   off = align256(off + size_t(n) * 24);
  L.refA = off;   off = align256(off + size_t(L.cap_refs) * 4);
  L.refB = off;   off = align256(off + size_t(L.cap_refs) * 4);
  L.nodeA = off;  off = align256(off + size_t(L.cap_refs) * 4);
  L.nodeB = off;  off = align256(off + size_t(L.cap_refs) * 4);
  L.lvA = off;    off = align256(off + size_t(L.cap_refs) * sizeof(LvNode));
  L.lvB = off;    off = align256(off + size_t(L.cap_refs) * sizeof(LvNode));
  L.bins = off;   off = align256(off + size_t(L.cap_refs) * 6 * kKdBins * 4);
  L.cnt = off;    off = align256(off + size_t(L.cap_refs) * 8 * 4);
  L.cur = off;    off = align256(off + size_t(L.cap_refs) * 4 * 4);
  L.ctl = off;    off = align256(off + 256);
  L.total = off;
  return L;
}

static float o2f_host(int i) {
  const int j = i >= 0 ? i : i ^ 0x7fffffff;
  float f;
  memcpy(&f, &j, 4);
  return f;
}

__device__ __forceinline__ int f2o(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// Box of the k-ellipsoid of the primitive in slot s from its record: W^-1 = R S, so the half
// extent along axis i is k |row i of W^-1|; widened by a few ulps like the BVH's boxes. Invalid
// records get an empty box that no ray meets.
__global__ void k_kd_boxes(int64_t n, const float4* __restrict__ recs, float k, float* __restrict__ aabb,
                           int* __restrict__ root) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float4 r0 = recs[4 * s], r1 = recs[4 * s + 1], r2 = recs[4 * s + 2], r3 = recs[4 * s + 3];
  float* b = aabb + 6 * s;
  if (r3.z == 0.f) {
    for (int a = 0; a < 3; ++a) { b[a] = 1.f; b[3 + a] = 0.f; }
    return;
  }
  const double W[9] = {r0.x, r0.y, r0.z, r1.x, r1.y, r1.z, r2.x, r2.y, r2.z};
  const double c00 = W[4] * W[8] - W[5] * W[7], c01 = W[5] * W[6] - W[3] * W[8], c02 = W[3] * W[7] - W[4] * W[6];
  const double det = W[0] * c00 + W[1] * c01 + W[2] * c02;
  const double inv[9] = {c00 / det, (W[2] * W[7] - W[1] * W[8]) / det, (W[1] * W[5] - W[2] * W[4]) / det,
                         c01 / det, (W[0] * W[8] - W[2] * W[6]) / det, (W[2] * W[3] - W[0] * W[5]) / det,
                         c02 / det, (W[1] * W[6] - W[0] * W[7]) / det, (W[0] * W[4] - W[1] * W[3]) / det};
  const float m[3] = {r0.w, r1.w, r2.w};
  for (int a = 0; a < 3; ++a) {
    const double e2 = inv[3 * a] * inv[3 * a] + inv[3 * a + 1] * inv[3 * a + 1] + inv[3 * a + 2] * inv[3 * a + 2];
    const float e = float(double(k) * sqrt(e2)) * (1.f + 4e-6f) + 2e-7f * fabsf(m[a]);
    b[a] = m[a] - e;
    b[3 + a] = m[a] + e;
    atomicMin(root + a, f2o(b[a]));
    atomicMin(root + 3 + a, f2o(-b[3 + a]));
  }
}

__global__ void k_kd_root(int64_t n, const int* __restrict__ root, LvNode* __restrict__ lv, int* __restrict__ refs,
                          int* __restrict__ rnode) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s == 0) {
    LvNode r;
    for (int a = 0; a < 3; ++a) {
      r.lo[a] = o2f(root[a]);
      r.hi[a] = -o2f(root[3 + a]);
    }
    r.first = 0;
    r.count = int(n);
    r.gid = 0;
    r.depth = 0;
    lv[0] = r;
  }
  if (s < n) {
    refs[s] = int(s);
    rnode[s] = 0;
  }
}

__device__ __forceinline__ int bin_of(float x, float lo, float hi) {
  const float w = hi - lo;
  if (!(w > 0.f)) return 0;
  return min(kKdBins - 1, max(0, int((x - lo) / w * float(kKdBins))));
}

// 1. start and end bins of every reference's box, clipped to its node
__global__ void k_kd_bin(int r_count, const int* __restrict__ refs, const int* __restrict__ rnode,
                         const LvNode* __restrict__ lv, const float* __restrict__ aabb, int* __restrict__ bins) {
  const int r = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= r_count) return;
  const int m = rnode[r];
  const LvNode& nd = lv[m];
  const float* b = aabb + 6 * size_t(refs[r]);
  int* bm = bins + size_t(m) * 6 * kKdBins;
  for (int a = 0; a < 3; ++a) {
    const float lo = fmaxf(b[a], nd.lo[a]), hi = fminf(b[3 + a], nd.hi[a]);
    atomicAdd(bm + (2 * a) * kKdBins + bin_of(lo, nd.lo[a], nd.hi[a]), 1);
    atomicAdd(bm + (2 * a + 1) * kKdBins + bin_of(hi, nd.lo[a], nd.hi[a]), 1);
  }
}

__device__ __forceinline__ float half_area(const float lo[3], const float hi[3]) {
  const float x = hi[0] - lo[0], y = hi[1] - lo[1], z = hi[2] - lo[2];
  return x * y + y * z + z * x;
}

// 2. plane of every node by the surface-area heuristic over the bin planes (or a leaf);
//    cnt[8 m + 0] = axis (-1: leaf), cnt[8 m + 1] = float bits of the plane.
__global__ void k_kd_choose(int m_count, const LvNode* __restrict__ lv, const int* __restrict__ bins,
                            int* __restrict__ cnt, int force_leaf) {
  const int m = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= m_count) return;
  const LvNode nd = lv[m];
  int best_axis = -1;
  float best_pos = 0.f;
  if (!force_leaf && nd.count > 1 && nd.depth < kKdMaxDepth) {
    float best = kKdIsect * float(nd.count);
    const float A = half_area(nd.lo, nd.hi);
    const int* bm = bins + size_t(m) * 6 * kKdBins;
    for (int a = 0; a < 3; ++a) {
      const float w = nd.hi[a] - nd.lo[a];
      if (!(w > 0.f) || !(A > 0.f)) continue;
      int nl = 0, ends_before = 0;
      for (int p = 1; p < kKdBins; ++p) {
        nl += bm[(2 * a) * kKdBins + p - 1];
        ends_before += bm[(2 * a + 1) * kKdBins + p - 1];
        const int nr = nd.count - ends_before;
        const float pos = nd.lo[a] + w * (float(p) / float(kKdBins));
        float Llo[3], Lhi[3], Rlo[3], Rhi[3];
        for (int c = 0; c < 3; ++c) { Llo[c] = Rlo[c] = nd.lo[c]; Lhi[c] = Rhi[c] = nd.hi[c]; }
        Lhi[a] = pos;
        Rlo[a] = pos;
        const float cost = kKdTrav + kKdIsect * (half_area(Llo, Lhi) * float(nl) + half_area(Rlo, Rhi) * float(nr)) / A;
        if (cost < best) {
          best = cost;
          best_axis = a;
          best_pos = pos;
        }
      }
    }
  }
  cnt[8 * m + 0] = best_axis;
  cnt[8 * m + 1] = __float_as_int(best_pos);
  cnt[8 * m + 2] = 0;  // left count
  cnt[8 * m + 3] = 0;  // right count
}

__device__ __forceinline__ void sides(const float* b, const LvNode& nd, int axis, float pos, bool& l, bool& r) {
  const float lo = fmaxf(b[axis], nd.lo[axis]), hi = fminf(b[3 + axis], nd.hi[axis]);
  l = lo < pos;
  r = hi > pos;
  if (!l && !r) l = true;  // a flat box on the plane
}

// 3a. exact child counts
__global__ void k_kd_count(int r_count, const int* __restrict__ refs, const int* __restrict__ rnode,
                           const LvNode* __restrict__ lv, const float* __restrict__ aabb, int* __restrict__ cnt) {
  const int r = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= r_count) return;
  const int m = rnode[r];
  const int axis = cnt[8 * m];
  if (axis < 0) return;
  bool l, rr;
  sides(aabb + 6 * size_t(refs[r]), lv[m], axis, __int_as_float(cnt[8 * m + 1]), l, rr);
  if (l) atomicAdd(cnt + 8 * m + 2, 1);
  if (rr) atomicAdd(cnt + 8 * m + 3, 1);
}

// 3b. one block: offsets of the children's reference lists and node slots, and of the leaves'
//     references in the final array (exclusive scans in node order).
__global__ void __launch_bounds__(1024) k_kd_scan(int m_count, const LvNode* __restrict__ lv, int* __restrict__ cnt,
                                                  KdCtl* __restrict__ ctl) {
  __shared__ int s_split[1024], s_refs[1024], s_leaf[1024];
  __shared__ int base_split, base_refs, base_leaf;
  if (threadIdx.x == 0) {
    base_split = 0;
    base_refs = 0;
    base_leaf = ctl->refs_total;
  }
  __syncthreads();
  for (int c0 = 0; c0 < m_count; c0 += 1024) {
    const int m = c0 + int(threadIdx.x);
    int sp = 0, rf = 0, lf = 0;
    if (m < m_count) {
      if (cnt[8 * m] >= 0) {
        sp = 1;
        rf = cnt[8 * m + 2] + cnt[8 * m + 3];
      } else {
        lf = lv[m].count;
      }
    }
    s_split[threadIdx.x] = sp;
    s_refs[threadIdx.x] = rf;
    s_leaf[threadIdx.x] = lf;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scans
      int a = 0, b = 0, c = 0;
      if (int(threadIdx.x) >= o) {
        a = s_split[threadIdx.x - o];
        b = s_refs[threadIdx.x - o];
        c = s_leaf[threadIdx.x - o];
      }
      __syncthreads();
      s_split[threadIdx.x] += a;
      s_refs[threadIdx.x] += b;
      s_leaf[threadIdx.x] += c;
      __syncthreads();
    }
    if (m < m_count) {
      cnt[8 * m + 4] = base_split + s_split[threadIdx.x] - sp;  // rank among splitting nodes
      cnt[8 * m + 5] = base_refs + s_refs[threadIdx.x] - rf;    // first reference of the left child
      cnt[8 * m + 6] = base_leaf + s_leaf[threadIdx.x] - lf;    // first final reference of a leaf
    }
    __syncthreads();
    if (threadIdx.x == 1023) {
      base_split += s_split[1023];
      base_refs += s_refs[1023];
      base_leaf += s_leaf[1023];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ctl->splits = base_split;
    ctl->next_m = 2 * base_split;
    ctl->next_r = base_refs;
    ctl->leaf_refs = base_leaf - ctl->refs_total;
  }
}

// 3c. final node records, and the children's level entries
__global__ void k_kd_emit(int m_count, const LvNode* __restrict__ lv, const int* __restrict__ cnt, int gid_base,
                          int4* __restrict__ nodes, LvNode* __restrict__ next, int* __restrict__ cursor) {
  const int m = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= m_count) return;
  const LvNode nd = lv[m];
  const int axis = cnt[8 * m];
  cursor[4 * m + 0] = 0;
  cursor[4 * m + 1] = 0;
  if (axis < 0) {
    nodes[nd.gid] = make_int4(kKdLeafType, nd.count, cnt[8 * m + 6], 0);
    return;
  }
  const float pos = __int_as_float(cnt[8 * m + 1]);
  const int rank = cnt[8 * m + 4];
  const int gl = gid_base + 2 * rank, gr = gl + 1;
  nodes[nd.gid] = make_int4(axis, __float_as_int(pos), gl, gr);
  LvNode L = nd, R = nd;
  L.hi[axis] = pos;
  R.lo[axis] = pos;
  L.first = cnt[8 * m + 5];
  L.count = cnt[8 * m + 2];
  R.first = L.first + L.count;
  R.count = cnt[8 * m + 3];
  L.gid = gl;
  R.gid = gr;
  L.depth = R.depth = nd.depth + 1;
  next[2 * rank] = L;
  next[2 * rank + 1] = R;
}

// 3d. references into the children's lists or the leaves' final lists
__global__ void k_kd_write(int r_count, const int* __restrict__ refs, const int* __restrict__ rnode,
                           const LvNode* __restrict__ lv, const float* __restrict__ aabb, const int* __restrict__ cnt,
                           int* __restrict__ cursor, int* __restrict__ out_refs, int* __restrict__ out_node,
                           int* __restrict__ final_refs) {
  const int r = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= r_count) return;
  const int m = rnode[r];
  const int slot = refs[r];
  const int axis = cnt[8 * m];
  if (axis < 0) {
    final_refs[cnt[8 * m + 6] + atomicAdd(cursor + 4 * m, 1)] = slot;
    return;
  }
  bool l, rr;
  sides(aabb + 6 * size_t(slot), lv[m], axis, __int_as_float(cnt[8 * m + 1]), l, rr);
  const int rank = cnt[8 * m + 4];
  const int first = cnt[8 * m + 5];
  if (l) {
    const int p = first + atomicAdd(cursor + 4 * m, 1);
    out_refs[p] = slot;
    out_node[p] = 2 * rank;
  }
  if (rr) {
    const int p = first + cnt[8 * m + 2] + atomicAdd(cursor + 4 * m + 1, 1);
    out_refs[p] = slot;
    out_node[p] = 2 * rank + 1;
  }
}

// Leaf references in ascending slot order (the leaf's order of the sampling rule).
__global__ void k_kd_sort_leaves(int n_nodes, const int4* __restrict__ nodes, int* __restrict__ refs) {
  const int i = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const int4 nd = nodes[i];
  if (nd.x != kKdLeafType) return;
  int* p = refs + nd.z;
  for (int a = 1; a < nd.y; ++a) {
    const int v = p[a];
    int b = a - 1;
    while (b >= 0 && p[b] > v) {
      p[b + 1] = p[b];
      --b;
    }
    p[b + 1] = v;
  }
}

// ------------------------------------------------------------------------------------ sampling
struct KdRay {
  TraceScene sc;
  Ray ray;
  float t0, t1, u, u2;
  int ex;
  float cdf;
  int prim;
  float ta_hit, tb_hit;  // the chosen primitive's clipped interval
  bool done;
  uint8_t st;
};

// The part of reference slot's clipped interval inside [lo, hi] (and its hit record).
__device__ __forceinline__ bool kd_part(const KdRay& R, int slot, float lo, float hi, PrimHit& h, float& x, float& y) {
  if (!prim_test(R.sc.prims, R.sc.wlo, slot, R.ray, R.t0, R.t1, R.sc.k2, R.ex, h)) return false;
  x = fmaxf(h.a, lo);
  y = fminf(h.b, hi);
  return x < y;
}

__device__ __forceinline__ float kd_mass(const PrimHit& h, float x, float y) {
  return seg_half_integral(x, y, h.a, h.b, h.a_end, h.b_end, h.tn, h.ts, h.s, h.e0, h.th);
}

// Masses over [lo, hi] in the leaf's order: the sample is the primitive whose mass u falls in.
__device__ bool kd_take_in_order(KdRay& R, const int* refs, int count, float lo, float hi) {
  for (int j = 0; j < count; ++j) {
    PrimHit h;
    float x, y;
    if (!kd_part(R, __ldg(refs + j), lo, hi, h, x, y)) continue;
    const float m = kd_mass(h, x, y);
    if (R.u < R.cdf + m) {
      R.prim = h.id;
      R.ta_hit = h.a;
      R.tb_hit = h.b;
      R.done = true;
      return true;
    }
    R.cdf += m;
  }
  return false;
}

// The bin [s0, s1] where the CDF reaches 1: t_u by Newton's method kept in a bracket (bisection
// where a step leaves it), then the primitive drawn proportionally to I_k(s0, t_u) among those
// overlapping the bin (Eq. 10).
__device__ void kd_disambiguate(KdRay& R, const int* refs, int count, float s0, float s1) {
  float lo = s0, hi = s1, t = 0.5f * (s0 + s1);
  bool conv = false;
  for (int it = 0; it < 64; ++it) {
    float f = R.cdf - R.u, fp = 0.f;
    for (int j = 0; j < count; ++j) {
      PrimHit h;
      float x, y;
      if (!kd_part(R, __ldg(refs + j), s0, s1, h, x, y)) continue;
      if (x < t) f += kd_mass(h, x, fminf(y, t));
      if (x <= t && t <= y) fp += 0.5f * gauss_at(t, h.tn, h.ts, h.s, h.e0);
    }
    if (f == 0.f) { conv = true; break; }
    if (f < 0.f) lo = t; else hi = t;
    float tn = fp > 0.f ? t - f / fp : 0.5f * (lo + hi);
    if (!(tn > lo && tn < hi)) tn = 0.5f * (lo + hi);
    if (fabsf(tn - t) <= 1e-7f * fmaxf(fabsf(t), 1e-3f) || !(nextafterf(lo, INFINITY) < hi)) {
      t = tn;
      conv = true;
      break;
    }
    t = tn;
  }
  if (!conv) R.st = UGP_RAY_SOLVE_LIMIT;
  float wsum = 0.f;
  for (int j = 0; j < count; ++j) {
    PrimHit h;
    float x, y;
    if (!kd_part(R, __ldg(refs + j), s0, s1, h, x, y)) continue;
    if (x < t) wsum += kd_mass(h, x, fminf(y, t));
  }
  const float target = R.u2 * wsum;
  float c = 0.f;
  int last = -1;
  float la = 0.f, lb = 0.f;
  for (int j = 0; j < count; ++j) {
    PrimHit h;
    float x, y;
    if (!kd_part(R, __ldg(refs + j), s0, s1, h, x, y)) continue;
    last = h.id;
    la = h.a;
    lb = h.b;
    const float w = x < t ? kd_mass(h, x, fminf(y, t)) : 0.f;
    if (w > 0.f && target < c + w) break;
    c += w;
  }
  // the last overlapping primitive when rounding leaves the running sum a hair below the target
  R.prim = last;
  R.ta_hit = la;
  R.tb_hit = lb;
  R.done = true;
}

// One leaf of the front-to-back walk over the ray-node interval [ta, tb].
__device__ void kd_leaf(KdRay& R, const int* refs, int count, float ta, float tb) {
  float total = 0.f;
  int nh = 0;
  for (int j = 0; j < count; ++j) {
    PrimHit h;
    float x, y;
    if (!kd_part(R, __ldg(refs + j), ta, tb, h, x, y)) continue;
    total += kd_mass(h, x, y);
    ++nh;
  }
  if (nh == 0) return;
  if (nh == 1 || R.cdf + total < 1.f) {
    kd_take_in_order(R, refs, count, ta, tb);
    return;
  }
  // the paper's GPU partition: kKdSegBins equal bins of the ray-node interval, each classified
  const float w = (tb - ta) / float(kKdSegBins);
  for (int b = 0; b < kKdSegBins && !R.done; ++b) {
    const float s0 = ta + w * float(b), s1 = b + 1 == kKdSegBins ? tb : ta + w * float(b + 1);
    float sum = 0.f;
    int na = 0;
    for (int j = 0; j < count; ++j) {
      PrimHit h;
      float x, y;
      if (!kd_part(R, __ldg(refs + j), s0, s1, h, x, y)) continue;
      sum += kd_mass(h, x, y);
      ++na;
    }
    if (na == 0) continue;
    if (na == 1 || R.cdf + sum < 1.f) {
      kd_take_in_order(R, refs, count, s0, s1);
      continue;
    }
    kd_disambiguate(R, refs, count, s0, s1);
  }
}

__global__ void __launch_bounds__(128)
k_kd_sample(TraceScene sc, const int4* __restrict__ nodes, const int* __restrict__ refs, int64_t n_nodes,
            float bx0, float by0, float bz0, float bx1, float by1, float bz1, int64_t n_rays,
            const float* __restrict__ o3, const float* __restrict__ d3, const float* __restrict__ t0a,
            const float* __restrict__ t1a, const float* __restrict__ ua, const float* __restrict__ u2a,
            const int32_t* __restrict__ excl, int32_t* __restrict__ prim_out, float* __restrict__ tsp_out,
            uint8_t* __restrict__ st_out) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= n_rays) return;
  KdRay R;
  R.sc = sc;
  R.ray = make_ray(ld3(o3, r), ld3(d3, r));
  R.t0 = t0a[r];
  R.t1 = t1a[r];
  R.u = ua[r];
  R.u2 = u2a[r];
  R.ex = excl ? excl[r] : -1;
  R.cdf = 0.f;
  R.prim = -1;
  R.done = false;
  R.st = UGP_RAY_OK;
  R.ta_hit = R.tb_hit = R.t1;
  float ta = R.t0, tb = R.t1;
  const float o[3] = {R.ray.o.x, R.ray.o.y, R.ray.o.z}, inv[3] = {R.ray.inv.x, R.ray.inv.y, R.ray.inv.z};
  const float d[3] = {R.ray.d.x, R.ray.d.y, R.ray.d.z};
  const float blo[3] = {bx0, by0, bz0}, bhi[3] = {bx1, by1, bz1};
  for (int a = 0; a < 3; ++a) {
    float x0 = (blo[a] - o[a]) * inv[a], x1 = (bhi[a] - o[a]) * inv[a];
    if (x0 > x1) { const float t = x0; x0 = x1; x1 = t; }
    ta = fmaxf(ta, x0);
    tb = fminf(tb, x1 * (1.f + 1e-6f) + 1e-7f);
  }
  int sn[kKdStack];
  float sa[kKdStack], sb[kKdStack];
  int sp = 0;
  if (n_nodes > 0 && ta < tb) {
    sn[0] = 0; sa[0] = ta; sb[0] = tb;
    sp = 1;
  }
  while (sp > 0 && !R.done && R.st == UGP_RAY_OK) {
    --sp;
    const int node = sn[sp];
    const float a0 = sa[sp], b0 = sb[sp];
    if (!(a0 < b0)) continue;
    if (unsigned(node) >= unsigned(n_nodes)) { R.st = UGP_RAY_BAD_NODE; break; }
    const int4 nd = __ldg(nodes + node);
    if (nd.x == kKdLeafType) {
      kd_leaf(R, refs + nd.z, nd.y, a0, b0);
      continue;
    }
    const int ax = nd.x;
    const float pos = __int_as_float(nd.y);
    const int nearc = (o[ax] < pos || (o[ax] == pos && d[ax] <= 0.f)) ? nd.z : nd.w;
    const int farc = nearc == nd.z ? nd.w : nd.z;
    if (sp + 2 > kKdStack) { R.st = UGP_RAY_STACK_OVERFLOW; break; }
    if (d[ax] == 0.f) {
      sn[sp] = nearc; sa[sp] = a0; sb[sp] = b0; ++sp;
      continue;
    }
    const float ts = (pos - o[ax]) * inv[ax];
    if (ts >= b0 || ts <= 0.f) {
      sn[sp] = nearc; sa[sp] = a0; sb[sp] = b0; ++sp;
    } else if (ts <= a0) {
      sn[sp] = farc; sa[sp] = a0; sb[sp] = b0; ++sp;
    } else {
      sn[sp] = farc; sa[sp] = ts; sb[sp] = b0; ++sp;   // popped after the near side
      sn[sp] = nearc; sa[sp] = a0; sb[sp] = ts; ++sp;
    }
  }
  prim_out[r] = R.done ? R.prim : -1;
  if (tsp_out) tsp_out[r] = R.done ? 0.5f * (R.ta_hit + R.tb_hit) : R.t1;
  if (st_out) st_out[r] = R.st;
}

}  // namespace
}  // namespace ugp

using namespace ugp;

extern "C" size_t ugp_build_kdtree_workspace_size(int64_t n_prims) {
  if (n_prims < 0 || n_prims > (int64_t(1) << 28)) return 0;
  return kd_layout(n_prims).total;
}

extern "C" ugp_status ugp_build_kdtree(const ugp_bvh* bvh, void* workspace, size_t workspace_bytes, void* stream,
                                       ugp_kdtree** out) {
  clear_error();
  if (!out) return fail(UGP_ERR_INVALID_ARG, "ugp_build_kdtree: NULL out");
  *out = nullptr;
  if (!valid_bvh(bvh)) return fail(UGP_ERR_NOT_BUILT, "ugp_build_kdtree: invalid BVH handle");
  const int64_t n = bvh->n_prims;
  if (n > (int64_t(1) << 28)) return fail(UGP_ERR_INVALID_ARG, "ugp_build_kdtree: more than 2^28 primitives");
  const KdLayout L = kd_layout(n);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(UGP_ERR_INVALID_ARG, "ugp_build_kdtree: NULL or misaligned workspace");
  if (workspace_bytes < L.total)
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_build_kdtree: need %zu bytes, got %zu", L.total, workspace_bytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  int4* nodes = reinterpret_cast<int4*>(ws + L.nodes);
  int* final_refs = reinterpret_cast<int*>(ws + L.refs);
  float* aabb = reinterpret_cast<float*>(ws + L.aabb);
  int* refs[2] = {reinterpret_cast<int*>(ws + L.refA), reinterpret_cast<int*>(ws + L.refB)};
  int* rnode[2] = {reinterpret_cast<int*>(ws + L.nodeA), reinterpret_cast<int*>(ws + L.nodeB)};
  LvNode* lv[2] = {reinterpret_cast<LvNode*>(ws + L.lvA), reinterpret_cast<LvNode*>(ws + L.lvB)};
  int* bins = reinterpret_cast<int*>(ws + L.bins);
  int* cnt = reinterpret_cast<int*>(ws + L.cnt);
  int* cursor = reinterpret_cast<int*>(ws + L.cur);
  KdCtl* ctl = reinterpret_cast<KdCtl*>(ws + L.ctl);
  int* root = reinterpret_cast<int*>(ws + L.ctl + 64);

  ugp_kdtree* kd = new ugp_kdtree();
  kd->magic = kKdMagic;
  kd->bvh = bvh;
  kd->nodes = nodes;
  kd->refs = final_refs;
  kd->n_nodes = 0;
  kd->n_refs = 0;
  kd->depth = 0;
  for (int a = 0; a < 6; ++a) kd->box[a] = 0.f;
  if (n == 0) {
    *out = kd;
    return UGP_OK;
  }
  auto bail = [&](ugp_status s) {
    delete kd;
    return s;
  };
  const int T = 256;
  prof_begin(kStBuild, st);
  const int big = 0x7f7fffff;  // ordered-int encodings start at +max float
  const int init[6] = {big, big, big, big, big, big};
  if (cudaMemcpyAsync(root, init, sizeof(init), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(ctl, 0, sizeof(KdCtl), st) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "ugp_build_kdtree: init"));
  k_kd_boxes<<<unsigned((n + T - 1) / T), T, 0, st>>>(n, bvh->prims, bvh->k, aabb, root);
  k_kd_root<<<unsigned((n + T - 1) / T), T, 0, st>>>(n, root, lv[0], refs[0], rnode[0]);
  int m = 1, R = int(n), cur = 0, gid_base = 1, depth = 0;
  int64_t launches = 2;
  KdCtl hc{};
  while (m > 0) {
    if (cudaMemsetAsync(bins, 0, size_t(m) * 6 * kKdBins * 4, st) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "ugp_build_kdtree: memset"));
    k_kd_bin<<<unsigned((R + T - 1) / T), T, 0, st>>>(R, refs[cur], rnode[cur], lv[cur], aabb, bins);
    for (int force = 0; force < 2; ++force) {
      k_kd_choose<<<unsigned((m + T - 1) / T), T, 0, st>>>(m, lv[cur], bins, cnt, force);
      k_kd_count<<<unsigned((R + T - 1) / T), T, 0, st>>>(R, refs[cur], rnode[cur], lv[cur], aabb, cnt);
      k_kd_scan<<<1, 1024, 0, st>>>(m, lv[cur], cnt, ctl);
      launches += 3;
      const cudaError_t e = cudaMemcpyAsync(&hc, ctl, sizeof(KdCtl), cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "ugp_build_kdtree: level counts"));
      // stop splitting when the children's references or nodes would not fit
      const bool fits = int64_t(hc.next_r) <= L.cap_refs && int64_t(gid_base) + hc.next_m <= L.cap_nodes &&
                        int64_t(hc.refs_total) + hc.leaf_refs <= L.cap_refs;
      if (fits) break;
      if (force == 1) return bail(fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_build_kdtree: references exceed 4 n"));
    }
    k_kd_emit<<<unsigned((m + T - 1) / T), T, 0, st>>>(m, lv[cur], cnt, gid_base, nodes, lv[cur ^ 1], cursor);
    k_kd_write<<<unsigned((R + T - 1) / T), T, 0, st>>>(R, refs[cur], rnode[cur], lv[cur], aabb, cnt, cursor,
                                                       refs[cur ^ 1], rnode[cur ^ 1], final_refs);
    launches += 3;
    hc.refs_total += hc.leaf_refs;
    if (cudaMemcpyAsync(&ctl->refs_total, &hc.refs_total, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "ugp_build_kdtree: counts"));
    gid_base += hc.next_m;
    m = hc.next_m;
    R = hc.next_r;
    cur ^= 1;
    ++depth;
  }
  k_kd_sort_leaves<<<unsigned((gid_base + T - 1) / T), T, 0, st>>>(gid_base, nodes, final_refs);
  prof_end(kStBuild, st, int(launches + 1));
  UGP_CUDA_CHECK(cudaGetLastError());
  int rb[6];
  UGP_CUDA_CHECK(cudaMemcpyAsync(rb, root, sizeof(rb), cudaMemcpyDeviceToHost, st));
  UGP_CUDA_CHECK(cudaStreamSynchronize(st));
  for (int a = 0; a < 3; ++a) {
    const int lo = rb[a], hi = rb[3 + a];
    kd->box[a] = o2f_host(lo);
    kd->box[3 + a] = -o2f_host(hi);
  }
  kd->n_nodes = gid_base;
  kd->n_refs = hc.refs_total;
  kd->depth = depth;
  *out = kd;
  return UGP_OK;
}

static bool valid_kd(const ugp_kdtree* kd) { return kd && kd->magic == kKdMagic && valid_bvh(kd->bvh); }

extern "C" void ugp_kdtree_release(ugp_kdtree* kd) {
  if (kd && kd->magic == kKdMagic) {
    kd->magic = 0;
    delete kd;
  }
}

extern "C" ugp_status ugp_kdtree_get_info(const ugp_kdtree* kd, int64_t* n_nodes, int64_t* n_refs, int32_t* depth,
                                          float* box6) {
  clear_error();
  if (!valid_kd(kd)) return fail(UGP_ERR_NOT_BUILT, "ugp_kdtree_get_info: invalid handle");
  if (n_nodes) *n_nodes = kd->n_nodes;
  if (n_refs) *n_refs = kd->n_refs;
  if (depth) *depth = kd->depth;
  if (box6)
    for (int a = 0; a < 6; ++a) box6[a] = kd->box[a];
  return UGP_OK;
}

extern "C" ugp_status ugp_kdtree_export(const ugp_kdtree* kd, int32_t* nodes4_host, int32_t* refs_host) {
  clear_error();
  if (!valid_kd(kd)) return fail(UGP_ERR_NOT_BUILT, "ugp_kdtree_export: invalid handle");
  if ((kd->n_nodes > 0 && !nodes4_host) || (kd->n_refs > 0 && !refs_host))
    return fail(UGP_ERR_INVALID_ARG, "ugp_kdtree_export: NULL output");
  if (kd->n_nodes > 0)
    UGP_CUDA_CHECK(cudaMemcpy(nodes4_host, kd->nodes, size_t(kd->n_nodes) * 16, cudaMemcpyDeviceToHost));
  if (kd->n_refs > 0) {
    UGP_CUDA_CHECK(cudaMemcpy(refs_host, kd->refs, size_t(kd->n_refs) * 4, cudaMemcpyDeviceToHost));
    // slots to the caller's primitive indices (record word 13)
    std::vector<float4> r3(size_t(kd->bvh->n_prims));
    UGP_CUDA_CHECK(cudaMemcpy2D(r3.data(), sizeof(float4), kd->bvh->prims + 3, 4 * sizeof(float4), sizeof(float4),
                                size_t(kd->bvh->n_prims), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < kd->n_refs; ++i) {
      const int slot = refs_host[i];
      if (slot < 0 || slot >= kd->bvh->n_prims) return fail(UGP_ERR_CUDA, "ugp_kdtree_export: bad reference");
      float y = r3[size_t(slot)].y;
      int id;
      memcpy(&id, &y, 4);
      refs_host[i] = id;
    }
  }
  return UGP_OK;
}

extern "C" ugp_status ugp_sample_free_flight_kdtree(const ugp_kdtree* kd, int64_t n_rays, const float* o3,
                                                    const float* d3, const float* t0, const float* t1,
                                                    const float* u, const float* u2, const int32_t* exclude_prim,
                                                    int32_t* prim_out, float* t_spawn_out, uint8_t* status_out,
                                                    void* stream) {
  clear_error();
  if (!valid_kd(kd)) return fail(UGP_ERR_NOT_BUILT, "ugp_sample_free_flight_kdtree: invalid handle");
  const ugp_status s = check_rays("ugp_sample_free_flight_kdtree", kd->bvh, n_rays, o3, d3, t0, t1);
  if (s != UGP_OK) return s;
  if (n_rays > 0 && (!u || !u2 || !prim_out))
    return fail(UGP_ERR_INVALID_ARG, "ugp_sample_free_flight_kdtree: NULL uniform or output array");
  if (n_rays == 0) return UGP_OK;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_begin(kStQuery, st);
  k_kd_sample<<<unsigned((n_rays + 127) / 128), 128, 0, st>>>(
      trace_scene(kd->bvh), kd->nodes, kd->refs, kd->n_nodes, kd->box[0], kd->box[1], kd->box[2], kd->box[3],
      kd->box[4], kd->box[5], n_rays, o3, d3, t0, t1, u, u2, exclude_prim, prim_out, t_spawn_out, status_out);
  prof_end(kStQuery, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}
