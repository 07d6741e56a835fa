// BVH construction over the primitives' bounding ellipsoids (Sec. 4.1, Eq. 4)
// and the per-primitive precompute of Eq. 1-2.
//
// Steps, all on the caller's stream:
//   1. k_prim_bounds   per primitive: rotation from the quaternion, bounding box of
//                      the k-ellipsoid, block-reduced centroid bounds
//   2. k_morton        30-bit Morton code of each box centre
//   3. radix sort      (ugp_sort.cu, on the caller's workspace) of (code, index), stable
//   4. k_hierarchy     binary radix tree over the sorted codes (Karras, HPG 2012)
//   5. k_records       64-byte hot records in leaf order (W = S^-1 R^T, mu, g0, index) and
//                      the low float parts of W (48 B, read only by ill-conditioned hits)
//   6. k_refit         bottom-up child boxes with one atomic counter per node
//   7. k_collapse4     the 4-wide quantised tree: each binary internal node at even depth with
//                      its children and grandchildren (layout in ugp_internal.cuh)

#include <math.h>
#include <string.h>

#include "ugp_internal.cuh"

namespace ugp {
namespace {


struct Layout {
  size_t prims, nodes, nodes4, wlo, persistent;
  size_t aabb, keys0, keys1, vals0, vals1, parent, flags, bounds, sort, total;
};

__device__ __forceinline__ int f2o(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// Rotation matrix (row-major) of the normalised quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rot(float4 q, float R[9]) {
  const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ bool prim_valid(float3 m, float4 q, float3 s, float c) {
  const float qn = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  return isfinite(m.x) && isfinite(m.y) && isfinite(m.z) && isfinite(qn) && qn > 1e-20f &&
         isfinite(s.x) && isfinite(s.y) && isfinite(s.z) && s.x > 0.f && s.y > 0.f && s.z > 0.f &&
         isfinite(c) && c >= 0.f;
}

__device__ __forceinline__ float3 ld3(const float* p, int64_t i) {
  return make_float3(p[3 * i], p[3 * i + 1], p[3 * i + 2]);
}
__device__ __forceinline__ float4 ld4(const float* p, int64_t i) {
  return make_float4(p[4 * i], p[4 * i + 1], p[4 * i + 2], p[4 * i + 3]);
}

// Bounding box of the k-ellipsoid x = mu + k R S v, |v| = 1: half extent along axis i is
// k * sqrt(sum_j (R_ij s_j)^2).  Widened by a few float32 ulps so the box stays
// conservative for the float32 interval test.
__global__ void k_prim_bounds(int64_t n, const float* __restrict__ mean3, const float* __restrict__ quat4,
                              const float* __restrict__ scale3, const float* __restrict__ mag, float k,
                              float4* __restrict__ aabb, int* __restrict__ bounds,
                              unsigned long long* __restrict__ n_invalid) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  float cx = 0.f, cy = 0.f, cz = 0.f;
  bool has = false;
  if (i < n) {
    const float3 m = ld3(mean3, i);
    const float4 q = ld4(quat4, i);
    const float3 s = ld3(scale3, i);
    const float c = mag[i];
    if (prim_valid(m, q, s, c)) {
      float R[9];
      quat_rot(q, R);
      float e[3];
      const float mm[3] = {m.x, m.y, m.z};
      for (int r = 0; r < 3; ++r) {
        const float a = R[3 * r] * s.x, b = R[3 * r + 1] * s.y, d = R[3 * r + 2] * s.z;
        e[r] = k * sqrtf(a * a + b * b + d * d) * (1.f + 4e-6f) + 2e-7f * fabsf(mm[r]);
      }
      aabb[2 * i] = make_float4(m.x - e[0], m.y - e[1], m.z - e[2], 0.f);
      aabb[2 * i + 1] = make_float4(m.x + e[0], m.y + e[1], m.z + e[2], 0.f);
      cx = m.x; cy = m.y; cz = m.z;
      has = true;
    } else {
      // An invalid primitive keeps a point box; its record is flagged and never hit.
      const float x = isfinite(m.x) ? m.x : 0.f, y = isfinite(m.y) ? m.y : 0.f,
                  z = isfinite(m.z) ? m.z : 0.f;
      aabb[2 * i] = make_float4(x, y, z, 0.f);
      aabb[2 * i + 1] = make_float4(x, y, z, 0.f);
      atomicAdd(n_invalid, 1ull);
    }
  }
  // Centroid bounds: warp min-reduction of the ordered-int encodings, one atomic per warp.
  const float big = 3.0e38f;
  const float v[6] = {has ? cx : big, has ? cy : big, has ? cz : big,
                      has ? -cx : big, has ? -cy : big, has ? -cz : big};
  for (int a = 0; a < 6; ++a) {
    const int r = __reduce_min_sync(0xffffffffu, f2o(v[a]));
    if ((threadIdx.x & 31) == 0) atomicMin(&bounds[a], r);
  }
}

__device__ __forceinline__ uint32_t expand10(uint32_t v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

__global__ void k_morton(int64_t n, const float4* __restrict__ aabb, const int* __restrict__ bounds,
                         uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float lo[3] = {o2f(bounds[0]), o2f(bounds[1]), o2f(bounds[2])};
  const float hi[3] = {-o2f(bounds[3]), -o2f(bounds[4]), -o2f(bounds[5])};
  const float4 a = aabb[2 * i], b = aabb[2 * i + 1];
  const float c[3] = {0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z)};
  uint32_t code = 0;
  for (int ax = 0; ax < 3; ++ax) {
    const float ext = hi[ax] - lo[ax];
    float t = ext > 0.f ? (c[ax] - lo[ax]) / ext : 0.5f;
    t = fminf(fmaxf(t * 1024.f, 0.f), 1023.f);
    code |= expand10(uint32_t(t)) << (2 - ax);
  }
  keys[i] = code;
  vals[i] = int32_t(i);
}

__device__ __forceinline__ int delta(const uint32_t* __restrict__ keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  const uint32_t a = keys[i], b = keys[j];
  if (a == b) return 32 + __clz(uint32_t(i) ^ uint32_t(j));
  return __clz(a ^ b);
}

// One internal node per thread (n - 1 of them); node 0 is the root.
__global__ void k_hierarchy(int n, const uint32_t* __restrict__ keys, int4* __restrict__ nodes,
                            int32_t* __restrict__ parent_int, int32_t* __restrict__ parent_leaf) {
  const int i = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = delta(keys, n, i, i - d);
  int lmax = 2;
  while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
  const int j = i + l * d;
  const int dnode = delta(keys, n, i, j);
  int s = 0;
  for (int div = 2;; div <<= 1) {
    const int t = (l + div - 1) / div;
    if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    if (t <= 1) break;
  }
  const int g = i + s * d + min(d, 0);
  const int lo = min(i, j), hi = max(i, j);
  int c0, c1;
  if (lo == g) { c0 = ~g;      parent_leaf[g] = (i << 1) | 0; }
  else         { c0 = g;       parent_int[g] = (i << 1) | 0; }
  if (hi == g + 1) { c1 = ~(g + 1); parent_leaf[g + 1] = (i << 1) | 1; }
  else             { c1 = g + 1;    parent_int[g + 1] = (i << 1) | 1; }
  nodes[4 * i + 3] = make_int4(c0, c1, 0, 0);
  if (i == 0) parent_int[0] = -1;
}

__global__ void k_single_root(int4* nodes, int32_t* parent_leaf, int32_t* parent_int) {
  nodes[3] = make_int4(~0, kEmptyChild, 0, 0);
  parent_leaf[0] = 0;
  parent_int[0] = -1;
}

// Hot record of the primitive in leaf slot `slot` (layout in ugp_internal.cuh), plus the
// low-order float parts of W for the double-float refinement of ill-conditioned hits.  W is
// formed in double precision from the float32 inputs and split as W = hi + lo.
__global__ void k_records(int64_t n, const int32_t* __restrict__ order, const float* __restrict__ mean3,
                          const float* __restrict__ quat4, const float* __restrict__ scale3,
                          const float* __restrict__ mag, float4* __restrict__ recs,
                          float4* __restrict__ wlo) {
  const int64_t slot = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (slot >= n) return;
  const int64_t i = order[slot];
  const float3 m = ld3(mean3, i);
  const float4 q = ld4(quat4, i);
  const float3 s = ld3(scale3, i);
  const float c = mag[i];
  float4 r0, r1, r2, r3, l0, l1, l2;
  if (prim_valid(m, q, s, c)) {
    const double qn = sqrt(double(q.x) * q.x + double(q.y) * q.y + double(q.z) * q.z + double(q.w) * q.w);
    const double w = q.x / qn, x = q.y / qn, y = q.z / qn, z = q.w / qn;
    const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                         2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                         2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
    const double is[3] = {1.0 / s.x, 1.0 / s.y, 1.0 / s.z};
    float hi[9], lo[9];
    for (int r = 0; r < 3; ++r)
      for (int cc = 0; cc < 3; ++cc) {
        const double v = R[3 * cc + r] * is[r];  // W_rc = R_cr / s_r
        hi[3 * r + cc] = float(v);
        lo[3 * r + cc] = float(v - double(hi[3 * r + cc]));
      }
    r0 = make_float4(hi[0], hi[1], hi[2], m.x);
    r1 = make_float4(hi[3], hi[4], hi[5], m.y);
    r2 = make_float4(hi[6], hi[7], hi[8], m.z);
    l0 = make_float4(lo[0], lo[1], lo[2], 0.f);
    l1 = make_float4(lo[3], lo[4], lo[5], 0.f);
    l2 = make_float4(lo[6], lo[7], lo[8], 0.f);
    // (2 pi)^{3/2} = 15.749609945722419
    const float g0 = float(double(c) / (15.749609945722419 * double(s.x) * double(s.y) * double(s.z)));
    r3 = make_float4(g0, __int_as_float(int(i)), 1.f, 0.f);
  } else {
    r0 = r1 = r2 = l0 = l1 = l2 = make_float4(0.f, 0.f, 0.f, 0.f);
    r3 = make_float4(0.f, __int_as_float(int(i)), 0.f, 0.f);
  }
  recs[4 * slot + 0] = r0;
  recs[4 * slot + 1] = r1;
  recs[4 * slot + 2] = r2;
  recs[4 * slot + 3] = r3;
  wlo[3 * slot + 0] = l0;
  wlo[3 * slot + 1] = l1;
  wlo[3 * slot + 2] = l2;
}

__device__ __forceinline__ void store_child_box(float* node, int side, const float b[6]) {
  float* p = node + (side ? 6 : 0);
  for (int k = 0; k < 6; ++k) p[k] = b[k];
}

// Bottom-up boxes: each leaf writes its box into its parent, and the second of a node's
// two children to arrive forms the union and continues upwards.
__global__ void k_refit(int n, const int32_t* __restrict__ order, const float4* __restrict__ aabb,
                        const int32_t* __restrict__ parent_int, const int32_t* __restrict__ parent_leaf,
                        int* __restrict__ flags, float* __restrict__ nodes_f, float* __restrict__ root_box) {
  const int slot = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (slot >= n) return;
  const int i = order[slot];
  const float4 lo = aabb[2 * i], hi = aabb[2 * i + 1];
  float b[6] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z};
  int ps = parent_leaf[slot];
  while (true) {
    const int p = ps >> 1, side = ps & 1;
    store_child_box(nodes_f + 16 * size_t(p), side, b);
    __threadfence();
    if (atomicAdd(&flags[p], 1) == 0) return;
    __threadfence();
    const float* nd = nodes_f + 16 * size_t(p);
    float c0[6], c1[6];
    for (int k = 0; k < 6; ++k) { c0[k] = __ldcg(nd + k); c1[k] = __ldcg(nd + 6 + k); }
    const int4 ch = *reinterpret_cast<const int4*>(nd + 12);
    if (ch.y == kEmptyChild) {
      for (int k = 0; k < 6; ++k) b[k] = c0[k];
    } else {
      for (int k = 0; k < 3; ++k) { b[k] = fminf(c0[k], c1[k]); b[3 + k] = fmaxf(c0[3 + k], c1[3 + k]); }
    }
    ps = parent_int[p];
    if (ps < 0) {
      for (int k = 0; k < 6; ++k) root_box[k] = b[k];
      return;
    }
  }
}

// One 4-wide node per binary internal node at even depth (the root has depth 0): its children,
// with every internal child replaced by that child's two children (odd-depth nodes are absorbed
// into their parent). Boxes are quantised outwards to 8 bits per face against a grid of spacing
// 2^e_a per axis anchored at the union's low corner.
__global__ void k_collapse4(int n_int, const float4* __restrict__ nodes, const int32_t* __restrict__ depth,
                            uint4* __restrict__ nodes4) {
  const int i = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_int) return;
  if (depth[i] & 1) return;
  float box[4][6];
  int ref[4];
  int m = 0;
  auto child_of = [&](int node, int side, float b[6], int& r) {
    const float4* nd = nodes + 4 * size_t(node);
    const float4 n0 = nd[0], n1 = nd[1], n2 = nd[2];
    const int4 n3 = reinterpret_cast<const int4*>(nd)[3];
    r = side ? n3.y : n3.x;
    if (side == 0) { b[0] = n0.x; b[1] = n0.y; b[2] = n0.z; b[3] = n0.w; b[4] = n1.x; b[5] = n1.y; }
    else           { b[0] = n1.z; b[1] = n1.w; b[2] = n2.x; b[3] = n2.y; b[4] = n2.z; b[5] = n2.w; }
  };
  for (int side = 0; side < 2; ++side) {
    float b[6];
    int r;
    child_of(i, side, b, r);
    if (r == kEmptyChild) continue;
    if (r < 0) {
      for (int k = 0; k < 6; ++k) box[m][k] = b[k];
      ref[m++] = r;
      continue;
    }
    for (int s2 = 0; s2 < 2; ++s2) {
      float g[6];
      int rg;
      child_of(r, s2, g, rg);
      if (rg == kEmptyChild) continue;
      for (int k = 0; k < 6; ++k) box[m][k] = g[k];
      ref[m++] = rg;
    }
  }
  float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
  for (int c = 0; c < m; ++c)
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(lo[a], box[c][a]);
      hi[a] = fmaxf(hi[a], box[c][3 + a]);
    }
  uint32_t qlo[3] = {0u, 0u, 0u}, qhi[3] = {0u, 0u, 0u}, ex = 0u;
  for (int a = 0; a < 3; ++a) {
    // a power-of-two spacing 2^e >= extent / 254 (frexp: extent / 254 = f 2^e, f in [1/2, 1));
    // the spare step absorbs the rounding of o + q 2^e
    const float ext = hi[a] - lo[a];
    int e = -126;
    if (ext > 0.f) {
      frexpf(ext * (1.f / 254.f) * (1.f + 1e-6f), &e);
      e = max(-126, min(e, 126));
    }
    const float sp = ldexpf(1.f, e), isp = ldexpf(1.f, -e);
    for (int c = 0; c < m; ++c) {
      int ql = int(floorf((box[c][a] - lo[a]) * isp));
      int qh = int(ceilf((box[c][3 + a] - lo[a]) * isp));
      ql = max(0, min(ql, 255));
      qh = max(0, min(qh, 255));
      while (ql > 0 && fmaf(float(ql), sp, lo[a]) > box[c][a]) --ql;
      while (qh < 255 && fmaf(float(qh), sp, lo[a]) < box[c][3 + a]) ++qh;
      qlo[a] |= uint32_t(ql) << (8 * c);
      qhi[a] |= uint32_t(qh) << (8 * c);
    }
    // an empty child slot gets an inverted box (low face 255, high face 0) that no ray enters,
    // so the node test needs no separate check for it
    for (int c = m; c < 4; ++c) qlo[a] |= 255u << (8 * c);
    ex |= uint32_t(e + 128) << (8 * a);
  }
  int r4[4] = {kEmptyChild, kEmptyChild, kEmptyChild, kEmptyChild};
  for (int c = 0; c < m; ++c) r4[c] = ref[c];
  uint4* q = nodes4 + 4 * size_t(i);
  q[0] = make_uint4(__float_as_uint(lo[0]), __float_as_uint(lo[1]), __float_as_uint(lo[2]), ex);
  q[1] = make_uint4(qlo[0], qlo[1], qlo[2], qhi[0]);
  q[2] = make_uint4(qhi[1], qhi[2], 0u, 0u);
  q[3] = make_uint4(uint32_t(r4[0]), uint32_t(r4[1]), uint32_t(r4[2]), uint32_t(r4[3]));
}

// Depth of every internal node by pointer jumping: each round adds the distance to the current
// ancestor and jumps to that ancestor's ancestor, so kJumps rounds reach the root of any tree up
// to 2^kJumps deep (binary radix trees over 32-bit keys with index tie-breaks are at most 64 deep).
constexpr int kJumps = 7;
__global__ void k_depth_init(int n_int, const int32_t* __restrict__ parent_int, int32_t* __restrict__ anc,
                             int32_t* __restrict__ dist) {
  const int i = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_int) return;
  const int p = parent_int[i];
  anc[i] = p >= 0 ? (p >> 1) : -1;
  dist[i] = p >= 0 ? 1 : 0;
}
__global__ void k_depth_jump(int n_int, const int32_t* __restrict__ anc_in, const int32_t* __restrict__ dist_in,
                             int32_t* __restrict__ anc_out, int32_t* __restrict__ dist_out) {
  const int i = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_int) return;
  const int a = anc_in[i];
  if (a >= 0) {
    dist_out[i] = dist_in[i] + dist_in[a];
    anc_out[i] = anc_in[a];
  } else {
    dist_out[i] = dist_in[i];
    anc_out[i] = -1;
  }
}

__global__ void k_init_bounds(int* bounds, int* n_flags_zero_dummy) {
  if (threadIdx.x < 6) bounds[threadIdx.x] = f2o(3.0e38f);
}

// For n == 1 the single child needs its box too; the empty child gets a box nobody reaches.
__global__ void k_single_refit(const float4* __restrict__ aabb, float* nodes_f, float* root_box) {
  const float4 lo = aabb[0], hi = aabb[1];
  const float b[6] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z};
  for (int k = 0; k < 6; ++k) { nodes_f[k] = b[k]; nodes_f[6 + k] = 0.f; root_box[k] = b[k]; }
}

bool layout_for(int64_t n, Layout* L) {
  const size_t N = size_t(n);
  const size_t ni = N > 1 ? N - 1 : 1;
  size_t off = 0;
  L->prims = off;      off = align256(off + N * 64);
  L->nodes = off;      off = align256(off + ni * 64);
  L->nodes4 = off;     off = align256(off + ni * 64);
  L->wlo = off;        off = align256(off + N * 48);
  L->bounds = off;     off = align256(off + 64);   // 6 ordered-int bounds, root box, invalid count
  L->persistent = off;
  L->aabb = off;       off = align256(off + N * 32);
  L->keys0 = off;      off = align256(off + N * 4);
  L->keys1 = off;      off = align256(off + N * 4);
  L->vals0 = off;      off = align256(off + N * 4);
  L->vals1 = off;      off = align256(off + N * 4);
  L->parent = off;     off = align256(off + (ni + N) * 4);
  L->flags = off;      off = align256(off + ni * 4);
  L->sort = off;       off = align256(off + radix_sort_workspace(int64_t(N)));
  L->total = off;
  return true;
}

}  // namespace
}  // namespace ugp

using namespace ugp;

extern "C" size_t ugp_build_bvh_workspace_size(int64_t n_prims) {
  if (n_prims < 0 || n_prims > (int64_t(1) << 30)) return 0;
  Layout L;
  if (!layout_for(n_prims, &L)) return 0;
  return L.total;
}

extern "C" ugp_status ugp_build_bvh(const ugp_prims* prims, float cutoff_eps, void* workspace,
                                    size_t workspace_bytes, void* stream_, ugp_bvh** out) {
  clear_error();
  if (!prims || !out) return fail(UGP_ERR_INVALID_ARG, "ugp_build_bvh: prims and out must be non-NULL");
  *out = nullptr;
  const int64_t n = prims->n;
  if (n < 0 || n > (int64_t(1) << 30))
    return fail(UGP_ERR_INVALID_ARG, "ugp_build_bvh: n_prims %lld out of range [0, 2^30]", (long long)n);
  if (!(cutoff_eps > 0.f && cutoff_eps < 1.f))
    return fail(UGP_ERR_INVALID_ARG, "ugp_build_bvh: cutoff_eps %g not in (0, 1)", double(cutoff_eps));
  if (n > 0 && (!prims->mean3 || !prims->quat4 || !prims->scale3 || !prims->magnitude))
    return fail(UGP_ERR_INVALID_ARG, "ugp_build_bvh: NULL primitive array");
  if (n > 0 && !workspace) return fail(UGP_ERR_INVALID_ARG, "ugp_build_bvh: NULL workspace");
  if (reinterpret_cast<uintptr_t>(workspace) & 255)
    return fail(UGP_ERR_INVALID_ARG, "ugp_build_bvh: workspace must be 256-byte aligned");
  Layout L;
  if (!layout_for(n, &L)) return fail(UGP_ERR_CUDA, "ugp_build_bvh: sort workspace query failed");
  if (workspace_bytes < L.total)
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_build_bvh: need %zu bytes, got %zu", L.total,
                workspace_bytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  const double kd = sqrt(-2.0 * log(double(cutoff_eps)));

  ugp_bvh* b = new ugp_bvh();
  b->magic = kBvhMagic;
  UGP_CUDA_CHECK(cudaGetDevice(&b->device));
  b->n_prims = n;
  b->n_nodes = n > 1 ? n - 1 : (n == 1 ? 1 : 0);
  b->k = float(kd);
  b->k2 = float(kd * kd);
  char* ws = static_cast<char*>(workspace);
  b->prims = reinterpret_cast<const float4*>(ws + L.prims);
  b->wlo = reinterpret_cast<const float4*>(ws + L.wlo);
  b->nodes = reinterpret_cast<const float4*>(ws + L.nodes);
  b->nodes4 = reinterpret_cast<const uint4*>(ws + L.nodes4);
  b->persistent_bytes = L.persistent;
  b->bounds_dev = reinterpret_cast<const float*>(ws + L.bounds);
  if (n == 0) {
    *out = b;
    return UGP_OK;
  }
  float4* aabb = reinterpret_cast<float4*>(ws + L.aabb);
  int* bounds = reinterpret_cast<int*>(ws + L.bounds);
  float* root_box = reinterpret_cast<float*>(ws + L.bounds + 32);
  unsigned long long* n_invalid = reinterpret_cast<unsigned long long*>(ws + L.bounds + 56);
  uint32_t* k0 = reinterpret_cast<uint32_t*>(ws + L.keys0);
  uint32_t* k1 = reinterpret_cast<uint32_t*>(ws + L.keys1);
  int32_t* v0 = reinterpret_cast<int32_t*>(ws + L.vals0);
  int32_t* v1 = reinterpret_cast<int32_t*>(ws + L.vals1);
  const size_t ni = n > 1 ? size_t(n - 1) : 1;
  int32_t* parent_int = reinterpret_cast<int32_t*>(ws + L.parent);
  int32_t* parent_leaf = parent_int + ni;
  int* flags = reinterpret_cast<int*>(ws + L.flags);

  const int T = 256;
  const unsigned G = unsigned((n + T - 1) / T);
  prof_begin(kStBuild, st);
  UGP_CUDA_CHECK(cudaMemsetAsync(ws + L.bounds, 0, 64, st));
  k_init_bounds<<<1, 32, 0, st>>>(bounds, nullptr);
  k_prim_bounds<<<G, T, 0, st>>>(n, prims->mean3, prims->quat4, prims->scale3, prims->magnitude, b->k,
                                 aabb, bounds, n_invalid);
  UGP_CUDA_CHECK(cudaGetLastError());
  int4* nodes_i = reinterpret_cast<int4*>(ws + L.nodes);
  float* nodes_f = reinterpret_cast<float*>(ws + L.nodes);
  int32_t* order = v0;
  if (n == 1) {
    UGP_CUDA_CHECK(cudaMemsetAsync(v0, 0, 4, st));
    k_single_root<<<1, 1, 0, st>>>(nodes_i, parent_leaf, parent_int);
    k_single_refit<<<1, 1, 0, st>>>(aabb, nodes_f, root_box);
  } else {
    k_morton<<<G, T, 0, st>>>(n, aabb, bounds, k0, v0);
    UGP_CUDA_CHECK(cudaGetLastError());
    const ugp_status ss = radix_sort_pairs(k0, k1, v0, v1, n, 30, ws + L.sort, st);
    if (ss != UGP_OK) return ss;
    const bool in1 = (radix_sort_passes(30) & 1) != 0;
    order = in1 ? v1 : v0;
    k_hierarchy<<<unsigned((n - 1 + T - 1) / T), T, 0, st>>>(int(n), in1 ? k1 : k0, nodes_i, parent_int, parent_leaf);
    UGP_CUDA_CHECK(cudaGetLastError());
    UGP_CUDA_CHECK(cudaMemsetAsync(flags, 0, (n - 1) * 4, st));
    k_refit<<<G, T, 0, st>>>(int(n), order, aabb, parent_int, parent_leaf, flags, nodes_f, root_box);
    UGP_CUDA_CHECK(cudaGetLastError());
  }
  k_records<<<G, T, 0, st>>>(n, order, prims->mean3, prims->quat4, prims->scale3, prims->magnitude,
                             reinterpret_cast<float4*>(ws + L.prims), reinterpret_cast<float4*>(ws + L.wlo));
  UGP_CUDA_CHECK(cudaGetLastError());
  {
    // depths by pointer jumping in the sort's key and value arrays (free after k_records)
    const int n_int = int(b->n_nodes);
    const unsigned Gi = unsigned((n_int + T - 1) / T);
    int32_t* anc[2] = {reinterpret_cast<int32_t*>(k0), v0};
    int32_t* dist[2] = {reinterpret_cast<int32_t*>(k1), flags};
    k_depth_init<<<Gi, T, 0, st>>>(n_int, parent_int, anc[0], dist[0]);
    for (int r = 0; r < kJumps; ++r)
      k_depth_jump<<<Gi, T, 0, st>>>(n_int, anc[r & 1], dist[r & 1], anc[(r + 1) & 1], dist[(r + 1) & 1]);
    k_collapse4<<<Gi, T, 0, st>>>(n_int, reinterpret_cast<const float4*>(ws + L.nodes), dist[kJumps & 1],
                                  reinterpret_cast<uint4*>(ws + L.nodes4));
    UGP_CUDA_CHECK(cudaGetLastError());
  }
  // own kernels, the radix sort's three per 8-bit digit of the 30-bit codes among them
  prof_end(kStBuild, st, (n == 1 ? 5 : 6 + 3 * radix_sort_passes(30)) + 2 + kJumps);
  b->stream = st;
  *out = b;
  return UGP_OK;
}

extern "C" void ugp_bvh_release(ugp_bvh* bvh) {
  if (bvh && bvh->magic == kBvhMagic) {
    bvh->magic = 0;
    delete bvh;
  }
}

extern "C" ugp_status ugp_bvh_get_info(const ugp_bvh* bvh, ugp_bvh_info* out) {
  clear_error();
  if (!valid_bvh(bvh)) return fail(UGP_ERR_NOT_BUILT, "ugp_bvh_get_info: invalid handle");
  if (!out) return fail(UGP_ERR_INVALID_ARG, "ugp_bvh_get_info: NULL out");
  out->n_prims = bvh->n_prims;
  out->n_nodes = bvh->n_nodes;
  out->cutoff_k = bvh->k;
  out->persistent_bytes = bvh->persistent_bytes;
  out->n_invalid = 0;
  for (int k = 0; k < 3; ++k) { out->bounds_lo[k] = 0.f; out->bounds_hi[k] = 0.f; }
  if (bvh->n_prims > 0) {
    float hb[16];
    UGP_CUDA_CHECK(cudaStreamSynchronize(bvh->stream));
    UGP_CUDA_CHECK(cudaMemcpy(hb, bvh->bounds_dev, 64, cudaMemcpyDeviceToHost));
    for (int k = 0; k < 3; ++k) { out->bounds_lo[k] = hb[8 + k]; out->bounds_hi[k] = hb[11 + k]; }
    unsigned long long inv;
    memcpy(&inv, reinterpret_cast<const char*>(hb) + 56, 8);
    out->n_invalid = int64_t(inv);
  }
  return UGP_OK;
}
