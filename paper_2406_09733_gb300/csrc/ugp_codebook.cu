// Codebook-quantised primitive records (the compression the paper pairs with its level-of-detail
// scheme: per-attribute codebooks with random-access decoding).
//
// A record keeps the mean and the magnitude in float32 and replaces each other attribute group by
// the 12-bit index of its nearest codebook entry:
//   scale      (log s_x, log s_y, log s_z)                         3 values
//   rotation   the unit quaternion with w >= 0 (q and -q are one rotation)   4 values
//   SGGX       (Sxx, Syy, Szz, Sxy, Sxz, Syz)                        6 values
//   material   albedo 3, roughness, emission 3, Disney 9             16 values
// plus the material type (4 bits, exact). 24 bytes per primitive:
//   bytes 0-11 mean (float x3), 12-15 magnitude (float), 16-17 scale code, 18-19 rotation code,
//   20-21 SGGX code, 22-23 material code | type << 12.
// Each codebook has kCodes entries, fitted by Lloyd iterations on the device: every point goes
// to its nearest entry (squared distance, ties to the lower index), then every entry with points
// moves to their mean. The sums are 64-bit fixed point (units of 2^-24), so the fit does not
// depend on the order of the atomic additions. Entries start at the points of index
// floor(k n / kCodes).
#include <math.h>
#include <string.h>

#include "ugp_internal.cuh"

namespace ugp {
namespace {

constexpr int kCodes = 4096;
constexpr int kGroups = 4;
constexpr int kDim[kGroups] = {3, 4, 6, 16};
constexpr int kOff[kGroups] = {0, 3, 7, 13};  // offsets of the groups in a 29-value feature row
constexpr int kFeat = 29;
constexpr float kFix = 16777216.f;  // 2^24

__host__ __device__ constexpr size_t book_floats() { return size_t(kCodes) * kFeat; }

// Feature row of primitive i (the values each codebook quantises).
__global__ void k_features(int64_t n, const float* __restrict__ quat4, const float* __restrict__ scale3,
                           const float* __restrict__ sggx6, const float* __restrict__ albedo3,
                           const float* __restrict__ rough, const float* __restrict__ emit3,
                           const float* __restrict__ dis9, float* __restrict__ X) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float* x = X + i * kFeat;
  for (int a = 0; a < 3; ++a) x[a] = logf(fmaxf(scale3[3 * i + a], 1e-30f));
  float q[4] = {quat4[4 * i], quat4[4 * i + 1], quat4[4 * i + 2], quat4[4 * i + 3]};
  const float inv = rsqrtf(fmaxf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3], 1e-30f));
  const float sg = q[0] < 0.f ? -inv : inv;
  for (int a = 0; a < 4; ++a) x[3 + a] = q[a] * sg;
  for (int a = 0; a < 6; ++a) x[7 + a] = sggx6[6 * i + a];
  for (int a = 0; a < 3; ++a) x[13 + a] = albedo3[3 * i + a];
  x[16] = rough[i];
  for (int a = 0; a < 3; ++a) x[17 + a] = emit3[3 * i + a];
  for (int a = 0; a < 9; ++a) x[20 + a] = dis9 ? dis9[9 * i + a] : 0.f;
}

// Entries start at the points of index floor(k n / kCodes).
__global__ void k_init_book(int64_t n, const float* __restrict__ X, float* __restrict__ book) {
  const int k = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= kCodes) return;
  const int64_t i = (int64_t(k) * n) / kCodes;
  for (int f = 0; f < kFeat; ++f) book[size_t(k) * kFeat + f] = X[i * kFeat + f];
}

// Nearest entry of group G for every point (ties to the lower index), entries staged in shared
// memory 512 at a time.
template <int G>
__global__ void __launch_bounds__(256) k_assign(int64_t n, const float* __restrict__ X,
                                                const float* __restrict__ book, uint16_t* __restrict__ code) {
  constexpr int D = kDim[G], O = kOff[G], kTile = 512;
  __shared__ float cb[kTile * D];
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  float x[D];
#pragma unroll
  for (int d = 0; d < D; ++d) x[d] = i < n ? X[i * kFeat + O + d] : 0.f;
  float best = INFINITY;
  int bk = 0;
  for (int t0 = 0; t0 < kCodes; t0 += kTile) {
    __syncthreads();
    for (int e = threadIdx.x; e < kTile * D; e += blockDim.x)
      cb[e] = book[size_t(t0 + e / D) * kFeat + O + e % D];
    __syncthreads();
    for (int k = 0; k < kTile; ++k) {
      float d2 = 0.f;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float v = x[d] - cb[k * D + d];
        d2 = fmaf(v, v, d2);
      }
      if (d2 < best) {
        best = d2;
        bk = t0 + k;
      }
    }
  }
  if (i < n) code[i] = uint16_t(bk);
}

// Fixed-point sums and counts of the points of every entry of group G.
template <int G>
__global__ void k_accumulate(int64_t n, const float* __restrict__ X, const uint16_t* __restrict__ code,
                             unsigned long long* __restrict__ sums, unsigned int* __restrict__ cnt) {
  constexpr int D = kDim[G], O = kOff[G];
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = code[i];
  atomicAdd(cnt + k, 1u);
  for (int d = 0; d < D; ++d)
    atomicAdd(sums + size_t(k) * D + d, (unsigned long long)__float2ll_rn(X[i * kFeat + O + d] * kFix));
}

// Entries with points move to their mean; the others stay.
template <int G>
__global__ void k_update(const unsigned long long* __restrict__ sums, const unsigned int* __restrict__ cnt,
                         float* __restrict__ book) {
  constexpr int D = kDim[G], O = kOff[G];
  const int k = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= kCodes || cnt[k] == 0) return;
  for (int d = 0; d < D; ++d) {
    const long long s = (long long)sums[size_t(k) * D + d];
    book[size_t(k) * kFeat + O + d] = float(double(s) / (double(kFix) * double(cnt[k])));
  }
}

__global__ void k_pack(int64_t n, const float* __restrict__ mean3, const float* __restrict__ mag,
                       const uint8_t* __restrict__ type, const uint16_t* __restrict__ codes,
                       uint32_t* __restrict__ rec) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t* r = rec + 6 * i;
  r[0] = __float_as_uint(mean3[3 * i]);
  r[1] = __float_as_uint(mean3[3 * i + 1]);
  r[2] = __float_as_uint(mean3[3 * i + 2]);
  r[3] = __float_as_uint(mag[i]);
  const uint32_t cs = codes[i], cr = codes[n + i], cg = codes[2 * n + i], cm = codes[3 * n + i];
  r[4] = cs | (cr << 16);
  r[5] = cg | ((cm | (uint32_t(type[i] & 15u) << 12)) << 16);
}

// Random-access decode of record i into the caller's layout (ugp_prims / ugp_materials).
__global__ void k_decode(int64_t n, const uint32_t* __restrict__ rec, const float* __restrict__ book,
                         float* __restrict__ mean3, float* __restrict__ quat4, float* __restrict__ scale3,
                         float* __restrict__ mag, float* __restrict__ sggx6, uint8_t* __restrict__ type,
                         float* __restrict__ albedo3, float* __restrict__ rough, float* __restrict__ emit3,
                         float* __restrict__ dis9) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t* r = rec + 6 * i;
  for (int a = 0; a < 3; ++a) mean3[3 * i + a] = __uint_as_float(r[a]);
  mag[i] = __uint_as_float(r[3]);
  const int cs = r[4] & 0xffffu, cr = r[4] >> 16, cg = r[5] & 0xffffu, cm = (r[5] >> 16) & 0xfffu;
  type[i] = uint8_t(r[5] >> 28);
  const float* bs = book + size_t(cs) * kFeat;
  for (int a = 0; a < 3; ++a) scale3[3 * i + a] = expf(bs[a]);
  const float* br = book + size_t(cr) * kFeat + 3;
  const float inv = rsqrtf(fmaxf(br[0] * br[0] + br[1] * br[1] + br[2] * br[2] + br[3] * br[3], 1e-30f));
  for (int a = 0; a < 4; ++a) quat4[4 * i + a] = br[a] * inv;
  const float* bg = book + size_t(cg) * kFeat + 7;
  for (int a = 0; a < 6; ++a) sggx6[6 * i + a] = bg[a];
  const float* bm = book + size_t(cm) * kFeat + 13;
  for (int a = 0; a < 3; ++a) albedo3[3 * i + a] = bm[a];
  rough[i] = bm[3];
  for (int a = 0; a < 3; ++a) emit3[3 * i + a] = bm[4 + a];
  if (dis9)
    for (int a = 0; a < 9; ++a) dis9[9 * i + a] = bm[7 + a];
}

struct CbLayout {
  size_t X, codes, sums, cnt, total;
};
CbLayout cb_layout(int64_t n) {
  CbLayout L;
  size_t off = 0;
  L.X = off;     off = align256(off + size_t(n) * kFeat * 4);
  L.codes = off; off = align256(off + size_t(n) * kGroups * 2);
  L.sums = off;  off = align256(off + size_t(kCodes) * 16 * 8);
  L.cnt = off;   off = align256(off + size_t(kCodes) * 4);
  L.total = off;
  return L;
}

template <int G>
ugp_status fit_group(int64_t n, const float* X, float* book, uint16_t* code, unsigned long long* sums,
                     unsigned int* cnt, int iters, cudaStream_t st) {
  const unsigned gp = unsigned((n + 255) / 256);
  for (int it = 0; it < iters; ++it) {
    k_assign<G><<<gp, 256, 0, st>>>(n, X, book, code);
    UGP_CUDA_CHECK(cudaMemsetAsync(sums, 0, size_t(kCodes) * kDim[G] * 8, st));
    UGP_CUDA_CHECK(cudaMemsetAsync(cnt, 0, size_t(kCodes) * 4, st));
    k_accumulate<G><<<gp, 256, 0, st>>>(n, X, code, sums, cnt);
    k_update<G><<<kCodes / 256, 256, 0, st>>>(sums, cnt, book);
  }
  k_assign<G><<<gp, 256, 0, st>>>(n, X, book, code);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

}  // namespace
}  // namespace ugp

using namespace ugp;

extern "C" size_t ugp_codebook_size(void) { return book_floats() * 4; }

extern "C" size_t ugp_codebook_workspace_size(int64_t n_prims) {
  if (n_prims < 0 || n_prims > (int64_t(1) << 30)) return 0;
  return cb_layout(n_prims).total;
}

extern "C" ugp_status ugp_codebook_encode(const ugp_prims* prims, const ugp_materials* materials, int32_t iters,
                                          void* codebook, void* records, void* workspace, size_t workspace_bytes,
                                          void* stream) {
  clear_error();
  if (!prims || !materials || !codebook || !records)
    return fail(UGP_ERR_INVALID_ARG, "ugp_codebook_encode: NULL argument");
  const int64_t n = prims->n;
  if (n < 1 || n > (int64_t(1) << 30))
    return fail(UGP_ERR_INVALID_ARG, "ugp_codebook_encode: n_prims %lld not in [1, 2^30]", (long long)n);
  if (iters < 0 || iters > 100) return fail(UGP_ERR_INVALID_ARG, "ugp_codebook_encode: iters not in [0, 100]");
  if (!prims->mean3 || !prims->quat4 || !prims->scale3 || !prims->magnitude || !materials->sggx6 ||
      !materials->type || !materials->albedo3 || !materials->roughness || !materials->emission3)
    return fail(UGP_ERR_INVALID_ARG, "ugp_codebook_encode: NULL primitive or material array");
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || (reinterpret_cast<uintptr_t>(codebook) & 15) ||
      (reinterpret_cast<uintptr_t>(records) & 3))
    return fail(UGP_ERR_INVALID_ARG, "ugp_codebook_encode: NULL or misaligned workspace, codebook or records");
  const CbLayout L = cb_layout(n);
  if (workspace_bytes < L.total)
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_codebook_encode: need %zu bytes, got %zu", L.total,
                workspace_bytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  float* X = reinterpret_cast<float*>(ws + L.X);
  uint16_t* codes = reinterpret_cast<uint16_t*>(ws + L.codes);
  unsigned long long* sums = reinterpret_cast<unsigned long long*>(ws + L.sums);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(ws + L.cnt);
  float* book = static_cast<float*>(codebook);
  const unsigned gp = unsigned((n + 255) / 256);
  prof_begin(kStBuild, st);
  k_features<<<gp, 256, 0, st>>>(n, prims->quat4, prims->scale3, materials->sggx6, materials->albedo3,
                                 materials->roughness, materials->emission3, materials->disney9, X);
  k_init_book<<<kCodes / 256, 256, 0, st>>>(n, X, book);
  UGP_CUDA_CHECK(cudaGetLastError());
  ugp_status s;
  if ((s = fit_group<0>(n, X, book, codes, sums, cnt, iters, st)) != UGP_OK) return s;
  if ((s = fit_group<1>(n, X, book, codes + n, sums, cnt, iters, st)) != UGP_OK) return s;
  if ((s = fit_group<2>(n, X, book, codes + 2 * n, sums, cnt, iters, st)) != UGP_OK) return s;
  if ((s = fit_group<3>(n, X, book, codes + 3 * n, sums, cnt, iters, st)) != UGP_OK) return s;
  k_pack<<<gp, 256, 0, st>>>(n, prims->mean3, prims->magnitude, materials->type, codes,
                             static_cast<uint32_t*>(records));
  prof_end(kStBuild, st, 3 + kGroups * (1 + 3 * iters));
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

extern "C" ugp_status ugp_codebook_decode(int64_t n, const void* records, const void* codebook, float* mean3,
                                          float* quat4, float* scale3, float* magnitude, float* sggx6,
                                          uint8_t* type, float* albedo3, float* roughness, float* emission3,
                                          float* disney9, void* stream) {
  clear_error();
  if (n < 0 || n > (int64_t(1) << 30)) return fail(UGP_ERR_INVALID_ARG, "ugp_codebook_decode: n out of range");
  if (n == 0) return UGP_OK;
  if (!records || !codebook || !mean3 || !quat4 || !scale3 || !magnitude || !sggx6 || !type || !albedo3 ||
      !roughness || !emission3)
    return fail(UGP_ERR_INVALID_ARG, "ugp_codebook_decode: NULL array (only disney9 may be NULL)");
  if ((reinterpret_cast<uintptr_t>(records) & 3) || (reinterpret_cast<uintptr_t>(codebook) & 3))
    return fail(UGP_ERR_INVALID_ARG, "ugp_codebook_decode: misaligned records or codebook");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_begin(kStBuild, st);
  k_decode<<<unsigned((n + 255) / 256), 256, 0, st>>>(n, static_cast<const uint32_t*>(records),
                                                      static_cast<const float*>(codebook), mean3, quat4, scale3,
                                                      magnitude, sggx6, type, albedo3, roughness, emission3, disney9);
  prof_end(kStBuild, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}
