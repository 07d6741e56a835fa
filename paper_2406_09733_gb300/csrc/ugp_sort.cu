// Stable least-significant-digit radix sort of (key, value) pairs, 8 bits per pass, used by the
// BVH build to order the primitives by Morton code.
//
// A pass over n pairs, in tiles of kTile keys (one block of 8 warps each):
//   1. k_rs_hist   each tile's 256-bin histogram of the pass's digit, stored digit-major
//                  (hist[d * tiles + b]), so that the offsets below are prefix sums along rows;
//   2. k_rs_rows   one block per digit: the exclusive prefix of its row (the keys of that digit
//                  in earlier tiles) and the row's total;
//   3. k_rs_scatter a tile's keys go to (keys of smaller digits) + (keys of this digit in earlier
//                  tiles) + (keys of this digit earlier in the tile). Within the tile each warp
//                  owns 1024 consecutive keys, counted per digit first; a warp then walks its
//                  keys 32 at a time in order, and lanes holding the same digit rank themselves
//                  by __match_any_sync, so equal keys keep their order (stable).
// Passes alternate between the two buffers; the result is in buffer (passes & 1).
#include "ugp_internal.cuh"

namespace ugp {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsPerWarp = 1024;
constexpr int kTile = kRsWarps * kRsPerWarp;  // 8192 keys per tile
constexpr unsigned kFull = 0xffffffffu;

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                         int tiles, uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kTile;
  for (int i = threadIdx.x; i < kTile; i += kRsThreads) {
    const int64_t idx = base + i;
    if (idx < n) atomicAdd(&cnt[(__ldg(keys + idx) >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[size_t(threadIdx.x) * tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive prefix of a 256-thread block's values; returns this thread's, and the total in *total.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t* warp_sums, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sums[w] = incl;
  __syncthreads();
  if (w == 0) {
    const uint32_t s = lane < kRsWarps ? warp_sums[lane] : 0u;
    uint32_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, si, o);
      if (lane >= o) si += y;
    }
    if (lane < kRsWarps) warp_sums[lane] = si - s;
    if (lane == kRsWarps - 1) warp_sums[kRsWarps] = si;
  }
  __syncthreads();
  const uint32_t r = warp_sums[w] + incl - v;
  *total = warp_sums[kRsWarps];
  __syncthreads();  // warp_sums may be reused by the caller's next call
  return r;
}

// One block per digit: exclusive prefix of its row of tile counts, in place, and the row total.
__global__ void __launch_bounds__(kRsThreads) k_rs_rows(uint32_t* __restrict__ hist, int tiles,
                                                         uint32_t* __restrict__ totals) {
  __shared__ uint32_t ws[kRsWarps + 1];
  uint32_t* row = hist + size_t(blockIdx.x) * tiles;
  uint32_t carry = 0u;
  for (int b0 = 0; b0 < tiles; b0 += kRsThreads) {
    const int b = b0 + int(threadIdx.x);
    const uint32_t v = b < tiles ? row[b] : 0u;
    uint32_t sum;
    const uint32_t ex = block_exclusive(v, ws, &sum);
    if (b < tiles) row[b] = carry + ex;
    carry += sum;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                            const int32_t* __restrict__ vin, int64_t n, int shift,
                                                            int tiles, const uint32_t* __restrict__ hist,
                                                            const uint32_t* __restrict__ totals,
                                                            uint32_t* __restrict__ kout, int32_t* __restrict__ vout) {
  __shared__ uint32_t wbase[kRsWarps][256];
  __shared__ uint32_t ws[kRsWarps + 1];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // this tile's first position for digit tid: keys of smaller digits, then of digit tid in
  // earlier tiles
  uint32_t all;
  const uint32_t dpre = block_exclusive(totals[tid], ws, &all);
  const uint32_t gofs = dpre + hist[size_t(tid) * tiles + blockIdx.x];
#pragma unroll
  for (int k = 0; k < kRsWarps; ++k) wbase[k][tid] = 0u;
  __syncthreads();
  const int64_t wstart = int64_t(blockIdx.x) * kTile + int64_t(w) * kRsPerWarp;
  for (int r = 0; r < kRsPerWarp; r += 32) {
    const int64_t idx = wstart + r + lane;
    if (idx < n) atomicAdd(&wbase[w][(__ldg(kin + idx) >> shift) & 255u], 1u);
  }
  __syncthreads();
  {
    uint32_t run = gofs;
#pragma unroll
    for (int k = 0; k < kRsWarps; ++k) {
      const uint32_t c = wbase[k][tid];
      wbase[k][tid] = run;
      run += c;
    }
  }
  __syncthreads();
  const unsigned below = (1u << lane) - 1u;
  for (int r = 0; r < kRsPerWarp; r += 32) {
    const int64_t idx = wstart + r + lane;
    const bool valid = idx < n;
    const uint32_t key = valid ? __ldg(kin + idx) : 0u;
    const int d = valid ? int((key >> shift) & 255u) : 256 + lane;  // padding lanes match nobody
    const unsigned peers = __match_any_sync(kFull, d);
    if (valid) {
      const uint32_t pos = wbase[w][d] + __popc(peers & below);
      kout[pos] = key;
      vout[pos] = __ldg(vin + idx);
    }
    __syncwarp();
    if (valid && (peers & below) == 0u) wbase[w][d] += __popc(peers);  // the digit's first lane
    __syncwarp();
  }
}

}  // namespace

size_t radix_sort_workspace(int64_t n) {
  const int64_t tiles = (n + kTile - 1) / kTile;
  return align256(size_t(256) * size_t(tiles > 0 ? tiles : 1) * 4) + 256 * 4;
}

int radix_sort_passes(int bits) { return (bits + 7) / 8; }

ugp_status radix_sort_pairs(uint32_t* k0, uint32_t* k1, int32_t* v0, int32_t* v1, int64_t n, int bits, void* ws,
                            cudaStream_t st) {
  if (n <= 1) return UGP_OK;
  const int tiles = int((n + kTile - 1) / kTile);
  uint32_t* hist = static_cast<uint32_t*>(ws);
  uint32_t* totals = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + align256(size_t(256) * tiles * 4));
  uint32_t* kb[2] = {k0, k1};
  int32_t* vb[2] = {v0, v1};
  for (int p = 0; p < radix_sort_passes(bits); ++p) {
    const int shift = 8 * p;
    k_rs_hist<<<tiles, kRsThreads, 0, st>>>(kb[p & 1], n, shift, tiles, hist);
    k_rs_rows<<<256, kRsThreads, 0, st>>>(hist, tiles, totals);
    k_rs_scatter<<<tiles, kRsThreads, 0, st>>>(kb[p & 1], vb[p & 1], n, shift, tiles, hist, totals, kb[(p + 1) & 1],
                                               vb[(p + 1) & 1]);
  }
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

}  // namespace ugp
