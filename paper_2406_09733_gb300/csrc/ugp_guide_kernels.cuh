// Tensor-core kernels of the learned guide (tcgen05.mma with TMEM accumulators, operands in
// shared memory, weights brought in by one bulk TMA copy per block).
//
// A block of 128 threads owns tiles of 128 rows (vertices); thread t owns row t, which is
// tensor-memory lane t of the M = 128 accumulator, so every epilogue is a per-thread
// tcgen05.ld of its own row. Per layer one thread issues four K = 16 MMAs
// (D[128 x 64] = X[128 x 64] W^T), commits them to an mbarrier, and all threads wait with a
// time limit (a wait that gives up sets the workspace's error word and the block leaves
// through its single exit, which frees its tensor memory).
//
// Training (k_guide_grad) runs the forward pass of a tile, the loss gradient of the head in
// the epilogue, and the backward pass layer by layer:
//   dW_l += dZ_l^T X_l   M = 128 (64 output rows + 64 unused), N = 80 (64 inputs, a ones
//                        column that yields the bias gradient, 15 unused), K = 128 rows;
//                        both operands MN-major views of the row-major tiles dZ_l and X_l
//   dX_l  = dZ_l W_l     M = 128, N = 64, K = 64; W_l as an MN-major view of its tile
// so no operand is ever transposed in shared memory. The five dW accumulators stay in tensor
// memory across all tiles of the block (5 x 80 columns) and are written once per block as a
// partial sum; a second kernel adds the partials in a fixed order, so the gradient is
// deterministic.
#pragma once
#include "ugp_guide.cuh"
#include "ugp_internal.cuh"
#include "ugp_umma.cuh"

namespace ugp {

constexpr int kGThreads = 128;
constexpr int kGMaxGradBlocks = 256;
constexpr uint64_t kGWaitNs = 2000000000ull;  // 2 s per tensor-core wait

struct GuideDev {
  GuideCfgDev cfg;
  const uint8_t* img;  // packed weights (kImgBytes, 256-byte aligned)
  int* err;            // error word (UGP_ERR_TIMEOUT when a wait gave up)
};

// Workspace of the guide calls: 256-byte header (error word), packed weights, gradient
// partials of up to kGMaxGradBlocks blocks and their loss partials.
struct GuideWs {
  int* err;
  uint8_t* img;
  float* partial;
  float* loss_partial;
};
inline size_t guide_ws_bytes() {
  return 256 + align256(kImgBytes) + align256(size_t(kGMaxGradBlocks) * UGP_GUIDE_NPARAMS * 4) +
         align256(kGMaxGradBlocks * 4);
}
inline GuideWs guide_ws_at(void* base) {
  char* p = static_cast<char*>(base);
  GuideWs w;
  w.err = reinterpret_cast<int*>(p);
  p += 256;
  w.img = reinterpret_cast<uint8_t*>(p);
  p += align256(kImgBytes);
  w.partial = reinterpret_cast<float*>(p);
  p += align256(size_t(kGMaxGradBlocks) * UGP_GUIDE_NPARAMS * 4);
  w.loss_partial = reinterpret_cast<float*>(p);
  return w;
}

GuideCfgDev guide_cfg_dev(const ugp_guide* g);
// Packs the FP32 master weights into the BF16 operand image (asynchronous on `st`).
ugp_status launch_guide_pack(const float* params, uint8_t* img, cudaStream_t st);
int guide_sm_count();

namespace gk {

using namespace umma;

constexpr uint32_t kIdescFwd = idesc_bf16_f32(128, 64);        // X W^T: both K-major
constexpr uint32_t kIdescDX = idesc_bf16_f32(128, 64, 0, 1);    // dZ W: B MN-major
constexpr uint32_t kIdescDW = idesc_bf16_f32(128, 80, 1, 1);    // dZ^T X: both MN-major
constexpr uint32_t kXTile = 128 * kGWidth * 2;  // 16384: one 128 x 64 BF16 activation tile

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Writes row r (64 values) of a 128-row tile as BF16.
__device__ __forceinline__ void store_row(uint8_t* tile, int r, const float (&v)[kGWidth]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint4 q;
    q.x = pack_bf16x2(v[8 * c], v[8 * c + 1]);
    q.y = pack_bf16x2(v[8 * c + 2], v[8 * c + 3]);
    q.z = pack_bf16x2(v[8 * c + 4], v[8 * c + 5]);
    q.w = pack_bf16x2(v[8 * c + 6], v[8 * c + 7]);
    *reinterpret_cast<uint4*>(tile + tile_off(uint32_t(r), uint32_t(8 * c), 128u)) = q;
  }
}

// Reads row r of a 128-row BF16 tile as raw 16-bit values.
__device__ __forceinline__ void load_row_bits(const uint8_t* tile, int r, uint16_t (&h)[kGWidth]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint4 q = *reinterpret_cast<const uint4*>(tile + tile_off(uint32_t(r), uint32_t(8 * c), 128u));
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[8 * c + 2 * j] = uint16_t(w[j] & 0xffffu);
      h[8 * c + 2 * j + 1] = uint16_t(w[j] >> 16);
    }
  }
}

// Loads `cols` (multiple of 16) accumulator columns of the calling thread's lane.
template <int kCols>
__device__ __forceinline__ void tmem_row(uint32_t taddr, float (&v)[kCols]) {
  uint32_t r[kCols / 16][16];
#pragma unroll
  for (int c = 0; c < kCols / 16; ++c) tmem_ld16(taddr + uint32_t(16 * c), r[c]);
  tmem_wait_ld();
#pragma unroll
  for (int c = 0; c < kCols / 16; ++c) {
    reg_fence(r[c]);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[16 * c + j] = __uint_as_float(r[c][j]);
  }
}

// An operand view of an R-row tile (layout in ugp_umma.cuh): start address, the descriptor's
// leading- and stride-dimension byte offsets, and the distance between K = 16 slices.
struct Operand {
  uint32_t addr, lbo, sbo, kstep;
};
// Rows are M or N, columns are K (X W^T reads X and W this way).
__device__ __forceinline__ Operand kmajor(const uint8_t* tile, uint32_t R) {
  return {smem_u32(tile), R * 16u, 128u, R * 32u};
}
// Rows are K, columns are M or N (dZ^T X reads dZ and X this way, dZ W reads W this way).
__device__ __forceinline__ Operand mnmajor(const uint8_t* tile, uint32_t R) {
  return {smem_u32(tile), 128u, R * 16u, 256u};
}

// Issues D = A B^T (+ D) over `ksteps` K = 16 slices. Called by one thread.
__device__ __forceinline__ void issue(uint32_t d, const Operand& a, const Operand& b, int ksteps, uint32_t idesc,
                                      bool accumulate) {
  for (int ks = 0; ks < ksteps; ++ks)
    mma_bf16(d, desc_smem(a.addr + uint32_t(ks) * a.kstep, a.lbo, a.sbo),
             desc_smem(b.addr + uint32_t(ks) * b.kstep, b.lbo, b.sbo), idesc, (accumulate || ks > 0) ? 1u : 0u);
}

__device__ __forceinline__ int64_t row_count(int64_t n_host, const int* n_dev) {
  return n_dev ? int64_t(*reinterpret_cast<const volatile int*>(n_dev)) : n_host;
}

// ------------------------------------------------------------------ forward
// A block (one per SM: 512 threads at up to 128 registers) holds kFwdGroups groups of 128
// threads (warpgroups) that share the weights. Each group runs its own 128-row tiles with its
// own activation tile, tensor-memory columns and mbarrier, synchronised by a named barrier of its
// own, so one group's epilogue (the per-thread bias, ReLU and BF16 packing, the encoding of the
// next tile, the mixture) overlaps the others' MMAs. The group's activation tile doubles as the
// staging buffer of its output rows, which the group then writes out row by row (coalesced).
constexpr int kFwdGroups = 4;
constexpr int kFwdStage = kGOut + 4;  // floats between staged rows: 16-byte stores without bank conflicts
constexpr uint32_t kFwdBuf = 128 * kFwdStage * 4;               // 22528: X tile or 128 output rows
constexpr uint32_t kFwdX = kImgBytes;                           // after W and biases
constexpr uint32_t kFwdValid = kFwdX + kFwdGroups * kFwdBuf;    // per group: 128 row flags
constexpr uint32_t kFwdBar = kFwdValid + kFwdGroups * 128 * 4;  // weights, then one per group
constexpr uint32_t kFwdTmemSlot = kFwdBar + 8 * (kFwdGroups + 1);
constexpr uint32_t kFwdSmem = kFwdTmemSlot + 16;
constexpr uint32_t kFwdTmemCols = 256;  // kFwdGroups x 64 columns
static_assert(kFwdBuf >= kXTile && kFwdTmemCols >= 64 * kFwdGroups, "forward buffers");
static_assert(kFwdSmem <= 227 * 1024, "forward block exceeds shared memory");

// Barrier of the 128 threads of group `grp` (ids 1..kFwdGroups; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, 128;" ::"r"(grp + 1) : "memory");
}
// The same barrier, returning whether p held on any of the group's threads.
__device__ __forceinline__ bool group_any(int grp, bool p) {
  uint32_t r;
  asm volatile(
      "{\n"
      " .reg .pred a, b;\n"
      " setp.ne.u32 a, %1, 0;\n"
      " bar.red.or.pred b, %2, 128, a;\n"
      " selp.u32 %0, 1, 0, b;\n"
      "}\n"
      : "=r"(r)
      : "r"(uint32_t(p)), "r"(grp + 1)
      : "memory");
  return r != 0;
}

// Packs two values as BF16 after a ReLU (round to nearest even; the ReLU commutes with it).
__device__ __forceinline__ uint32_t pack_bf16x2_relu(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Src: __device__ bool vertex(int64_t row, float3& x, float3& wo) const  (false: row unused)
// Dst: __device__ float* row_out(int64_t row) const        where the row's 40 output values go
//      __device__ void values(int64_t row, const float (&Y)[40], float (&out)[40]) const
//                                                             the output values from the head Y
template <class Src, class Dst>
__global__ void __launch_bounds__(kGThreads * kFwdGroups, 1) k_guide_fwd(GuideDev g, Src src, Dst dst, int64_t n_host,
                                                                      const int* n_dev) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int tid = int(threadIdx.x), warp = tid >> 5, grp = tid >> 7, t = tid & 127, lane = tid & 31;
  const int64_t n = row_count(n_host, n_dev);
  const int64_t ntiles = (n + kGThreads - 1) / kGThreads;
  if (int64_t(blockIdx.x) * kFwdGroups >= ntiles) return;  // whole block, before any resource is taken
  uint8_t* X = sm + kFwdX + grp * kFwdBuf;
  float* stage = reinterpret_cast<float*>(X);
  int* vflag = reinterpret_cast<int*>(sm + kFwdValid) + grp * 128;
  const uint32_t wbar = smem_u32(sm + kFwdBar), gbar = wbar + 8u * uint32_t(grp + 1);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kFwdTmemSlot);
  if (tid == 0) {
    for (int b = 0; b <= kFwdGroups; ++b) mbar_init(wbar + 8u * uint32_t(b), 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tslot), kFwdTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t tmem = tbase + 64u * uint32_t(grp);
  const uint32_t lane_addr = tmem + (uint32_t((warp & 3) * 32) << 16);
  if (tid == 0) {
    mbar_expect_tx(wbar, kImgBytes);
    bulk_g2s(smem_u32(sm), g.img, kImgBytes, wbar);
  }
  bool failed = __syncthreads_or(!mbar_wait(wbar, 0u, kGWaitNs));
  uint32_t phase = 0;
  const float* bias = reinterpret_cast<const float*>(sm + kImgBias);
  for (int64_t tile = int64_t(blockIdx.x) * kFwdGroups + grp; tile < ntiles && !failed;
       tile += int64_t(gridDim.x) * kFwdGroups) {
    const int64_t row = tile * kGThreads + t;
    bool valid = false;
    {
      float f[kGWidth];
      float3 x = f3(0.f, 0.f, 0.f), wo = f3(0.f, 0.f, 1.f);
      valid = row < n && src.vertex(row, x, wo);
      if (valid) {
        guide_encode(g.cfg, x, wo, f);
      } else {
#pragma unroll
        for (int i = 0; i < kGWidth; ++i) f[i] = 0.f;
      }
      store_row(X, t, f);
    }
    float out[kGOut];
    for (int l = 0; l <= kGLayers; ++l) {
      fence_async_smem();
      tc_fence_before();
      group_sync(grp);
      if (t == 0) {
        tc_fence_after();
        issue(tmem, kmajor(X, 128), kmajor(sm + kImgW + l * kImgTile, 64), 4, kIdescFwd, false);
        mma_commit(gbar);
      }
      const bool ok = mbar_wait(gbar, phase, kGWaitNs);
      phase ^= 1u;
      if (group_any(grp, !ok)) {
        failed = true;
        break;
      }
      tc_fence_after();
      if (l < kGLayers) {
        float v[kGWidth];
        tmem_row<kGWidth>(lane_addr, v);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float* b = bias + l * kGWidth + 8 * c;
          uint4 q;
          q.x = pack_bf16x2_relu(v[8 * c] + b[0], v[8 * c + 1] + b[1]);
          q.y = pack_bf16x2_relu(v[8 * c + 2] + b[2], v[8 * c + 3] + b[3]);
          q.z = pack_bf16x2_relu(v[8 * c + 4] + b[4], v[8 * c + 5] + b[5]);
          q.w = pack_bf16x2_relu(v[8 * c + 6] + b[6], v[8 * c + 7] + b[7]);
          *reinterpret_cast<uint4*>(X + tile_off(uint32_t(t), uint32_t(8 * c), 128u)) = q;
        }
      } else {
        float v[48];
        tmem_row<48>(lane_addr, v);
        float Y[kGOut];
#pragma unroll
        for (int i = 0; i < kGOut; ++i) Y[i] = v[i] + bias[kGLayers * kGWidth + i];
        if (valid) dst.values(row, Y, out);
      }
    }
    if (failed) break;
    // the last MMA has read X: stage the rows there and write them out, 160 bytes per row
    vflag[t] = valid ? 1 : 0;
    if (valid) {
      float4* srow = reinterpret_cast<float4*>(stage + t * kFwdStage);
#pragma unroll
      for (int j = 0; j < kGOut / 4; ++j) srow[j] = make_float4(out[4 * j], out[4 * j + 1], out[4 * j + 2], out[4 * j + 3]);
    }
    group_sync(grp);
    // warp w of the group writes rows 32 w .. 32 w + 31, three rows (30 lanes) at a time
    const int wbase = (warp & 3) * 32;
    for (int i0 = 0; i0 < 32; i0 += 3) {
      const int i = wbase + i0 + lane / 10, k = lane % 10;
      if (lane < 30 && i0 + lane / 10 < 32 && vflag[i]) {
        float* dp = dst.row_out(tile * kGThreads + i);
        const float4 val = reinterpret_cast<const float4*>(stage + i * kFwdStage)[k];
        if ((reinterpret_cast<uintptr_t>(dp) & 15) == 0) {
          reinterpret_cast<float4*>(dp)[k] = val;
        } else {
          dp[4 * k] = val.x; dp[4 * k + 1] = val.y; dp[4 * k + 2] = val.z; dp[4 * k + 3] = val.w;
        }
      }
    }
    group_sync(grp);  // the staged rows are read before the next tile's encoding overwrites them
  }
  if (failed && t == 0 && g.err) atomicExch(g.err, int(UGP_ERR_TIMEOUT));
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, kFwdTmemCols);
  }
}

// ------------------------------------------------------------------ training
// X_l tiles carry 80 columns: 64 activations, a ones column (64) and 15 zeros, so the dW MMA's
// N = 80 view of X_l yields the bias gradient in column 64.
constexpr uint32_t kGrXCols = 80;
constexpr uint32_t kGrXTile = 128 * kGrXCols * 2;       // 20480
constexpr uint32_t kGrDZ = kImgBytes;                   // 42240: dZ, 128 rows x 64 outputs
constexpr uint32_t kGrX = kGrDZ + kXTile;               // 58624: X_0 .. X_4
constexpr uint32_t kGrBar = kGrX + 5 * kGrXTile;        // 161024
constexpr uint32_t kGrTmemSlot = kGrBar + 8;
constexpr uint32_t kGrRed = kGrBar + 16;                // 4 floats of loss reduction
constexpr uint32_t kGrSmem = kGrBar + 128;              // 161152
static_assert(kGrSmem <= 227 * 1024, "guide training block exceeds shared memory");
// The dW MMA's M = 128 view of dZ reads 16 column chunks, the upper 8 (unused accumulator lanes)
// up to 16 KB past the dZ tile; that range is X_0, inside the block's shared memory.
static_assert(kGrX == kGrDZ + kXTile && 5 * kGrXTile >= kXTile, "dZ must be followed by readable shared memory");

constexpr uint32_t kTmScratch = 0;   // 64 columns: layer output / dX
constexpr uint32_t kTmDW = 64;       // 5 x 80 columns: dW_l and db_l
constexpr uint32_t kTmCols = 512;

// Src: __device__ bool sample(int64_t row, float3& x, float3& wo, float3& wi, float& w) const
template <class Src>
__global__ void __launch_bounds__(kGThreads, 1) k_guide_grad(GuideDev g, Src src, int64_t n_host, const int* n_dev,
                                                             float* __restrict__ partial,
                                                             float* __restrict__ loss_partial) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int tid = int(threadIdx.x), warp = tid >> 5;
  const int64_t n = row_count(n_host, n_dev);
  const int64_t ntiles = (n + kGThreads - 1) / kGThreads;
  float* my_partial = partial + size_t(blockIdx.x) * UGP_GUIDE_NPARAMS;
  if (int64_t(blockIdx.x) >= ntiles) {
    for (int p = tid; p < UGP_GUIDE_NPARAMS; p += kGThreads) my_partial[p] = 0.f;
    if (tid == 0) loss_partial[blockIdx.x] = 0.f;
    return;
  }
  const float inv_n = 1.f / float(n);
  uint8_t* X = sm + kGrX;
  uint8_t* DZ = sm + kGrDZ;
  const uint32_t bar = smem_u32(sm + kGrBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kGrTmemSlot);
  float* red = reinterpret_cast<float*>(sm + kGrRed);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tslot), kTmCols);
    tmem_relinquish();
  }
  // Columns 64..79 of every X_l: a ones column (bias gradient) and zeros; written once.
  {
    const uint4 ones = make_uint4(pack_bf16x2(1.f, 0.f), 0u, 0u, 0u), zeros = make_uint4(0u, 0u, 0u, 0u);
    for (int l = 0; l <= kGLayers; ++l) {
      uint8_t* t = X + l * kGrXTile;
      *reinterpret_cast<uint4*>(t + tile_off(uint32_t(tid), 64u, 128u)) = ones;
      *reinterpret_cast<uint4*>(t + tile_off(uint32_t(tid), 72u, 128u)) = zeros;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t lane_addr = tmem + (uint32_t(warp * 32) << 16);
  uint32_t phase = 0;
  if (tid == 0) {
    mbar_expect_tx(bar, kImgBytes);
    bulk_g2s(smem_u32(sm), g.img, kImgBytes, bar);
  }
  bool failed = __syncthreads_or(!mbar_wait(bar, phase, kGWaitNs));
  phase ^= 1u;
  const float* bias = reinterpret_cast<const float*>(sm + kImgBias);
  float loss_acc = 0.f;
  bool first = true;
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t row = tile * kGThreads + tid;
    float3 x = f3(0.f, 0.f, 0.f), wo = f3(0.f, 0.f, 1.f), wi = f3(0.f, 0.f, 1.f);
    float w = 0.f;
    const bool valid = row < n && src.sample(row, x, wo, wi, w);
    {
      float f[kGWidth];
      if (valid) {
        guide_encode(g.cfg, x, wo, f);
      } else {
#pragma unroll
        for (int i = 0; i < kGWidth; ++i) f[i] = 0.f;
      }
      store_row(X, tid, f);
    }
    // forward
    for (int l = 0; l <= kGLayers && !failed; ++l) {
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        issue(tmem + kTmScratch, kmajor(X + l * kGrXTile, 128), kmajor(sm + kImgW + l * kImgTile, 64), 4, kIdescFwd,
              false);
        mma_commit(bar);
      }
      const bool ok = mbar_wait(bar, phase, kGWaitNs);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after();
      if (l < kGLayers) {
        float v[kGWidth];
        tmem_row<kGWidth>(lane_addr + kTmScratch, v);
#pragma unroll
        for (int i = 0; i < kGWidth; ++i) v[i] = fmaxf(v[i] + bias[l * kGWidth + i], 0.f);
        store_row(X + (l + 1) * kGrXTile, tid, v);
      } else {
        float v[48];
        tmem_row<48>(lane_addr + kTmScratch, v);
        float Y[kGOut], dY[kGOut];
#pragma unroll
        for (int i = 0; i < kGOut; ++i) Y[i] = v[i] + bias[kGLayers * kGWidth + i];
        if (valid && w != 0.f) {
          loss_acc += mixture_loss_grad(g.cfg, Y, wi, w * inv_n, dY);
        } else {
#pragma unroll
          for (int i = 0; i < kGOut; ++i) dY[i] = 0.f;
        }
        float d64[kGWidth];
#pragma unroll
        for (int i = 0; i < kGWidth; ++i) d64[i] = i < kGOut ? dY[i] : 0.f;
        store_row(DZ, tid, d64);
      }
    }
    // backward, head first
    for (int l = kGLayers; l >= 0 && !failed; --l) {
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        issue(tmem + kTmDW + 80u * uint32_t(l), mnmajor(DZ, 128), mnmajor(X + l * kGrXTile, 128), 8, kIdescDW,
              !first);
        if (l > 0)
          issue(tmem + kTmScratch, kmajor(DZ, 128), mnmajor(sm + kImgW + l * kImgTile, 64), 4, kIdescDX, false);
        mma_commit(bar);
      }
      const bool ok = mbar_wait(bar, phase, kGWaitNs);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      if (l > 0) {
        tc_fence_after();
        float v[kGWidth];
        tmem_row<kGWidth>(lane_addr + kTmScratch, v);
        uint16_t h[kGWidth];
        load_row_bits(X + l * kGrXTile, tid, h);  // X_l = relu(Z_{l-1}) rounded: > 0 iff Z_{l-1} > 0
#pragma unroll
        for (int i = 0; i < kGWidth; ++i) v[i] = (h[i] != 0 && !(h[i] & 0x8000u)) ? v[i] : 0.f;
        store_row(DZ, tid, v);
      }
    }
    first = false;
  }
  // Block partials: lanes 0..63 of the dW accumulators (warps 0 and 1) hold the output rows.
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (!failed && warp < 2) {
    const int o = tid;
#pragma unroll 1
    for (int l = 0; l <= kGLayers; ++l) {
      float v[80];
      tmem_row<80>(lane_addr + kTmDW + 80u * uint32_t(l), v);
      if (o < guide_out_dim(l)) {
        float* pw = my_partial + guide_w_off(l) + o * kGWidth;
#pragma unroll
        for (int i = 0; i < kGWidth; ++i) pw[i] = first ? 0.f : v[i];
        my_partial[guide_b_off(l) + o] = first ? 0.f : v[64];
      }
    }
  }
  // loss partial
  {
    float s = loss_acc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((tid & 31) == 0) red[warp] = s;
    __syncthreads();
    if (tid == 0) loss_partial[blockIdx.x] = failed ? 0.f : red[0] + red[1] + red[2] + red[3];
  }
  if (failed && tid == 0 && g.err) atomicExch(g.err, int(UGP_ERR_TIMEOUT));
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmCols);
  }
}

}  // namespace gk

// Launches the forward kernel over n rows (n_dev: device row count, overrides n_host) on a
// persistent grid. Requires the packed weights at g.img.
template <class Src, class Dst>
ugp_status launch_guide_forward(const GuideDev& g, const Src& src, const Dst& dst, int64_t n_host, const int* n_dev,
                                int64_t max_rows, cudaStream_t st) {
  auto kern = gk::k_guide_fwd<Src, Dst>;
  static bool attr_set = false;
  if (!attr_set) {
    UGP_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(gk::kFwdSmem)));
    attr_set = true;
  }
  const int64_t tiles = (max_rows + kGThreads - 1) / kGThreads;
  const int64_t need = (tiles + gk::kFwdGroups - 1) / gk::kFwdGroups;
  const int64_t cap = int64_t(guide_sm_count());  // one block of four groups per SM (registers)
  const int grid = int(need < cap ? (need > 0 ? need : 1) : cap);
  kern<<<grid, kGThreads * gk::kFwdGroups, gk::kFwdSmem, st>>>(g, src, dst, n_host, n_dev);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

// Launches the gradient kernel (one block per SM at most) and returns the grid used.
template <class Src>
ugp_status launch_guide_grad(const GuideDev& g, const Src& src, int64_t n_host, const int* n_dev, int64_t max_rows,
                             const GuideWs& ws, int* grid_out, cudaStream_t st) {
  auto kern = gk::k_guide_grad<Src>;
  static bool attr_set = false;
  if (!attr_set) {
    UGP_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(gk::kGrSmem)));
    attr_set = true;
  }
  const int64_t tiles = (max_rows + kGThreads - 1) / kGThreads;
  // at most kGMaxGradBlocks - 1 blocks: the last partial slot stays free as scratch
  int64_t cap = guide_sm_count();
  if (cap > kGMaxGradBlocks - 1) cap = kGMaxGradBlocks - 1;
  const int grid = int(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
  kern<<<grid, kGThreads, gk::kGrSmem, st>>>(g, src, n_host, n_dev, ws.partial, ws.loss_partial);
  UGP_CUDA_CHECK(cudaGetLastError());
  *grid_out = grid;
  return UGP_OK;
}

// Sums `grid` block partials into grad (UGP_GUIDE_NPARAMS) and loss (1 float, may be NULL).
ugp_status launch_guide_reduce(const GuideWs& ws, int grid, float* grad, float* loss, cudaStream_t st);

}  // namespace ugp
