// Emitter table for light sampling toward emissive primitives: the emitters in caller order
// with the running sums of their power c mean(L_e) (double), and per emitter the matrix RS =
// W^-1 that maps the whitened ball back to the primitive, its mean, c m and L_e.
#include <cub/cub.cuh>

#include "ugp_emitters.cuh"
#include "ugp_trace.cuh"

namespace ugp {
namespace {

constexpr int kEmBlock = 1024;

// map[id] = leaf slot of every valid record (the inverse of the build's reordering).
__global__ void k_em_inverse(const float4* __restrict__ recs, int64_t n, int* __restrict__ map) {
  for (int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
    const int id = __float_as_int(__ldg(recs + 4 * s + 3).y);
    if (id >= 0 && id < n) map[id] = int(s);
  }
}

// One block walks the caller's primitives in order: weights, compaction and running sums by
// block scans, carried across chunks in double.
__global__ void __launch_bounds__(kEmBlock) k_em_build(const float4* __restrict__ recs, const float4* __restrict__ wlo,
                                                       int64_t n, const uint8_t* __restrict__ type,
                                                       const float* __restrict__ emission3, float mass,
                                                       long long* hdr, double* cdf, float4* rec, int* map) {
  using ScanI = cub::BlockScan<int, kEmBlock>;
  using ScanD = cub::BlockScan<double, kEmBlock>;
  __shared__ union {
    typename ScanI::TempStorage i;
    typename ScanD::TempStorage d;
  } tmp;
  __shared__ double run_total;
  __shared__ int run_count;
  const int tid = threadIdx.x;
  if (tid == 0) {
    run_total = 0.0;
    run_count = 0;
  }
  __syncthreads();
  const double two_pi_15 = 15.749609945722419;  // (2 pi)^{3/2}
  for (int64_t base = 0; base < n; base += kEmBlock) {
    const int64_t i = base + tid;
    double w = 0.0, M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, c = 0.0;
    float4 r0 = make_float4(0, 0, 0, 0), r1 = r0, r2 = r0;
    float3 Le = make_float3(0, 0, 0);
    if (i < n && type[i] == 2) {
      const int s = map[i];
      if (s >= 0) {
        r0 = recs[4 * s];
        r1 = recs[4 * s + 1];
        r2 = recs[4 * s + 2];
        const float4 r3 = recs[4 * s + 3];
        const float4 l0 = wlo[3 * s], l1 = wlo[3 * s + 1], l2 = wlo[3 * s + 2];
        if (r3.z != 0.f) {
          const double W[9] = {double(r0.x) + l0.x, double(r0.y) + l0.y, double(r0.z) + l0.z,
                               double(r1.x) + l1.x, double(r1.y) + l1.y, double(r1.z) + l1.z,
                               double(r2.x) + l2.x, double(r2.y) + l2.y, double(r2.z) + l2.z};
          const double a0 = W[4] * W[8] - W[5] * W[7], a1 = W[5] * W[6] - W[3] * W[8], a2 = W[3] * W[7] - W[4] * W[6];
          const double det = W[0] * a0 + W[1] * a1 + W[2] * a2;
          if (det != 0.0) {
            // adjugate / det: M = W^-1 = R S
            M[0] = a0 / det;
            M[1] = (W[2] * W[7] - W[1] * W[8]) / det;
            M[2] = (W[1] * W[5] - W[2] * W[4]) / det;
            M[3] = a1 / det;
            M[4] = (W[0] * W[8] - W[2] * W[6]) / det;
            M[5] = (W[2] * W[3] - W[0] * W[5]) / det;
            M[6] = a2 / det;
            M[7] = (W[1] * W[6] - W[0] * W[7]) / det;
            M[8] = (W[0] * W[4] - W[1] * W[3]) / det;
            c = double(r3.x) * two_pi_15 / fabs(det);  // g0 = c / ((2 pi)^{3/2} |Sigma|^{1/2}), |det W| = |Sigma|^{-1/2}
            Le = make_float3(emission3[3 * i], emission3[3 * i + 1], emission3[3 * i + 2]);
            w = c * (double(Le.x) + double(Le.y) + double(Le.z)) / 3.0;
            if (!(w > 0.0)) w = 0.0;
          }
        }
      }
    }
    const int flag = w > 0.0 ? 1 : 0;
    int rank, chunk_count;
    ScanI(tmp.i).ExclusiveSum(flag, rank, chunk_count);
    __syncthreads();
    double incl, chunk_total;
    ScanD(tmp.d).InclusiveSum(w, incl, chunk_total);
    __syncthreads();
    if (i < n) {
      int e = -1;
      if (flag) {
        e = run_count + rank;
        cdf[e] = run_total + incl;
        rec[4 * e] = make_float4(float(M[0]), float(M[1]), float(M[2]), r0.w);
        rec[4 * e + 1] = make_float4(float(M[3]), float(M[4]), float(M[5]), r1.w);
        rec[4 * e + 2] = make_float4(float(M[6]), float(M[7]), float(M[8]), r2.w);
        rec[4 * e + 3] = make_float4(float(c * mass), Le.x, Le.y, Le.z);
      }
      map[i] = e;  // replaces the slot this thread read above
    }
    __syncthreads();
    if (tid == 0) {
      run_count += chunk_count;
      run_total += chunk_total;
    }
    __syncthreads();
  }
  if (tid == 0) {
    hdr[0] = run_count;
    hdr[1] = __double_as_longlong(run_total);
    hdr[2] = n;
  }
}

double chi3_cdf_host(double r) {
  return erf(r / sqrt(2.0)) - sqrt(2.0 / 3.14159265358979323846) * r * exp(-0.5 * r * r);
}

}  // namespace

EmitterDev emitter_dev(const void* table, const ugp_bvh* bvh) {
  EmitterDev E{};
  if (!table) return E;
  const char* t = static_cast<const char*>(table);
  const EmitterLayout L = emitter_layout(bvh->n_prims);
  E.hdr = reinterpret_cast<const long long*>(t);
  E.cdf = reinterpret_cast<const double*>(t + L.cdf);
  E.rec = reinterpret_cast<const float4*>(t + L.rec);
  E.map = reinterpret_cast<const int*>(t + L.map);
  E.n_prims = bvh->n_prims;
  E.k = bvh->k;
  E.mass = float(chi3_cdf_host(double(bvh->k)));
  return E;
}

}  // namespace ugp

using namespace ugp;

extern "C" size_t ugp_emitter_table_size(int64_t n_prims) {
  if (n_prims < 0 || n_prims > (int64_t(1) << 31) - 1) return 0;
  return emitter_layout(n_prims).total;
}

extern "C" ugp_status ugp_build_emitter_table(const ugp_bvh* bvh, const ugp_materials* materials, void* table,
                                              size_t table_bytes, void* stream) {
  clear_error();
  if (!valid_bvh(bvh)) return fail(UGP_ERR_NOT_BUILT, "ugp_build_emitter_table: invalid BVH handle");
  if (!materials || !table) return fail(UGP_ERR_INVALID_ARG, "ugp_build_emitter_table: NULL argument");
  if (bvh->n_prims > 0 && (!materials->type || !materials->emission3))
    return fail(UGP_ERR_INVALID_ARG, "ugp_build_emitter_table: NULL type or emission array");
  if (reinterpret_cast<uintptr_t>(table) & 255)
    return fail(UGP_ERR_INVALID_ARG, "ugp_build_emitter_table: table must be 256-byte aligned");
  const int64_t n = bvh->n_prims;
  if (n > (int64_t(1) << 31) - 1) return fail(UGP_ERR_INVALID_ARG, "ugp_build_emitter_table: too many primitives");
  const EmitterLayout L = emitter_layout(n);
  if (table_bytes < L.total)
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_build_emitter_table: need %zu bytes, got %zu", L.total, table_bytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* t = static_cast<char*>(table);
  int* map = reinterpret_cast<int*>(t + L.map);
  UGP_CUDA_CHECK(cudaMemsetAsync(t, 0, 256, st));
  if (n > 0) {
    UGP_CUDA_CHECK(cudaMemsetAsync(map, 0xff, size_t(n) * 4, st));  // -1: no valid record
    prof_begin(kStBuild, st);
    const int grid = int((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_em_inverse<<<grid, 256, 0, st>>>(bvh->prims, n, map);
    k_em_build<<<1, kEmBlock, 0, st>>>(bvh->prims, bvh->wlo, n, materials->type, materials->emission3,
                                       float(chi3_cdf_host(double(bvh->k))), reinterpret_cast<long long*>(t),
                                       reinterpret_cast<double*>(t + L.cdf), reinterpret_cast<float4*>(t + L.rec),
                                       map);
    prof_end(kStBuild, st, 2);
    UGP_CUDA_CHECK(cudaGetLastError());
  }
  return UGP_OK;
}
