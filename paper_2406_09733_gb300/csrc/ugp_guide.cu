// C entry points of the learned guide: weight packing, the tensor-core forward and gradient
// kernels over caller arrays, the deterministic partial-sum reduction, Adam, and the mixture
// density and sampler.
#include <math.h>

#include "ugp_guide_kernels.cuh"

namespace ugp {

GuideCfgDev guide_cfg_dev(const ugp_guide* g) {
  GuideCfgDev c;
  c.lo = make_float3(g->pos_lo[0], g->pos_lo[1], g->pos_lo[2]);
  float ie[3];
  for (int a = 0; a < 3; ++a) {
    const double ext = double(g->pos_hi[a]) - double(g->pos_lo[a]);
    ie[a] = ext > 0 ? float(1.0 / ext) : 0.f;
  }
  c.inv_ext = make_float3(ie[0], ie[1], ie[2]);
  c.kappa_min = g->kappa_min;
  c.kappa_max = g->kappa_max;
  return c;
}

int guide_sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

namespace {

__global__ void __launch_bounds__(256) k_guide_pack(const float* __restrict__ params, uint8_t* __restrict__ img) {
  const int t = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (t < 5 * kGWidth * kGWidth) {
    const int l = t / (kGWidth * kGWidth), o = (t / kGWidth) % kGWidth, i = t % kGWidth;
    const float w = o < guide_out_dim(l) ? params[guide_w_off(l) + o * kGWidth + i] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(w);
    *reinterpret_cast<__nv_bfloat16*>(img + kImgW + l * kImgTile + umma::tile_off(o, i, 64)) = h;
  } else if (t < 5 * kGWidth * kGWidth + 5 * kGWidth) {
    const int u = t - 5 * kGWidth * kGWidth, l = u / kGWidth, o = u % kGWidth;
    reinterpret_cast<float*>(img + kImgBias)[u] = o < guide_out_dim(l) ? params[guide_b_off(l) + o] : 0.f;
  }
}

__global__ void __launch_bounds__(256) k_guide_reduce(const float* __restrict__ partial, int grid,
                                                      float* __restrict__ grad, const float* __restrict__ loss_partial,
                                                      float* __restrict__ loss) {
  for (int p = int(blockIdx.x * blockDim.x + threadIdx.x); p < UGP_GUIDE_NPARAMS; p += int(gridDim.x * blockDim.x)) {
    float s = 0.f;
    for (int c = 0; c < grid; ++c) s += partial[size_t(c) * UGP_GUIDE_NPARAMS + p];
    grad[p] = s;
  }
  if (loss && blockIdx.x == 0 && threadIdx.x == 0) {
    float s = 0.f;
    for (int c = 0; c < grid; ++c) s += loss_partial[c];
    *loss = s;
  }
}

__global__ void __launch_bounds__(256) k_guide_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                                                    const float* __restrict__ g, float lr, float b1, float b2, float eps,
                                                    float c1, float c2) {
  for (int i = int(blockIdx.x * blockDim.x + threadIdx.x); i < UGP_GUIDE_NPARAMS; i += int(gridDim.x * blockDim.x)) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void k_mixture_pdf(int64_t n, const float* __restrict__ mix, const float* __restrict__ wi3,
                              float* __restrict__ pdf) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    float m[kGOut];
#pragma unroll
    for (int j = 0; j < kGOut; ++j) m[j] = mix[kGOut * i + j];
    pdf[i] = mixture_pdf(m, f3(wi3[3 * i], wi3[3 * i + 1], wi3[3 * i + 2]));
  }
}

__global__ void k_mixture_sample(int64_t n, const float* __restrict__ mix, const float* __restrict__ u3,
                                 float* __restrict__ wi3, float* __restrict__ pdf) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    float m[kGOut];
#pragma unroll
    for (int j = 0; j < kGOut; ++j) m[j] = mix[kGOut * i + j];
    const float3 w = mixture_sample(m, u3[3 * i], u3[3 * i + 1], u3[3 * i + 2]);
    wi3[3 * i] = w.x;
    wi3[3 * i + 1] = w.y;
    wi3[3 * i + 2] = w.z;
    if (pdf) pdf[i] = mixture_pdf(m, w);
  }
}

// Rows from caller arrays (float3 arrays of positions and directions).
struct ArraySrc {
  const float *x3, *wo3, *wi3, *w;
  __device__ bool vertex(int64_t r, float3& x, float3& wo) const {
    x = f3(x3[3 * r], x3[3 * r + 1], x3[3 * r + 2]);
    wo = f3(wo3[3 * r], wo3[3 * r + 1], wo3[3 * r + 2]);
    return true;
  }
  __device__ bool sample(int64_t r, float3& x, float3& wo, float3& wi, float& wt) const {
    vertex(r, x, wo);
    wi = f3(wi3[3 * r], wi3[3 * r + 1], wi3[3 * r + 2]);
    wt = w[r];
    return true;
  }
};

struct ArrayDst {
  float *head, *mix;
  GuideCfgDev cfg;
  // the mixture when asked for (then a head asked for as well is written here, per thread),
  // else the head
  __device__ float* row_out(int64_t r) const { return (mix ? mix : head) + kGOut * r; }
  __device__ void values(int64_t r, const float (&Y)[kGOut], float (&out)[kGOut]) const {
    if (mix) {
      if (head) {
#pragma unroll
        for (int j = 0; j < kGOut; ++j) head[kGOut * r + j] = Y[j];
      }
      mixture_from_head(cfg, Y, out);
    } else {
#pragma unroll
      for (int j = 0; j < kGOut; ++j) out[j] = Y[j];
    }
  }
};

int elementwise_grid(int64_t n, int block) {
  const int64_t need = (n + block - 1) / block;
  const int64_t cap = int64_t(guide_sm_count()) * 8;
  return int(need < cap ? (need > 0 ? need : 1) : cap);
}

ugp_status check_guide(const char* fn, const ugp_guide* g) {
  if (!g || !g->params) return fail(UGP_ERR_INVALID_ARG, "%s: NULL guide or parameters", fn);
  if (!(g->kappa_min > 0.f) || !(g->kappa_max >= g->kappa_min))
    return fail(UGP_ERR_INVALID_ARG, "%s: need 0 < kappa_min <= kappa_max", fn);
  for (int a = 0; a < 3; ++a)
    if (!(g->pos_hi[a] > g->pos_lo[a]))
      return fail(UGP_ERR_INVALID_ARG, "%s: pos_hi must exceed pos_lo on every axis", fn);
  return UGP_OK;
}

ugp_status check_ws(const char* fn, void* ws, size_t bytes) {
  if (!ws) return fail(UGP_ERR_INVALID_ARG, "%s: NULL workspace", fn);
  if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(UGP_ERR_INVALID_ARG, "%s: workspace must be 256-byte aligned", fn);
  if (bytes < guide_ws_bytes())
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "%s: need %zu bytes, got %zu", fn, guide_ws_bytes(), bytes);
  return UGP_OK;
}

}  // namespace

ugp_status launch_guide_pack(const float* params, uint8_t* img, cudaStream_t st) {
  const int total = 5 * kGWidth * kGWidth + 5 * kGWidth;
  prof_begin(kStGuide, st);
  k_guide_pack<<<(total + 255) / 256, 256, 0, st>>>(params, img);
  prof_end(kStGuide, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

ugp_status launch_guide_reduce(const GuideWs& ws, int grid, float* grad, float* loss, cudaStream_t st) {
  prof_begin(kStGuide, st);
  k_guide_reduce<<<(UGP_GUIDE_NPARAMS + 255) / 256, 256, 0, st>>>(ws.partial, grid, grad, ws.loss_partial, loss);
  prof_end(kStGuide, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

}  // namespace ugp

using namespace ugp;

extern "C" size_t ugp_guide_workspace_size(void) { return guide_ws_bytes(); }

extern "C" ugp_status ugp_guide_forward(const ugp_guide* g, int64_t n, const float* x3, const float* wo3,
                                        float* head_out, float* mix_out, void* workspace, size_t workspace_bytes,
                                        void* stream) {
  clear_error();
  ugp_status s = check_guide("ugp_guide_forward", g);
  if (s != UGP_OK) return s;
  if ((s = check_ws("ugp_guide_forward", workspace, workspace_bytes)) != UGP_OK) return s;
  if (n < 0 || n > (int64_t(1) << 31) - 1) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_forward: bad n %lld", (long long)n);
  if (n > 0 && (!x3 || !wo3)) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_forward: NULL input array");
  if (n == 0 || (!head_out && !mix_out)) return UGP_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const GuideWs ws = guide_ws_at(workspace);
  if ((s = launch_guide_pack(g->params, ws.img, st)) != UGP_OK) return s;
  const GuideDev gd{guide_cfg_dev(g), ws.img, ws.err};
  prof_begin(kStGuide, st);
  s = launch_guide_forward(gd, ArraySrc{x3, wo3, nullptr, nullptr}, ArrayDst{head_out, mix_out, gd.cfg}, n, nullptr,
                           n, st);
  prof_end(kStGuide, st);
  return s;
}

extern "C" ugp_status ugp_guide_mixture_pdf(int64_t n, const float* mix, const float* wi3, float* pdf_out,
                                            void* stream) {
  clear_error();
  if (n < 0) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_mixture_pdf: n < 0");
  if (n == 0) return UGP_OK;
  if (!mix || !wi3 || !pdf_out) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_mixture_pdf: NULL array");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_begin(kStGuide, st);
  k_mixture_pdf<<<elementwise_grid(n, 256), 256, 0, st>>>(n, mix, wi3, pdf_out);
  prof_end(kStGuide, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

extern "C" ugp_status ugp_guide_mixture_sample(int64_t n, const float* mix, const float* u3, float* wi_out,
                                               float* pdf_out, void* stream) {
  clear_error();
  if (n < 0) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_mixture_sample: n < 0");
  if (n == 0) return UGP_OK;
  if (!mix || !u3 || !wi_out) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_mixture_sample: NULL array");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_begin(kStGuide, st);
  k_mixture_sample<<<elementwise_grid(n, 256), 256, 0, st>>>(n, mix, u3, wi_out, pdf_out);
  prof_end(kStGuide, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}

extern "C" ugp_status ugp_guide_grad(const ugp_guide* g, int64_t n, const float* x3, const float* wo3,
                                     const float* wi3, const float* weight, float* grad_out, float* loss_out,
                                     void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  ugp_status s = check_guide("ugp_guide_grad", g);
  if (s != UGP_OK) return s;
  if ((s = check_ws("ugp_guide_grad", workspace, workspace_bytes)) != UGP_OK) return s;
  if (n < 0 || n > (int64_t(1) << 31) - 1) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_grad: bad n %lld", (long long)n);
  if (!grad_out) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_grad: NULL grad_out");
  if (n > 0 && (!x3 || !wo3 || !wi3 || !weight)) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_grad: NULL input array");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const GuideWs ws = guide_ws_at(workspace);
  if (n == 0) {
    UGP_CUDA_CHECK(cudaMemsetAsync(grad_out, 0, sizeof(float) * UGP_GUIDE_NPARAMS, st));
    if (loss_out) UGP_CUDA_CHECK(cudaMemsetAsync(loss_out, 0, sizeof(float), st));
    return UGP_OK;
  }
  if ((s = launch_guide_pack(g->params, ws.img, st)) != UGP_OK) return s;
  const GuideDev gd{guide_cfg_dev(g), ws.img, ws.err};
  int grid = 0;
  prof_begin(kStGuide, st);
  s = launch_guide_grad(gd, ArraySrc{x3, wo3, wi3, weight}, n, nullptr, n, ws, &grid, st);
  prof_end(kStGuide, st);
  if (s != UGP_OK) return s;
  return launch_guide_reduce(ws, grid, grad_out, loss_out, st);
}

extern "C" ugp_status ugp_guide_adam_step(ugp_guide* g, const float* grad, void* stream) {
  clear_error();
  ugp_status s = check_guide("ugp_guide_adam_step", g);
  if (s != UGP_OK) return s;
  if (!g->adam_m || !g->adam_v || !grad) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_adam_step: NULL moment or gradient");
  if (!(g->lr > 0.f) || !(g->beta1 >= 0.f && g->beta1 < 1.f) || !(g->beta2 >= 0.f && g->beta2 < 1.f) || !(g->eps > 0.f))
    return fail(UGP_ERR_INVALID_ARG, "ugp_guide_adam_step: bad hyper-parameters");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t t = g->step + 1;
  const float c1 = float(1.0 - pow(double(g->beta1), double(t)));
  const float c2 = float(1.0 - pow(double(g->beta2), double(t)));
  prof_begin(kStGuide, st);
  k_guide_adam<<<(UGP_GUIDE_NPARAMS + 255) / 256, 256, 0, st>>>(g->params, g->adam_m, g->adam_v, grad, g->lr,
                                                                 g->beta1, g->beta2, g->eps, c1, c2);
  prof_end(kStGuide, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  g->step = t;
  return UGP_OK;
}

extern "C" ugp_status ugp_guide_check(const void* workspace, void* stream) {
  clear_error();
  if (!workspace) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_check: NULL workspace");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int err = 0;
  UGP_CUDA_CHECK(cudaMemcpyAsync(&err, workspace, sizeof(int), cudaMemcpyDeviceToHost, st));
  UGP_CUDA_CHECK(cudaStreamSynchronize(st));
  if (err != 0) return fail(ugp_status(err), "ugp_guide_check: a tensor-core wait of the guide kernels gave up");
  return UGP_OK;
}

extern "C" ugp_status ugp_guide_reset_workspace(void* workspace, void* stream) {
  clear_error();
  if (!workspace) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_reset_workspace: NULL workspace");
  UGP_CUDA_CHECK(cudaMemsetAsync(workspace, 0, 256, static_cast<cudaStream_t>(stream)));
  return UGP_OK;
}
