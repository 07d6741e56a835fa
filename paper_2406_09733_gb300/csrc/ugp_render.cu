// Wavefront path tracer (Table 1, right column) over Gaussian primitives.
//
// One path per pixel per sample pass; per bounce three kernels run on the caller's stream:
//   k_extend   quad-light clip and free-flight sampling (Sec. 5.2) of every live path
//   k_shade    emission, light sampling with MIS, phase sampling (Sec. 6); live paths and
//              shadow rays are appended to queues with warp-aggregated atomics
//   k_shadow   transmittance of the shadow rays (Sec. 5.3)
// Queue lengths stay on the device, so a whole frame runs without host synchronisation;
// kernels walk their queue with grid-stride loops over a grid sized to the GPU.
//
// Readings of the paper (the oracle follows the same ones):
//  * max_depth D allows D scattering vertices: D + 1 free flights, the last only for
//    emission, and no light sampling from a vertex that cannot scatter again.
//  * Emissive primitives are pure emitters; escape adds the background, or the area light's
//    radiance if the ray reaches its front face.
//  * Scattered and shadow rays start at the centre of the chosen primitive's clipped interval
//    and skip that primitive (Sec. 6).
#include <cooperative_groups.h>

#include <math.h>

#include "ugp_dense.cuh"
#include "ugp_freeflight.cuh"
#include "ugp_phase.cuh"
#include "ugp_philox.cuh"
#include "ugp_transmit.cuh"

namespace cg = cooperative_groups;

namespace ugp {
namespace {

struct PathSoA {
  float *ox, *oy, *oz, *dx, *dy, *dz;
  float *br, *bg, *bb;   // throughput beta
  float *lr, *lg, *lb;   // radiance so far
  float* pdf_prev;       // approximate phase pdf of the last scattering (< 0: none)
  int* excl;             // primitive the current ray skips
  int* prim;             // free-flight result
  float* tsp;            // spawn distance along the current ray
  float* tq;             // distance to the area light along the current ray
  int* qflag;            // 0 no light hit, 1 front face, 2 back face
};

struct ShadowSoA {
  int* path;
  float *ox, *oy, *oz, *dx, *dy, *dz, *dist;
  int* excl;
  float *cr, *cg, *cb;   // contribution if unoccluded
};

struct LightsDev {
  int has_quad;
  float3 corner, e1, e2, Le, bg, nrm;  // nrm = unit e1 x e2
  float area;
};

struct CameraDev {
  float3 eye, fwd, right, up;
  float th, aspect;
  int width, height;
};

struct MatDev {
  const float* sggx6;
  const uint8_t* type;
  const float* albedo3;
  const float* roughness;
  const float* emission3;
};

__device__ __forceinline__ float4 rng(uint2 key, int pixel, int sample, int bounce, int slot) {
  const uint4 x = philox4x32_10(make_uint4(uint32_t(pixel), uint32_t(sample), uint32_t(16 * bounce + slot), 0u), key);
  return make_float4(u24(x.x), u24(x.y), u24(x.z), u24(x.w));
}

__device__ __forceinline__ int load_count(const int* c) { return *reinterpret_cast<const volatile int*>(c); }

// Ray / parallelogram intersection with t in (0, tmax).
__device__ __forceinline__ int quad_hit(const LightsDev& L, float3 o, float3 d, float& t) {
  if (!L.has_quad) return 0;
  const float den = dot3(d, L.nrm);
  if (fabsf(den) < 1e-30f) return 0;
  const float tt = dot3(L.corner - o, L.nrm) / den;
  if (!(tt > 0.f && tt < 1e30f)) return 0;
  const float3 q = o + tt * d - L.corner;
  const float e11 = dot3(L.e1, L.e1), e22 = dot3(L.e2, L.e2), e12 = dot3(L.e1, L.e2);
  const float q1 = dot3(q, L.e1), q2 = dot3(q, L.e2);
  const float det = e11 * e22 - e12 * e12;
  const float al = (q1 * e22 - q2 * e12) / det, be = (q2 * e11 - q1 * e12) / det;
  if (al < 0.f || al > 1.f || be < 0.f || be > 1.f) return 0;
  t = tt;
  return den < 0.f ? 1 : 2;
}

// Appends the calling thread to a queue; the threads of a warp that take the same call share
// one atomic.
__device__ __forceinline__ int queue_append(int* counter) {
  cg::coalesced_group g = cg::coalesced_threads();
  int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(counter, int(g.size()));
  base = g.shfl(base, 0);
  return base + int(g.thread_rank());
}

__global__ void __launch_bounds__(256) k_camera(CameraDev cam, int n, uint2 key, int sample, PathSoA ps, int* q,
                                                int* cnt, int* dense_cnt) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int px = p % cam.width, py = p / cam.width;
    const float4 U = rng(key, p, sample, 15, 0);
    const float x = (2.f * (float(px) + U.x) / float(cam.width) - 1.f) * cam.th * cam.aspect;
    const float y = (1.f - 2.f * (float(py) + U.y) / float(cam.height)) * cam.th;
    const float3 d = normalize3(cam.fwd + x * cam.right + y * cam.up);
    ps.ox[p] = cam.eye.x; ps.oy[p] = cam.eye.y; ps.oz[p] = cam.eye.z;
    ps.dx[p] = d.x; ps.dy[p] = d.y; ps.dz[p] = d.z;
    ps.br[p] = 1.f; ps.bg[p] = 1.f; ps.bb[p] = 1.f;
    ps.lr[p] = 0.f; ps.lg[p] = 0.f; ps.lb[p] = 0.f;
    ps.pdf_prev[p] = -1.f;
    ps.excl[p] = -1;
    q[p] = p;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *cnt = n;
    *dense_cnt = 0;
  }
}

__global__ void __launch_bounds__(kFFBlock) k_extend(TraceScene sc, LightsDev L, uint2 key, int sample, int bounce,
                                                     int spawn_mode, PathSoA ps, const int* __restrict__ q,
                                                     const int* cnt, int* reset_next, int* reset_shadow,
                                                     unsigned long long* rays, unsigned long long* stats,
                                                     DenseQueue dq) {
  __shared__ FFSmem sm;
  const int count = load_count(cnt);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *reset_next = 0;
    *reset_shadow = 0;
    if (rays) atomicAdd(rays, (unsigned long long)count);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const int p = q[i];
    const float3 o = f3(ps.ox[p], ps.oy[p], ps.oz[p]), d = f3(ps.dx[p], ps.dy[p], ps.dz[p]);
    float tq = 1e30f;
    const int qf = quad_hit(L, o, d, tq);
    const float t1 = qf ? tq : 1e30f;
    const float4 U = rng(key, p, sample, bounce, 0);
    Ctx c{sm, int(threadIdx.x), sc, make_ray(o, d), 0.f, t1, ps.excl[p], 0u, 0u, UGP_RAY_OK,
          dq.list ? const_cast<int*>(dq.list) + size_t(p) * kListCap : nullptr, 0};
    const FFResult r = ff_sample(c, U.x, U.y);
    if (r.pending) dense_push(dq, p, r.lo, r.hi, r.Flo, U.x, U.y, o, d, 0.f, t1, c.ex, r.nlist);
    ps.prim[p] = r.prim;
    ps.tsp[p] = spawn_mode == 1 ? r.t_u : r.t_spawn;
    ps.tq[p] = tq;
    ps.qflag[p] = qf;
    if (c.st != UGP_RAY_OK && rays) atomicAdd(rays + 2, 1ull);
    if (stats) add_counters(stats, c.n_nodes, c.n_prims, 1u, 1u, r.pending ? 1u : 0u);
  }
}

__device__ __forceinline__ Material load_material(const MatDev& m, int k) {
  Material M;
  M.type = m.type[k];
  M.albedo = f3(m.albedo3[3 * k], m.albedo3[3 * k + 1], m.albedo3[3 * k + 2]);
  M.alpha = m.roughness[k];
  for (int j = 0; j < 6; ++j) M.S[j] = m.sggx6[6 * k + j];
  return M;
}

__global__ void __launch_bounds__(128) k_shade(MatDev mats, LightsDev L, uint2 key, int sample, int bounce, int max_depth,
                                               int nee, PathSoA ps, const int* __restrict__ q, const int* cnt,
                                               int* __restrict__ q_next, int* cnt_next, ShadowSoA sh, int* cnt_shadow,
                                               int* dense_cnt) {
  const int count = load_count(cnt);
  if (blockIdx.x == 0 && threadIdx.x == 0) *dense_cnt = 0;  // the dense pass of this bounce has run
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const int p = q[i];
    float3 beta = f3(ps.br[p], ps.bg[p], ps.bb[p]);
    float3 Lr = f3(ps.lr[p], ps.lg[p], ps.lb[p]);
    const float3 o = f3(ps.ox[p], ps.oy[p], ps.oz[p]), d = f3(ps.dx[p], ps.dy[p], ps.dz[p]);
    const int k = ps.prim[p];
    bool alive = false;
    if (k < 0) {
      const int qf = ps.qflag[p];
      if (qf == 1) {
        float w = 1.f;
        const float pdf_prev = ps.pdf_prev[p];
        if (nee && pdf_prev >= 0.f) {
          const float tq = ps.tq[p];
          const float pl = tq * tq / (L.area * -dot3(d, L.nrm));
          w = mis_w(pdf_prev, pl);
        }
        Lr = Lr + w * (beta * L.Le);
      } else if (qf == 0) {
        Lr = Lr + beta * L.bg;
      }
    } else if (mats.type[k] == kMatEmissive) {
      Lr = Lr + beta * f3(mats.emission3[3 * k], mats.emission3[3 * k + 1], mats.emission3[3 * k + 2]);
    } else if (bounce < max_depth) {
      const Material M = load_material(mats, k);
      const float t = ps.tsp[p];
      const float3 x = o + t * d, wo = -d;
      if (nee && L.has_quad && L.area > 0.f) {
        const float4 Uy = rng(key, p, sample, bounce, 3);
        const float3 y = L.corner + Uy.x * L.e1 + Uy.y * L.e2;
        const float3 w = y - x;
        const float r2 = dot3(w, w), r = sqrtf(r2);
        const float3 wl = (1.f / r) * w;
        const float cl = -dot3(wl, L.nrm);
        if (cl > 0.f) {
          const float pl = r2 / (L.area * cl);
          const float4 Ua = rng(key, p, sample, bounce, 4), Ub = rng(key, p, sample, bounce, 5);
          const float Ue[6] = {Ua.x, Ua.y, Ua.z, Ua.w, Ub.x, Ub.y};
          const float3 f = phase_eval(M, wl, wo, Ue);
          if (f.x > 0.f || f.y > 0.f || f.z > 0.f) {
            const float wm = mis_w(pl, phase_pdf_approx(M, wl, wo));
            const float3 contrib = (wm / pl) * (beta * (f * L.Le));
            const int j = queue_append(cnt_shadow);
            sh.path[j] = p;
            sh.ox[j] = x.x; sh.oy[j] = x.y; sh.oz[j] = x.z;
            sh.dx[j] = wl.x; sh.dy[j] = wl.y; sh.dz[j] = wl.z;
            sh.dist[j] = r;
            sh.excl[j] = k;
            sh.cr[j] = contrib.x; sh.cg[j] = contrib.y; sh.cb[j] = contrib.z;
          }
        }
      }
      const float4 Us = rng(key, p, sample, bounce, 1);
      const float U4[4] = {Us.x, Us.y, Us.z, Us.w};
      float3 wi, wgt;
      if (phase_sample(M, wo, U4, wi, wgt)) {
        beta = beta * wgt;
        if (beta.x > 0.f || beta.y > 0.f || beta.z > 0.f) {
          ps.pdf_prev[p] = phase_pdf_approx(M, wi, wo);
          ps.ox[p] = x.x; ps.oy[p] = x.y; ps.oz[p] = x.z;
          ps.dx[p] = wi.x; ps.dy[p] = wi.y; ps.dz[p] = wi.z;
          ps.br[p] = beta.x; ps.bg[p] = beta.y; ps.bb[p] = beta.z;
          ps.excl[p] = k;
          alive = true;
        }
      }
    }
    ps.lr[p] = Lr.x; ps.lg[p] = Lr.y; ps.lb[p] = Lr.z;
    if (alive) q_next[queue_append(cnt_next)] = p;
  }
}

__global__ void __launch_bounds__(kTrBlock) k_shadow(TraceScene sc, ShadowSoA sh, const int* cnt, PathSoA ps,
                                                     unsigned long long* rays, unsigned long long* stats) {
  __shared__ int stk[kTrStack * kTrBlock];
  const int count = load_count(cnt);
  if (blockIdx.x == 0 && threadIdx.x == 0 && rays) atomicAdd(rays + 1, (unsigned long long)count);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x) {
    const Ray ray = make_ray(f3(sh.ox[j], sh.oy[j], sh.oz[j]), f3(sh.dx[j], sh.dy[j], sh.dz[j]));
    TrStats ts{0u, 0u, UGP_RAY_OK};
    const float tau = tr_optical_depth(sc, ray, 0.f, sh.dist[j], sh.excl[j], stk + threadIdx.x, kTrBlock, ts);
    const float T = fmaxf(0.f, 1.f - tau);
    if (T > 0.f) {
      const int p = sh.path[j];
      ps.lr[p] += T * sh.cr[j];
      ps.lg[p] += T * sh.cg[j];
      ps.lb[p] += T * sh.cb[j];
    }
    if (ts.st != UGP_RAY_OK && rays) atomicAdd(rays + 2, 1ull);
    if (stats) add_counters(stats + 6, ts.n_nodes, ts.n_prims, 1u, 1u, 0u);
  }
}

__global__ void __launch_bounds__(256) k_accumulate(int n, PathSoA ps, float* __restrict__ acc, float* __restrict__ acc2) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const float r = ps.lr[p], g = ps.lg[p], b = ps.lb[p];
    acc[3 * p] += r;
    acc[3 * p + 1] += g;
    acc[3 * p + 2] += b;
    acc2[3 * p] += r * r;
    acc2[3 * p + 1] += g * g;
    acc2[3 * p + 2] += b * b;
  }
}

struct RenderLayout {
  size_t total;
  size_t state, queues, shadow, counts, dense, lists;
};

RenderLayout render_layout(int64_t n) {
  RenderLayout L;
  size_t off = 0;
  const size_t col = align256(size_t(n) * 4);
  L.state = off;   off += 18 * col;
  L.queues = off;  off += 2 * col;
  L.shadow = off;  off += 12 * col;
  L.counts = off;  off += 256;
  L.dense = off;   off += dense_queue_bytes(n);
  L.lists = off;   off += slot_list_bytes(n);
  L.total = off;
  return L;
}

int grid_for(const void* kernel, int block, int64_t n) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm <= 0) per_sm = 1;
  const int64_t need = (n + block - 1) / block;
  return int(need < int64_t(sms) * per_sm ? (need > 0 ? need : 1) : int64_t(sms) * per_sm);
}

float3 h3(const float* v) { return make_float3(v[0], v[1], v[2]); }

}  // namespace
}  // namespace ugp

using namespace ugp;

extern "C" size_t ugp_render_workspace_size(int32_t width, int32_t height) {
  if (width <= 0 || height <= 0 || int64_t(width) * height > (int64_t(1) << 31) - 1) return 0;
  return render_layout(int64_t(width) * height).total;
}

extern "C" ugp_status ugp_render(const ugp_bvh* bvh, const ugp_materials* materials, const ugp_camera* camera,
                                 const ugp_lights* lights, const ugp_render_params* params, float* accum_rgb,
                                 float* accum_sq_rgb, void* workspace, size_t workspace_bytes,
                                 unsigned long long* ray_counts, void* stream_) {
  clear_error();
  if (!valid_bvh(bvh)) return fail(UGP_ERR_NOT_BUILT, "ugp_render: invalid BVH handle");
  if (!materials || !camera || !lights || !params || !accum_rgb || !accum_sq_rgb || !workspace)
    return fail(UGP_ERR_INVALID_ARG, "ugp_render: NULL argument");
  if (bvh->n_prims > 0 && (!materials->sggx6 || !materials->type || !materials->albedo3 ||
                           !materials->roughness || !materials->emission3))
    return fail(UGP_ERR_INVALID_ARG, "ugp_render: NULL material array");
  const int W = camera->width, H = camera->height;
  if (W <= 0 || H <= 0 || int64_t(W) * H > (int64_t(1) << 31) - 1)
    return fail(UGP_ERR_INVALID_ARG, "ugp_render: bad image size %d x %d", W, H);
  if (params->spp < 0 || params->spp_begin < 0 || params->max_depth < 0 || params->max_depth > 14)
    return fail(UGP_ERR_INVALID_ARG, "ugp_render: spp, spp_begin must be >= 0 and max_depth in [0, 14]");
  if (!(camera->vfov_deg > 0.f && camera->vfov_deg < 180.f))
    return fail(UGP_ERR_INVALID_ARG, "ugp_render: vfov_deg must be in (0, 180)");
  if (reinterpret_cast<uintptr_t>(workspace) & 255)
    return fail(UGP_ERR_INVALID_ARG, "ugp_render: workspace must be 256-byte aligned");
  const int64_t n = int64_t(W) * H;
  const RenderLayout RL = render_layout(n);
  if (workspace_bytes < RL.total)
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_render: need %zu bytes, got %zu", RL.total, workspace_bytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream_);

  char* ws = static_cast<char*>(workspace);
  const size_t col = align256(size_t(n) * 4);
  auto F = [&](size_t base, int k) { return reinterpret_cast<float*>(ws + base + k * col); };
  auto I = [&](size_t base, int k) { return reinterpret_cast<int*>(ws + base + k * col); };
  PathSoA ps{F(RL.state, 0), F(RL.state, 1), F(RL.state, 2), F(RL.state, 3), F(RL.state, 4), F(RL.state, 5),
             F(RL.state, 6), F(RL.state, 7), F(RL.state, 8), F(RL.state, 9), F(RL.state, 10), F(RL.state, 11),
             F(RL.state, 12), I(RL.state, 13), I(RL.state, 14), F(RL.state, 15), F(RL.state, 16), I(RL.state, 17)};
  ShadowSoA sh{I(RL.shadow, 0), F(RL.shadow, 1), F(RL.shadow, 2), F(RL.shadow, 3), F(RL.shadow, 4),
               F(RL.shadow, 5), F(RL.shadow, 6), F(RL.shadow, 7), I(RL.shadow, 8), F(RL.shadow, 9),
               F(RL.shadow, 10), F(RL.shadow, 11)};
  int* queue[2] = {I(RL.queues, 0), I(RL.queues, 1)};
  int* counts = reinterpret_cast<int*>(ws + RL.counts);  // [0], [1] queue lengths, [2] shadow
  DenseQueue dq = dense_queue_at(ws + RL.dense, n);
  dq.list = reinterpret_cast<const int*>(ws + RL.lists);

  LightsDev Ld;
  Ld.has_quad = lights->has_quad != 0;
  Ld.corner = h3(lights->quad_corner);
  Ld.e1 = h3(lights->quad_e1);
  Ld.e2 = h3(lights->quad_e2);
  Ld.Le = h3(lights->quad_Le);
  Ld.bg = h3(lights->bg);
  {
    const double e1[3] = {lights->quad_e1[0], lights->quad_e1[1], lights->quad_e1[2]};
    const double e2[3] = {lights->quad_e2[0], lights->quad_e2[1], lights->quad_e2[2]};
    const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double a = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    Ld.area = float(a);
    Ld.nrm = a > 0 ? make_float3(float(c[0] / a), float(c[1] / a), float(c[2] / a)) : make_float3(0.f, 0.f, 1.f);
    if (Ld.has_quad && !(a > 0)) Ld.has_quad = 0;
  }
  CameraDev cd;
  {
    double f[3] = {double(camera->look[0]) - camera->eye[0], double(camera->look[1]) - camera->eye[1],
                   double(camera->look[2]) - camera->eye[2]};
    const double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fl > 0)) return fail(UGP_ERR_INVALID_ARG, "ugp_render: eye and look coincide");
    for (double& v : f) v /= fl;
    const double up[3] = {camera->up[0], camera->up[1], camera->up[2]};
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    const double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rl > 0)) return fail(UGP_ERR_INVALID_ARG, "ugp_render: up is parallel to the view direction");
    for (double& v : r) v /= rl;
    const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    cd.eye = h3(camera->eye);
    cd.fwd = make_float3(float(f[0]), float(f[1]), float(f[2]));
    cd.right = make_float3(float(r[0]), float(r[1]), float(r[2]));
    cd.up = make_float3(float(u[0]), float(u[1]), float(u[2]));
    cd.th = float(tan(0.5 * double(camera->vfov_deg) * 3.14159265358979323846 / 180.0));
    cd.aspect = float(double(W) / double(H));
    cd.width = W;
    cd.height = H;
  }
  const MatDev md{materials->sggx6, materials->type, materials->albedo3, materials->roughness, materials->emission3};
  const TraceScene sc = trace_scene(bvh);
  const uint2 key = make_uint2(uint32_t(params->seed & 0xffffffffu), uint32_t(params->seed >> 32));
  unsigned long long* stats = trace_counters();

  const int g_cam = grid_for((const void*)k_camera, 256, n);
  const int g_ext = grid_for((const void*)k_extend, kFFBlock, n);
  const int g_shade = grid_for((const void*)k_shade, 128, n);
  const int g_shadow = grid_for((const void*)k_shadow, kTrBlock, n);
  const int g_acc = grid_for((const void*)k_accumulate, 256, n);
  for (int si = 0; si < params->spp; ++si) {
    const int sample = params->spp_begin + si;
    prof_begin(kStCamera, st);
    k_camera<<<g_cam, 256, 0, st>>>(cd, int(n), key, sample, ps, queue[0], counts + 0, dq.count);
    prof_end(kStCamera, st);
    int cur = 0;
    for (int b = 0; b <= params->max_depth; ++b) {
      const int nxt = 1 - cur;
      prof_begin(kStExtend, st);
      k_extend<<<g_ext, kFFBlock, 0, st>>>(sc, Ld, key, sample, b, params->spawn_mode, ps, queue[cur], counts + cur,
                                            counts + nxt, counts + 2, ray_counts, stats, dq);
      prof_end(kStExtend, st);
      {
        const ugp_status ds = launch_dense(sc, dq, ps.prim, nullptr, ps.tsp, nullptr, params->spawn_mode, stats,
                                           ray_counts ? ray_counts + 2 : nullptr, st);
        if (ds != UGP_OK) return ds;
      }
      prof_begin(kStShade, st);
      k_shade<<<g_shade, 128, 0, st>>>(md, Ld, key, sample, b, params->max_depth, params->nee, ps, queue[cur],
                                        counts + cur, queue[nxt], counts + nxt, sh, counts + 2, dq.count);
      prof_end(kStShade, st);
      if (params->nee && Ld.has_quad) {
        prof_begin(kStShadow, st);
        k_shadow<<<g_shadow, kTrBlock, 0, st>>>(sc, sh, counts + 2, ps, ray_counts, stats);
        prof_end(kStShadow, st);
      }
      cur = nxt;
    }
    prof_begin(kStAccum, st);
    k_accumulate<<<g_acc, 256, 0, st>>>(int(n), ps, accum_rgb, accum_sq_rgb);
    prof_end(kStAccum, st);
    UGP_CUDA_CHECK(cudaGetLastError());
  }
  return UGP_OK;
}
