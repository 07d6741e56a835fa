// Wavefront path tracer (Table 1, right column) over Gaussian primitives.
//
// One path per pixel per sample pass; per bounce these kernels run on the caller's stream (the
// free-flight finish passes of ugp_dense.cu follow k_extend):
//   k_extend   quad-light clip and free-flight sampling (Sec. 5.2) of every live path
//   k_shade    emission, light sampling with MIS, phase sampling (Sec. 6); live paths and
//              shadow rays are appended to queues with warp-aggregated atomics
//   k_shadow   transmittance of the shadow rays (Sec. 5.3): one launch for the area light's
//              samples, one for the emitters' (each path's two contributions then add up in
//              a fixed order)
// Queue lengths stay on the device, so a whole frame runs without host synchronisation;
// kernels walk their queue with grid-stride loops over a grid sized to the GPU.
//
// Readings of the paper (the oracle follows the same ones):
//  * max_depth D allows D scattering vertices: D + 1 free flights, the last only for
//    emission, and no light sampling from a vertex that cannot scatter again.
//  * Emissive primitives are pure emitters; escape adds the background, or the area light's
//    radiance if the ray reaches its front face.
//  * With an emitter table, each scattering vertex also takes a light sample of an emissive
//    primitive (ugp_emitters.cuh), balanced against phase sampling; with the area light as well,
//    a vertex takes one light sample of each, each balanced against phase sampling alone.
//  * Scattered and shadow rays start at the centre of the chosen primitive's clipped interval
//    and skip that primitive (Sec. 6).
//  * With a learned guide, a vertex draws its direction from the guide with probability alpha,
//    else by phase sampling, and weights it by the balance heuristic over both techniques with
//    the approximate phase pdf p~ of App. B (one-sample MIS, unbiased for any guide, Sec. 6);
//    alpha q + (1 - alpha) p~ is then the MIS partner of light sampling. The guide's mixtures
//    of a bounce come from one tensor-core pass over the shade queue before k_shade.
#include <cooperative_groups.h>

#include <cub/cub.cuh>
#include <math.h>

#include "ugp_dense.cuh"
#include "ugp_emitters.cuh"
#include "ugp_freeflight.cuh"
#include "ugp_guide_kernels.cuh"
#include "ugp_phase.cuh"
#include "ugp_philox.cuh"
#include "ugp_transmit.cuh"
#include "ugp_wavefront.cuh"

namespace ugp {
namespace {

// Training log of a guided frame: one entry per (bounce b, path p), e = b * n + p, as columns
// of E = max_depth * n floats:
//   0-2 vertex position, 3-5 wo, 6-8 sampled wi, 9 pdf of wi (alpha q + (1 - alpha) p~; 0:
//   no vertex), 10-12 throughput after the vertex, 13-15 path radiance before anything the
//   path gathers after the vertex (written at bounce b + 1), 16 training weight,
//   17 selection key (int), 18 selected entry indices (int), 19-21 throughput before the vertex.
constexpr int kLogCols = 22;
struct GuideLog {
  float* c[kLogCols];
  int64_t E;
};

struct GuidedShade {
  const float* mix;  // n x 40 mixtures, by path
  float alpha;
  float min_rough;   // vertices with a smoother glossy base use phase sampling alone
  int log;           // 1: write the training log
  GuideLog L;
  int n;             // paths per frame
};

__global__ void __launch_bounds__(256) k_camera(CameraDev cam, LightsDev L, int n, uint2 key, int sample, PathSoA ps,
                                                int* q, int* cnt, int* dense_cnt, int* scan_next) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const float3 d = camera_dir(cam, key, p, sample);
    ps.ox[p] = cam.eye.x; ps.oy[p] = cam.eye.y; ps.oz[p] = cam.eye.z;
    ps.dx[p] = d.x; ps.dy[p] = d.y; ps.dz[p] = d.z;
    ps.br[p] = 1.f; ps.bg[p] = 1.f; ps.bb[p] = 1.f;
    ps.lr[p] = 0.f; ps.lg[p] = 0.f; ps.lb[p] = 0.f;
    ps.pdf_prev[p] = -1.f;
    ps.excl[p] = -1;
    prepare_extend(ps, p, L, key, p, sample, 0, cam.eye, d);
    q[p] = p;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *cnt = n;
    *dense_cnt = 0;
    *scan_next = 0;
  }
}

// Rays of a bounce: the live paths in the queue.
struct PathScanSrc {
  TraceScene sc;
  int spawn_mode, count_;
  PathSoA ps;
  const int* q;
  DenseQueue dq;
  unsigned long long *rays, *stats;
  int i_, p, qf;
  float tq, u, u2;
  __device__ int count() const { return count_; }
  __device__ TraceScene scene() const { return sc; }
  __device__ bool begin(int i, ScanState& s, float& uo) {
    i_ = i;
    p = q[i];
    const float3 o = f3(ps.ox[p], ps.oy[p], ps.oz[p]), d = f3(ps.dx[p], ps.dy[p], ps.dz[p]);
    tq = ps.tq[p];
    qf = ps.qflag[p];
    s.ray = make_ray(o, d);
    s.t0 = 0.f;
    s.t1 = qf ? tq : 1e30f;
    s.ex = ps.excl[p];
    s.list = dq.list ? const_cast<int*>(dq.list) + size_t(p) * kListCap : nullptr;
    u = ps.fu[p];
    u2 = ps.fu2[p];
    uo = u;
    return true;
  }
  __device__ void finish(const ScanState& s, const FFResult& r) {
    if (r.pending) dense_push(dq, i_, p, r.lo, r.hi, r.Flo, u, u2, s.ray.o, s.ray.d, 0.f, s.t1, s.ex, r.nlist);
    else dense_none(dq, i_);
    ps.prim[p] = r.prim;
    ps.tsp[p] = spawn_mode == 1 ? r.t_u : r.t_spawn;
    if (s.st != UGP_RAY_OK && rays) atomicAdd(rays + 2, 1ull);
    if (stats) add_counters(stats, s.n_nodes, s.n_prims, 1u, 1u, r.pending ? 1u : 0u);
  }
};

__global__ void __launch_bounds__(kFFBlock, kFFBlocksPerSM) k_extend(TraceScene sc, LightsDev L, uint2 key, int sample, int bounce,
                                                     int spawn_mode, PathSoA ps, const int* __restrict__ q,
                                                     const int* cnt, int* reset_next, int* reset_shadow, int* reset_shadow_e,
                                                     unsigned long long* rays, unsigned long long* stats,
                                                     DenseQueue dq, int* scan_next) {
  __shared__ FFSmem sm;
  const int count = load_count(cnt);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *reset_next = 0;
    *reset_shadow = 0;
    *reset_shadow_e = 0;
    if (rays) atomicAdd(rays, (unsigned long long)count);
  }
  PathScanSrc src{sc, spawn_mode, count, ps, q, dq, rays, stats, 0, 0, 0, 0.f, 0.f, 0.f};
  scan_persistent(sm, src, scan_next);
}

template <bool kGuided>
__global__ void __launch_bounds__(128) k_shade(MatDev mats, LightsDev L, uint2 key, int sample, int bounce, int max_depth,
                                               int nee, PathSoA ps, const int* __restrict__ q, const int* cnt,
                                               int* __restrict__ q_next, int* cnt_next, ShadowSoA sh, int* cnt_shadow,
                                               ShadowSoA she, int* cnt_shadow_e,
                                               int* dense_cnt, int* scan_next, GuidedShade gs, EmitterDev E) {
  const bool em_on = emitters_on(E);
  const int count = load_count(cnt);
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // the extend and dense passes of this bounce have run
    *dense_cnt = 0;
    *scan_next = 0;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const int p = q[i];
    float3 beta = f3(ps.br[p], ps.bg[p], ps.bb[p]);
    float3 Lr = f3(ps.lr[p], ps.lg[p], ps.lb[p]);
    if (kGuided && gs.log && bounce > 0) {
      // radiance before anything gathered after the previous vertex (its light sample included)
      const int64_t e = int64_t(bounce - 1) * gs.n + p;
      gs.L.c[13][e] = Lr.x; gs.L.c[14][e] = Lr.y; gs.L.c[15][e] = Lr.z;
    }
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
      float w = 1.f;
      const float pdf_prev = ps.pdf_prev[p];
      const int e = em_on && pdf_prev >= 0.f ? E.map[k] : -1;
      if (e >= 0) {  // reached by phase sampling: the complement of the light-sampling weight
        const float4 m0 = E.rec[4 * e], m1 = E.rec[4 * e + 1], m2 = E.rec[4 * e + 2], m3 = E.rec[4 * e + 3];
        const float3 c = f3(m0.w, m1.w, m2.w) - o;
        w = mis_w(m3.x * pdf_prev, 2.f * dot3(c, c) * emitter_prob(E, e));
      }
      Lr = Lr + w * (beta * f3(mats.emission3[3 * k], mats.emission3[3 * k + 1], mats.emission3[3 * k + 2]));
    } else if (bounce < max_depth) {
      const Material M = load_material(mats, k);
      const float t = ps.tsp[p];
      const float3 x = o + t * d, wo = -d;
      // the guide's share at this vertex: none where the base is glossier than min_rough (its
      // lobe is already sampled well; the guide, trained on radiance alone, would spread samples
      // outside it)
      const float al_v = kGuided && !guide_smooth(M, gs.min_rough) ? gs.alpha : 0.f;
      float mix[kGuided ? kGOut : 1];
      if (kGuided) {
        const float4* m4 = reinterpret_cast<const float4*>(gs.mix + size_t(p) * kGOut);
#pragma unroll
        for (int j = 0; j < kGOut / 4; ++j) {
          const float4 v = m4[j];
          mix[4 * j] = v.x; mix[4 * j + 1] = v.y; mix[4 * j + 2] = v.z; mix[4 * j + 3] = v.w;
        }
      }
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
            float ps_l = phase_pdf_approx(M, wl, wo);
            if (kGuided) ps_l = al_v * mixture_pdf(mix, wl) + (1.f - al_v) * ps_l;
            const float wm = mis_w(pl, ps_l);
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
      if (em_on) {
        // light sampling of the emitters: emitter by power, point from its Gaussian inside the
        // ellipsoid (radius from the truncated chi-3 law, direction uniform), Philox slots 8-10
        const float4 Ua = rng(key, p, sample, bounce, 8);
        const long long e = emitter_pick(E, Ua.x);
        const float pj = emitter_prob(E, e);
        const float4 m0 = E.rec[4 * e], m1 = E.rec[4 * e + 1], m2 = E.rec[4 * e + 2], m3 = E.rec[4 * e + 3];
        const float rr = chi3_radius(Ua.y * E.mass, E.k);
        const float cz = 1.f - 2.f * Ua.z, sz = sqrtf(fmaxf(0.f, 1.f - cz * cz));
        float sp, cp;
        sincospif(2.f * Ua.w, &sp, &cp);
        const float zx = rr * sz * cp, zy = rr * sz * sp, zz = rr * cz;
        const float3 y = f3(m0.w + m0.x * zx + m0.y * zy + m0.z * zz, m1.w + m1.x * zx + m1.y * zy + m1.z * zz,
                            m2.w + m2.x * zx + m2.y * zy + m2.z * zz);
        const float3 w = y - x;
        const float r2 = dot3(w, w);
        if (r2 > 0.f && pj > 0.f) {
          const float r = sqrtf(r2);
          const float3 wl = (1.f / r) * w;
          const float4 Ub = rng(key, p, sample, bounce, 9), Uc = rng(key, p, sample, bounce, 10);
          const float Ue[6] = {Ub.x, Ub.y, Ub.z, Ub.w, Uc.x, Uc.y};
          const float3 f = phase_eval(M, wl, wo, Ue);
          if (f.x > 0.f || f.y > 0.f || f.z > 0.f) {
            float ps_l = phase_pdf_approx(M, wl, wo);
            if (kGuided) ps_l = al_v * mixture_pdf(mix, wl) + (1.f - al_v) * ps_l;
            const float3 c = f3(m0.w, m1.w, m2.w) - x;
            const float wm = mis_w(2.f * dot3(c, c) * pj, m3.x * ps_l);
            const float3 contrib = (wm * 0.5f * m3.x / (r2 * pj)) * (beta * (f * f3(m3.y, m3.z, m3.w)));
            const int j = queue_append(cnt_shadow_e);
            she.path[j] = p;
            she.ox[j] = x.x; she.oy[j] = x.y; she.oz[j] = x.z;
            she.dx[j] = wl.x; she.dy[j] = wl.y; she.dz[j] = wl.z;
            she.dist[j] = -r;  // negative: the contribution counts when T > 0, unscaled
            she.excl[j] = k;
            she.cr[j] = contrib.x; she.cg[j] = contrib.y; she.cb[j] = contrib.z;
          }
        }
      }
      float3 wi, wgt;
      float pdf_s = 0.f;
      bool sampled = false;
      if (!kGuided) {
        const float4 Us = rng(key, p, sample, bounce, 1);
        const float U4[4] = {Us.x, Us.y, Us.z, Us.w};
        sampled = phase_sample(M, wo, U4, wi, wgt);
        if (sampled) pdf_s = phase_pdf_approx(M, wi, wo);
      } else {
        const float al = al_v;
        const float4 G = rng(key, p, sample, bounce, 2);
        if (G.y < al) {
          wi = mixture_sample(mix, G.x, G.z, G.w);
          const float4 Ga = rng(key, p, sample, bounce, 6), Gb = rng(key, p, sample, bounce, 7);
          const float Ug[6] = {Ga.x, Ga.y, Ga.z, Ga.w, Gb.x, Gb.y};
          const float3 f = phase_eval(M, wi, wo, Ug);
          pdf_s = al * mixture_pdf(mix, wi) + (1.f - al) * phase_pdf_approx(M, wi, wo);
          sampled = pdf_s > 0.f;
          if (sampled) wgt = (1.f / pdf_s) * f;
        } else {
          const float4 Us = rng(key, p, sample, bounce, 1);
          const float U4[4] = {Us.x, Us.y, Us.z, Us.w};
          float3 w0;
          if (phase_sample(M, wo, U4, wi, w0)) {
            const float pt = phase_pdf_approx(M, wi, wo);
            pdf_s = al * mixture_pdf(mix, wi) + (1.f - al) * pt;
            sampled = pdf_s > 0.f;
            if (sampled) wgt = (pt / pdf_s) * w0;
          }
        }
      }
      if (sampled) {
        const float3 beta_in = beta;
        beta = beta * wgt;
        if (beta.x > 0.f || beta.y > 0.f || beta.z > 0.f) {
          ps.pdf_prev[p] = pdf_s;
          prepare_extend(ps, p, L, key, p, sample, bounce + 1, x, wi);
          if (kGuided && gs.log) {
            const int64_t e = int64_t(bounce) * gs.n + p;
            float* const* c = gs.L.c;
            c[0][e] = x.x; c[1][e] = x.y; c[2][e] = x.z;
            c[3][e] = wo.x; c[4][e] = wo.y; c[5][e] = wo.z;
            c[6][e] = wi.x; c[7][e] = wi.y; c[8][e] = wi.z;
            c[9][e] = pdf_s;
            c[10][e] = beta.x; c[11][e] = beta.y; c[12][e] = beta.z;
            c[19][e] = beta_in.x; c[20][e] = beta_in.y; c[21][e] = beta_in.z;
          }
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

__global__ void __launch_bounds__(kTrBlock, kTrBlocksPerSM) k_shadow(TraceScene sc, ShadowSoA sh, const int* cnt, PathSoA ps,
                                                     unsigned long long* rays, unsigned long long* stats) {
  __shared__ int stk[kTrStack * kTrBlock];
  __shared__ unsigned long long tr_acc[kTrBlock];
  __shared__ int tr_owner[kTrBlock];
  const int count = load_count(cnt);
  if (blockIdx.x == 0 && threadIdx.x == 0 && rays) atomicAdd(rays + 1, (unsigned long long)count);
  // one ray per thread over a grid sized for the longest queue: the hardware spreads the blocks
  const int j = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (j >= count) return;
  const Ray ray = make_ray(f3(sh.ox[j], sh.oy[j], sh.oz[j]), f3(sh.dx[j], sh.dy[j], sh.dz[j]));
  TrStats ts{0u, 0u, UGP_RAY_OK};
  // a negative distance marks a light sample of an emissive primitive: it counts when the
  // point lies before saturation (T > 0) and is not scaled by T
  const float dist = sh.dist[j];
  const float tau = tr_optical_depth(sc, ray, 0.f, fabsf(dist), sh.excl[j], stk + threadIdx.x, kTrBlock,
                                     tr_acc + threadIdx.x, tr_owner + threadIdx.x, ts);
  const float T = fmaxf(0.f, 1.f - tau);
  if (T > 0.f) {
    const float s = dist < 0.f ? 1.f : T;
    const int p = sh.path[j];
    ps.lr[p] += s * sh.cr[j];
    ps.lg[p] += s * sh.cg[j];
    ps.lb[p] += s * sh.cb[j];
  }
  if (ts.st != UGP_RAY_OK && rays) atomicAdd(rays + 2, 1ull);
  if (stats) add_counters(stats + 6, ts.n_nodes, ts.n_prims, 1u, 1u, 0u);
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

// Rows of the guide's forward pass in a bounce: the entries of the shade queue; a row is a
// vertex when its path scatters here (a non-emissive primitive before the depth limit).
struct ShadeQueueSrc {
  PathSoA ps;
  const int* q;
  const uint8_t* type;
  int bounce, max_depth;
  __device__ bool vertex(int64_t r, float3& x, float3& wo) const {
    const int p = q[r];
    const int k = ps.prim[p];
    if (k < 0 || bounce >= max_depth || type[k] == kMatEmissive) return false;
    const float3 o = f3(ps.ox[p], ps.oy[p], ps.oz[p]), d = f3(ps.dx[p], ps.dy[p], ps.dz[p]);
    x = o + ps.tsp[p] * d;
    wo = -d;
    return true;
  }
};

struct MixByPathDst {
  const int* q;
  float* mix;
  GuideCfgDev cfg;
  __device__ float* row_out(int64_t r) const { return mix + size_t(q[r]) * kGOut; }
  __device__ void values(int64_t, const float (&Y)[kGOut], float (&out)[kGOut]) const {
    mixture_from_head(cfg, Y, out);
  }
};

// Training rows: selected log entries, taken cyclically from `offset` (n_sel entries).
struct LogSrc {
  GuideLog L;
  const int* idx;
  int64_t offset, n_sel;
  __device__ bool sample(int64_t r, float3& x, float3& wo, float3& wi, float& w) const {
    const int64_t e = idx[(offset + r) % n_sel];
    x = f3(L.c[0][e], L.c[1][e], L.c[2][e]);
    wo = f3(L.c[3][e], L.c[4][e], L.c[5][e]);
    wi = f3(L.c[6][e], L.c[7][e], L.c[8][e]);
    w = L.c[16][e];
    return true;
  }
};

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  // integer finaliser of MurmurHash3 (public domain)
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}

// Training weight of every logged vertex; counts the usable ones. Target 0: the incident-
// radiance estimate L_i (gathered radiance over the throughput after the vertex) over the pdf;
// target 1: f_p L_i / pdf, the gathered radiance over the throughput before the vertex.
__global__ void __launch_bounds__(256) k_log_finalize(GuideLog L, int n, PathSoA ps, int* count, int target) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < L.E; e += int64_t(gridDim.x) * blockDim.x) {
    const float pdf = L.c[9][e];
    float w = 0.f;
    if (pdf > 0.f) {
      const int p = int(e % n);
      const float Lf[3] = {ps.lr[p], ps.lg[p], ps.lb[p]};
      const float lum[3] = {0.2126f, 0.7152f, 0.0722f};
      float Li = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float b = L.c[(target == 1 ? 19 : 10) + c][e];
        if (b > 0.f) Li += lum[c] * fmaxf(0.f, (Lf[c] - L.c[13 + c][e]) / b);
      }
      w = target == 1 ? Li : Li / pdf;
      if (!(w > 0.f) || !isfinite(w)) w = 0.f;
    }
    L.c[16][e] = w;
    if (w > 0.f) atomicAdd(count, 1);
  }
}

// Keeps about max_samples of the usable entries (hash thinning): key = e if kept, else -1.
__global__ void __launch_bounds__(256) k_log_thin(GuideLog L, const int* count, int64_t max_samples) {
  const int c = *count;
  const double keep = c > max_samples ? double(max_samples) / double(c) : 1.0;
  const uint32_t thr = keep >= 1.0 ? 0xffffffffu : uint32_t(keep * 4294967295.0);
  int* key = reinterpret_cast<int*>(L.c[17]);
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < L.E; e += int64_t(gridDim.x) * blockDim.x) {
    const bool use = L.c[16][e] > 0.f && (keep >= 1.0 || hash32(uint32_t(e) * 0x9e3779b9u + 0x2406u) <= thr);
    key[e] = use ? int(e) : -1;
  }
}

struct NonNegative {
  __device__ __forceinline__ bool operator()(const int& v) const { return v >= 0; }
};

struct RenderLayout {
  size_t total;
  size_t state, queues, shadow, counts, dense, lists;
  // guided renders only
  size_t mix, log, img, cub, cub_bytes;
  int64_t E;
};

RenderLayout render_layout(int64_t n, int max_depth = -1) {
  RenderLayout L;
  size_t off = 0;
  const size_t col = align256(size_t(n) * 4);
  L.state = off;   off += 20 * col;
  L.queues = off;  off += 2 * col;
  L.shadow = off;  off += 24 * col;  // light samples of the area light, then of the emitters
  L.counts = off;  off += 256;
  L.dense = off;   off += dense_queue_bytes(n);
  L.lists = off;   off += slot_list_bytes(n);
  L.mix = L.log = L.img = L.cub = L.cub_bytes = 0;
  L.E = 0;
  if (max_depth >= 0) {
    L.E = int64_t(max_depth > 0 ? max_depth : 1) * n;
    L.mix = off;   off += align256(size_t(n) * kGOut * 4);
    L.log = off;   off += size_t(kLogCols) * align256(size_t(L.E) * 4);
    L.img = off;   off += 256 + align256(kImgBytes);
    size_t cb = 0;
    cub::DeviceSelect::If(nullptr, cb, (const int*)nullptr, (int*)nullptr, (int*)nullptr, int(L.E), NonNegative());
    L.cub_bytes = cb;
    L.cub = off;   off += align256(cb + 256);
  }
  L.total = off;
  return L;
}

GuideLog log_at(char* ws, const RenderLayout& RL) {
  GuideLog g;
  const size_t col = align256(size_t(RL.E) * 4);
  for (int c = 0; c < kLogCols; ++c) g.c[c] = reinterpret_cast<float*>(ws + RL.log + c * col);
  g.E = RL.E;
  return g;
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

}  // namespace
}  // namespace ugp

using namespace ugp;

extern "C" size_t ugp_render_workspace_size(int32_t width, int32_t height) {
  if (width <= 0 || height <= 0 || int64_t(width) * height > (int64_t(1) << 31) - 1) return 0;
  return render_layout(int64_t(width) * height).total;
}

extern "C" size_t ugp_render_guided_workspace_size(int32_t width, int32_t height, int32_t max_depth) {
  if (width <= 0 || height <= 0 || max_depth < 0 || max_depth > 14) return 0;
  const int64_t n = int64_t(width) * height;
  if (n * (max_depth > 0 ? max_depth : 1) > (int64_t(1) << 31) - 1) return 0;
  return render_layout(n, max_depth).total;
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
  const ugp_guide* guide = params->guide;
  if (guide) {
    if (!(params->guide_alpha > 0.f && params->guide_alpha < 1.f))
      return fail(UGP_ERR_INVALID_ARG, "ugp_render: guide_alpha must be in (0, 1)");
    if (!guide->params || !(guide->kappa_min > 0.f) || !(guide->kappa_max >= guide->kappa_min))
      return fail(UGP_ERR_INVALID_ARG, "ugp_render: bad guide (NULL parameters or kappa range)");
    for (int a = 0; a < 3; ++a)
      if (!(guide->pos_hi[a] > guide->pos_lo[a]))
        return fail(UGP_ERR_INVALID_ARG, "ugp_render: guide pos_hi must exceed pos_lo");
  }
  if (params->guide_log && (!guide || params->spp != 1))
    return fail(UGP_ERR_INVALID_ARG, "ugp_render: guide_log needs a guide and spp == 1");
  const int64_t n = int64_t(W) * H;
  if (guide && n * (params->max_depth > 0 ? params->max_depth : 1) > (int64_t(1) << 31) - 1)
    return fail(UGP_ERR_INVALID_ARG, "ugp_render: image too large for a guided render");
  const RenderLayout RL = render_layout(n, guide ? params->max_depth : -1);
  if (workspace_bytes < RL.total)
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_render: need %zu bytes, got %zu", RL.total, workspace_bytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream_);

  char* ws = static_cast<char*>(workspace);
  const size_t col = align256(size_t(n) * 4);
  auto F = [&](size_t base, int k) { return reinterpret_cast<float*>(ws + base + k * col); };
  auto I = [&](size_t base, int k) { return reinterpret_cast<int*>(ws + base + k * col); };
  PathSoA ps{F(RL.state, 0), F(RL.state, 1), F(RL.state, 2), F(RL.state, 3), F(RL.state, 4), F(RL.state, 5),
             F(RL.state, 6), F(RL.state, 7), F(RL.state, 8), F(RL.state, 9), F(RL.state, 10), F(RL.state, 11),
             F(RL.state, 12), I(RL.state, 13), I(RL.state, 14), F(RL.state, 15), F(RL.state, 16), I(RL.state, 17),
             F(RL.state, 18), F(RL.state, 19)};
  ShadowSoA sh{I(RL.shadow, 0), F(RL.shadow, 1), F(RL.shadow, 2), F(RL.shadow, 3), F(RL.shadow, 4),
               F(RL.shadow, 5), F(RL.shadow, 6), F(RL.shadow, 7), I(RL.shadow, 8), F(RL.shadow, 9),
               F(RL.shadow, 10), F(RL.shadow, 11)};
  ShadowSoA she{I(RL.shadow, 12), F(RL.shadow, 13), F(RL.shadow, 14), F(RL.shadow, 15), F(RL.shadow, 16),
                F(RL.shadow, 17), F(RL.shadow, 18), F(RL.shadow, 19), I(RL.shadow, 20), F(RL.shadow, 21),
                F(RL.shadow, 22), F(RL.shadow, 23)};
  int* queue[2] = {I(RL.queues, 0), I(RL.queues, 1)};
  // [0], [1] queue lengths, [2] shadow rays toward the area light, [3] scan ray counter,
  // [4] shadow rays toward emitters
  int* counts = reinterpret_cast<int*>(ws + RL.counts);
  int* scan_next = counts + 3;
  DenseQueue dq = dense_queue_at(ws + RL.dense, n);
  dq.list = reinterpret_cast<const int*>(ws + RL.lists);

  const LightsDev Ld = lights_dev(lights);
  CameraDev cd;
  {
    const ugp_status cs = camera_dev(camera, "ugp_render", &cd);
    if (cs != UGP_OK) return cs;
  }
  const MatDev md{materials->sggx6, materials->type, materials->albedo3, materials->roughness, materials->emission3,
                  materials->disney9};
  const TraceScene sc = trace_scene(bvh);
  const uint2 key = make_uint2(uint32_t(params->seed & 0xffffffffu), uint32_t(params->seed >> 32));
  unsigned long long* stats = trace_counters();
  if (params->emitters && (reinterpret_cast<uintptr_t>(params->emitters) & 255))
    return fail(UGP_ERR_INVALID_ARG, "ugp_render: emitter table must be 256-byte aligned");
  const EmitterDev Em = emitter_dev(params->emitters, bvh);

  GuidedShade gs{};
  GuideDev gd{};
  if (guide) {
    gs.mix = reinterpret_cast<const float*>(ws + RL.mix);
    gs.alpha = params->guide_alpha;
    gs.min_rough = params->guide_min_roughness;
    gs.log = params->guide_log;
    gs.L = log_at(ws, RL);
    gs.n = int(n);
    gd.cfg = guide_cfg_dev(guide);
    gd.err = reinterpret_cast<int*>(ws + RL.img);
    gd.img = reinterpret_cast<const uint8_t*>(ws + RL.img + 256);
    const ugp_status s = launch_guide_pack(guide->params, const_cast<uint8_t*>(gd.img), st);
    if (s != UGP_OK) return s;
    if (params->guide_log)  // no vertex yet: every entry's pdf is zero
      UGP_CUDA_CHECK(cudaMemsetAsync(gs.L.c[9], 0, size_t(RL.E) * 4, st));
  }
  const int g_cam = grid_for((const void*)k_camera, 256, n);
  const int g_ext = grid_for((const void*)k_extend, kFFBlock, n);
  const int g_shade = guide ? grid_for((const void*)k_shade<true>, 128, n) : grid_for((const void*)k_shade<false>, 128, n);
  const int g_shadow = int((n + kTrBlock - 1) / kTrBlock);
  const int g_acc = grid_for((const void*)k_accumulate, 256, n);
  for (int si = 0; si < params->spp; ++si) {
    const int sample = params->spp_begin + si;
    prof_begin(kStCamera, st);
    k_camera<<<g_cam, 256, 0, st>>>(cd, Ld, int(n), key, sample, ps, queue[0], counts + 0, dq.count, scan_next);
    prof_end(kStCamera, st);
    int cur = 0;
    for (int b = 0; b <= params->max_depth; ++b) {
      const int nxt = 1 - cur;
      prof_begin(kStExtend, st);
      k_extend<<<g_ext, kFFBlock, 0, st>>>(sc, Ld, key, sample, b, params->spawn_mode, ps, queue[cur], counts + cur,
                                            counts + nxt, counts + 2, counts + 4, ray_counts, stats, dq, scan_next);
      prof_end(kStExtend, st);
      {
        const ugp_status ds = launch_dense(sc, dq, 0, counts + cur, n, ps.prim, nullptr, ps.tsp, nullptr,
                                           params->spawn_mode, stats, ray_counts ? ray_counts + 2 : nullptr, st);
        if (ds != UGP_OK) return ds;
      }
      if (guide && b < params->max_depth) {
        prof_begin(kStGuide, st);
        const ugp_status gsx = launch_guide_forward(
            gd, ShadeQueueSrc{ps, queue[cur], md.type, b, params->max_depth},
            MixByPathDst{queue[cur], const_cast<float*>(gs.mix), gd.cfg}, n, counts + cur, n, st);
        prof_end(kStGuide, st);
        if (gsx != UGP_OK) return gsx;
      }
      prof_begin(kStShade, st);
      if (guide)
        k_shade<true><<<g_shade, 128, 0, st>>>(md, Ld, key, sample, b, params->max_depth, params->nee, ps, queue[cur],
                                                counts + cur, queue[nxt], counts + nxt, sh, counts + 2, she, counts + 4, dq.count,
                                                scan_next, gs, Em);
      else
        k_shade<false><<<g_shade, 128, 0, st>>>(md, Ld, key, sample, b, params->max_depth, params->nee, ps,
                                                 queue[cur], counts + cur, queue[nxt], counts + nxt, sh, counts + 2, she, counts + 4,
                                                 dq.count, scan_next, gs, Em);
      prof_end(kStShade, st);
      // one launch per kind of light sample: a path's two shadow rays add to its radiance in
      // this order, so the sum does not depend on scheduling
      if (params->nee && Ld.has_quad) {
        prof_begin(kStShadow, st);
        k_shadow<<<g_shadow, kTrBlock, 0, st>>>(sc, sh, counts + 2, ps, ray_counts, stats);
        prof_end(kStShadow, st);
      }
      if (Em.cdf) {
        prof_begin(kStShadow, st);
        k_shadow<<<g_shadow, kTrBlock, 0, st>>>(sc, she, counts + 4, ps, ray_counts, stats);
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

extern "C" ugp_status ugp_guide_train_from_render(ugp_guide* g, const void* render_ws, size_t render_ws_bytes,
                                                  int32_t width, int32_t height, int32_t max_depth,
                                                  int64_t max_samples, int32_t minibatch, int32_t min_steps,
                                                  void* guide_ws,
                                                  size_t guide_ws_bytes, int64_t* n_samples_out,
                                                  float* mean_loss_out, void* stream_) {
  clear_error();
  if (!g || !g->params || !g->adam_m || !g->adam_v)
    return fail(UGP_ERR_INVALID_ARG, "ugp_guide_train_from_render: NULL guide, parameters or moments");
  if (!render_ws || !guide_ws) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_train_from_render: NULL workspace");
  if (width <= 0 || height <= 0 || max_depth < 1 || max_depth > 14 || max_samples < 1 || minibatch < 1 ||
      min_steps < 0)
    return fail(UGP_ERR_INVALID_ARG, "ugp_guide_train_from_render: bad size argument");
  const int64_t n = int64_t(width) * height;
  if (n * max_depth > (int64_t(1) << 31) - 1) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_train_from_render: too large");
  const RenderLayout RL = render_layout(n, max_depth);
  if (render_ws_bytes < RL.total)
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_guide_train_from_render: render workspace needs %zu bytes", RL.total);
  if (guide_ws_bytes < ugp::guide_ws_bytes())
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_guide_train_from_render: guide workspace needs %zu bytes",
                ugp::guide_ws_bytes());
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  char* ws = static_cast<char*>(const_cast<void*>(render_ws));
  const size_t col = align256(size_t(n) * 4);
  PathSoA ps{};
  ps.lr = reinterpret_cast<float*>(ws + RL.state + 9 * col);
  ps.lg = reinterpret_cast<float*>(ws + RL.state + 10 * col);
  ps.lb = reinterpret_cast<float*>(ws + RL.state + 11 * col);
  const GuideLog L = log_at(ws, RL);
  int* cnt = reinterpret_cast<int*>(ws + RL.cub);  // [0] usable entries, [1] selected entries
  void* cub_tmp = ws + RL.cub + 256;
  UGP_CUDA_CHECK(cudaMemsetAsync(cnt, 0, 2 * sizeof(int), st));
  const int grid = grid_for((const void*)k_log_finalize, 256, RL.E);
  prof_begin(kStGuide, st);
  k_log_finalize<<<grid, 256, 0, st>>>(L, int(n), ps, cnt, g->train_target == 1 ? 1 : 0);
  prof_end(kStGuide, st);
  prof_begin(kStGuide, st);
  k_log_thin<<<grid, 256, 0, st>>>(L, cnt, max_samples);
  prof_end(kStGuide, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  int* sel = reinterpret_cast<int*>(L.c[18]);
  size_t cb = RL.cub_bytes;
  prof_begin(kStGuide, st);
  UGP_CUDA_CHECK(cub::DeviceSelect::If(cub_tmp, cb, reinterpret_cast<const int*>(L.c[17]), sel, cnt + 1, int(RL.E),
                                       NonNegative(), st));
  prof_end(kStGuide, st, 1);
  int n_sel = 0;
  UGP_CUDA_CHECK(cudaMemcpyAsync(&n_sel, cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  UGP_CUDA_CHECK(cudaStreamSynchronize(st));
  if (n_samples_out) *n_samples_out = n_sel;
  const GuideWs gw = guide_ws_at(guide_ws);
  ugp_status s = launch_guide_pack(g->params, gw.img, st);
  if (s != UGP_OK) return s;
  // gradient and loss of each minibatch land in the guide workspace's scratch after the partials
  float* grad = gw.partial + size_t(kGMaxGradBlocks - 1) * UGP_GUIDE_NPARAMS;
  float* loss = gw.loss_partial + kGMaxGradBlocks - 1;
  const GuideDev gd{guide_cfg_dev(g), gw.img, gw.err};
  // one pass over the samples, or min_steps minibatches taken cyclically if that is more
  const int64_t m = n_sel < minibatch ? n_sel : minibatch;
  const int64_t pass = n_sel > 0 ? (n_sel + minibatch - 1) / minibatch : 0;
  const int64_t steps = n_sel > 0 ? (pass > min_steps ? pass : min_steps) : 0;
  for (int64_t k = 0; k < steps; ++k) {
    const int64_t i0 = (k * m) % n_sel;
    const int64_t rows = (k < pass && n_sel - i0 < m) ? n_sel - i0 : m;
    if (k > 0 && (s = launch_guide_pack(g->params, gw.img, st)) != UGP_OK) return s;
    int gg = 0;
    prof_begin(kStGuide, st);
    s = launch_guide_grad(gd, LogSrc{L, sel, i0, n_sel}, rows, nullptr, rows, gw, &gg, st);
    prof_end(kStGuide, st);
    if (s != UGP_OK) return s;
    if (gg >= kGMaxGradBlocks) return fail(UGP_ERR_INVALID_ARG, "ugp_guide_train_from_render: too many blocks");
    if ((s = launch_guide_reduce(gw, gg, grad, loss, st)) != UGP_OK) return s;
    if ((s = ugp_guide_adam_step(g, grad, st)) != UGP_OK) return s;
  }
  if (mean_loss_out) {
    float lv = 0.f;
    if (n_sel > 0) {
      UGP_CUDA_CHECK(cudaMemcpyAsync(&lv, loss, sizeof(float), cudaMemcpyDeviceToHost, st));
      UGP_CUDA_CHECK(cudaStreamSynchronize(st));
    }
    *mean_loss_out = lv;
  }
  return UGP_OK;
}
