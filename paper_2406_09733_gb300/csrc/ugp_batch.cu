// Batched rendering: many independent render requests, each with its own scene, camera, lights,
// image size, spp and depth, served together by one wavefront over a shared pool of paths.
//
// Work is a list of items (request r, sample s, image tile t), in request order, then sample,
// then tile. A wave
//   1. claims as many items as the free pool slots hold (one thread) and turns every tile
//      pixel into a camera path in a free slot, appended to the live queue;
//   2. extends every live path (free-flight sampling in its request's scene), finishes the
//      bracketed ones (16 lanes per ray), shades them (emission, light sampling with MIS, phase
//      sampling with the request's materials and lights), and traces the shadow rays;
//   3. retires the paths that ended: adds their radiance to the request's image, counts them,
//      stamps the request's completion time (%globaltimer) when its last path lands, and
//      returns the slots to the free stack.
// Every path keeps its pixel, sample and bounce, and draws the same Philox numbers as
// ugp_render would for that request, so each image equals the single-request render up to the
// order of the floating-point sums.
//
// The waves run inside one CUDA graph launch: a conditional while-node whose body is one wave,
// with the last kernel of the wave setting the condition (more work or live paths, and fewer
// waves than the bound). Without graphs the host runs the same waves and polls the flag.
#include <algorithm>
#include <mutex>
#include <vector>

#include "ugp_dense.cuh"
#include "ugp_freeflight.cuh"
#include "ugp_transmit.cuh"
#include "ugp_umma.cuh"
#include "ugp_wavefront.cuh"

namespace ugp {
namespace {

// Device record of one request.
struct BReq {
  MatDev md;
  LightsDev L;
  CameraDev cam;
  uint2 key;
  int spp, depth, nee, spawn;
  int tiles_x, n_tiles;
  long long item_begin, items, paths;
  float *acc, *acc2;
};

// Counters and per-wave bookkeeping (one 256-byte block of the workspace).
struct BCtl {
  unsigned long long work_next, items_total;
  unsigned long long start_ns;
  int live[2];
  int shadow, retire, free_top, wave;
  int claim_n, claim_base, claim_stack, claim_items;
  long long claim_item0;
  int n_req, tile, tile_px, pool, max_waves, status, more;
  unsigned long long* rays;        // caller's ray counters of this batch (may be NULL)
  unsigned long long dense_err;    // rays of the warp finish that ended with a non-zero status
  int scan_next;                   // ray counter of the persistent scan of this wave
  int dense_slots;                 // slots of this wave's finish table (the live paths)
};
static_assert(sizeof(BCtl) <= 256, "control block");

struct BPaths {
  PathSoA ps;
  float* tu;  // t_u of the free flight (spawn_mode 1)
  int *req, *pix, *smp, *bounce;
};

struct BState {
  int64_t pool;
  BCtl* ctl;
  const BReq* reqs;
  const TraceScene* scenes;
  unsigned long long *done, *finish_ns;
  BPaths P;
  int* live[2];
  int* retire;
  int* stack;
  ShadowSoA sh;
  DenseQueue dq;
};
// Kernel parameters hold only workspace addresses (fixed for a cached graph); per-call values
// such as the caller's ray counters live in the control block.

constexpr int kPathCols = 25;  // PathSoA (20) + tu, req, pix, smp, bounce

__device__ __forceinline__ int find_request(const BReq* reqs, int n, long long item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {  // last request with item_begin <= item
    const int mid = (lo + hi + 1) >> 1;
    if (reqs[mid].item_begin <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_b_init(BState S, int n_req, unsigned long long items_total, int tile, int pool, int max_waves,
                         unsigned long long* rays) {
  const int tid = int(blockIdx.x * blockDim.x + threadIdx.x), nt = int(gridDim.x * blockDim.x);
  for (int i = tid; i < pool; i += nt) S.stack[i] = pool - 1 - i;
  for (int r = tid; r < n_req; r += nt) {
    S.done[r] = 0ull;
    S.finish_ns[r] = 0ull;
  }
  if (tid == 0) {
    BCtl& c = *S.ctl;
    c.work_next = 0ull;
    c.items_total = items_total;
    c.live[0] = c.live[1] = 0;
    c.shadow = c.retire = 0;
    c.free_top = pool;
    c.wave = 0;
    c.claim_n = c.claim_base = c.claim_stack = c.claim_items = 0;
    c.claim_item0 = 0;
    c.n_req = n_req;
    c.tile = tile;
    c.tile_px = tile * tile;
    c.pool = pool;
    c.max_waves = max_waves;
    c.status = 0;
    c.more = items_total > 0 ? 1 : 0;
    c.rays = rays;
    c.dense_err = 0ull;
    c.scan_next = 0;
    *S.dq.count = 0;
    c.start_ns = umma::global_timer_ns();
  }
}

// Claims the items of this wave (one thread).
__global__ void k_b_claim(BState S) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  BCtl& c = *S.ctl;
  const int cur = c.wave & 1;
  const unsigned long long left = c.items_total - c.work_next;
  unsigned long long n = (unsigned long long)(c.free_top / c.tile_px);
  if (n > left) n = left;
  c.claim_items = int(n);
  c.claim_item0 = (long long)c.work_next;
  c.claim_n = int(n) * c.tile_px;
  c.claim_base = c.live[cur];
  c.claim_stack = c.free_top - c.claim_n;
  c.free_top -= c.claim_n;
  c.work_next += n;
  c.live[cur] += c.claim_n;
  c.dense_slots = c.live[cur];
}

// New camera paths for the claimed items (tile pixels outside the image become empty paths,
// pix = -1, retired in the same wave without a contribution).
__global__ void __launch_bounds__(256) k_b_regen(BState S) {
  const BCtl& c = *S.ctl;
  const int n = c.claim_n;
  const int cur = c.wave & 1;
  const int T = c.tile, TP = c.tile_px;
  const BPaths& P = S.P;
  for (int k = int(blockIdx.x * blockDim.x + threadIdx.x); k < n; k += int(gridDim.x * blockDim.x)) {
    const int slot = S.stack[c.claim_stack + k];
    const long long item = c.claim_item0 + k / TP;
    const int local = k % TP;
    const int r = find_request(S.reqs, c.n_req, item);
    const BReq& R = S.reqs[r];
    const long long j = item - R.item_begin;
    const int sample = int(j / R.n_tiles), tile = int(j % R.n_tiles);
    const int px = (tile % R.tiles_x) * T + local % T, py = (tile / R.tiles_x) * T + local / T;
    const bool inside = px < R.cam.width && py < R.cam.height;
    const int p = py * R.cam.width + px;
    P.req[slot] = r;
    P.pix[slot] = inside ? p : -1;
    P.smp[slot] = sample;
    P.bounce[slot] = 0;
    if (inside) {
      const float3 d = camera_dir(R.cam, R.key, p, sample);
      P.ps.ox[slot] = R.cam.eye.x; P.ps.oy[slot] = R.cam.eye.y; P.ps.oz[slot] = R.cam.eye.z;
      P.ps.dx[slot] = d.x; P.ps.dy[slot] = d.y; P.ps.dz[slot] = d.z;
      P.ps.br[slot] = 1.f; P.ps.bg[slot] = 1.f; P.ps.bb[slot] = 1.f;
      P.ps.lr[slot] = 0.f; P.ps.lg[slot] = 0.f; P.ps.lb[slot] = 0.f;
      P.ps.pdf_prev[slot] = -1.f;
      P.ps.excl[slot] = -1;
      prepare_extend(P.ps, slot, R.L, R.key, p, sample, 0, R.cam.eye, d);
    }
    S.live[cur][c.claim_base + k] = slot;
  }
}

// Rays of a wave: the live paths, each in its own request's scene. S refers to the kernel's
// parameter (read through the constant bank, not copied into local memory).
struct BatchScanSrc {
  const BState& S;
  int cur, count_;
  int i_, p, r, qf;
  float tq, u, u2;
  TraceScene sc;
  __device__ int count() const { return count_; }
  __device__ TraceScene scene() const { return sc; }
  __device__ bool begin(int i, ScanState& s, float& uo) {
    i_ = i;
    p = S.live[cur][i];
    const int pix = S.P.pix[p];
    if (pix < 0) {  // empty path of a partial tile
      dense_none(S.dq, i);
      return false;
    }
    r = S.P.req[p];
    const BReq& R = S.reqs[r];
    sc = S.scenes[r];
    const PathSoA& ps = S.P.ps;
    const float3 o = f3(ps.ox[p], ps.oy[p], ps.oz[p]), d = f3(ps.dx[p], ps.dy[p], ps.dz[p]);
    tq = ps.tq[p];
    qf = ps.qflag[p];
    s.ray = make_ray(o, d);
    s.t0 = 0.f;
    s.t1 = qf ? tq : 1e30f;
    s.ex = ps.excl[p];
    s.list = S.dq.list ? const_cast<int*>(S.dq.list) + size_t(p) * kListCap : nullptr;
    u = ps.fu[p];
    u2 = ps.fu2[p];
    uo = u;
    return true;
  }
  __device__ void finish(const ScanState& s, const FFResult& fr) {
    if (fr.pending) dense_push(S.dq, i_, p, fr.lo, fr.hi, fr.Flo, u, u2, s.ray.o, s.ray.d, 0.f, s.t1, s.ex, fr.nlist, r);
    else dense_none(S.dq, i_);
    S.P.ps.prim[p] = fr.prim;
    S.P.ps.tsp[p] = fr.t_spawn;
    S.P.tu[p] = fr.t_u;
    unsigned long long* rays = S.ctl->rays;
    if (rays) {
      atomicAdd(rays, 1ull);
      if (s.st != UGP_RAY_OK) atomicAdd(rays + 2, 1ull);
    }
  }
};

__global__ void __launch_bounds__(kFFBlock, kFFBlocksPerSM) k_b_extend(BState S) {
  __shared__ FFSmem sm;
  const BCtl& c = *S.ctl;
  const int cur = c.wave & 1;
  BatchScanSrc src{S, cur, c.live[cur], 0, 0, 0, 0, 0.f, 0.f, 0.f, TraceScene{}};
  scan_persistent(sm, src, &S.ctl->scan_next);
}

__global__ void __launch_bounds__(128) k_b_shade(BState S) {
  const BCtl& c = *S.ctl;
  const int cur = c.wave & 1, nxt = cur ^ 1;
  const int count = c.live[cur];
  const BPaths& P = S.P;
  BCtl* cw = S.ctl;
  for (int i = int(blockIdx.x * blockDim.x + threadIdx.x); i < count; i += int(gridDim.x * blockDim.x)) {
    const int p = S.live[cur][i];
    const int pix = P.pix[p];
    bool alive = false;
    if (pix >= 0) {
      const int r = P.req[p];
      const BReq& R = S.reqs[r];
      const LightsDev& L = R.L;
      const int bounce = P.bounce[p], sample = P.smp[p];
      float3 beta = f3(P.ps.br[p], P.ps.bg[p], P.ps.bb[p]);
      float3 Lr = f3(P.ps.lr[p], P.ps.lg[p], P.ps.lb[p]);
      const float3 o = f3(P.ps.ox[p], P.ps.oy[p], P.ps.oz[p]), d = f3(P.ps.dx[p], P.ps.dy[p], P.ps.dz[p]);
      const int k = P.ps.prim[p];
      if (k < 0) {
        const int qf = P.ps.qflag[p];
        if (qf == 1) {
          float w = 1.f;
          const float pdf_prev = P.ps.pdf_prev[p];
          if (R.nee && pdf_prev >= 0.f) {
            const float tq = P.ps.tq[p];
            const float pl = tq * tq / (L.area * -dot3(d, L.nrm));
            w = mis_w(pdf_prev, pl);
          }
          Lr = Lr + w * (beta * L.Le);
        } else if (qf == 0) {
          Lr = Lr + beta * L.bg;
        }
      } else if (R.md.type[k] == kMatEmissive) {
        Lr = Lr + beta * f3(R.md.emission3[3 * k], R.md.emission3[3 * k + 1], R.md.emission3[3 * k + 2]);
      } else if (bounce < R.depth) {
        const Material M = load_material(R.md, k);
        const float t = R.spawn == 1 ? P.tu[p] : P.ps.tsp[p];
        const float3 x = o + t * d, wo = -d;
        if (R.nee && L.has_quad && L.area > 0.f) {
          const float4 Uy = rng(R.key, pix, sample, bounce, 3);
          const float3 y = L.corner + Uy.x * L.e1 + Uy.y * L.e2;
          const float3 w = y - x;
          const float r2 = dot3(w, w), rr = sqrtf(r2);
          const float3 wl = (1.f / rr) * w;
          const float cl = -dot3(wl, L.nrm);
          if (cl > 0.f) {
            const float pl = r2 / (L.area * cl);
            const float4 Ua = rng(R.key, pix, sample, bounce, 4), Ub = rng(R.key, pix, sample, bounce, 5);
            const float Ue[6] = {Ua.x, Ua.y, Ua.z, Ua.w, Ub.x, Ub.y};
            const float3 f = phase_eval(M, wl, wo, Ue);
            if (f.x > 0.f || f.y > 0.f || f.z > 0.f) {
              const float wm = mis_w(pl, phase_pdf_approx(M, wl, wo));
              const float3 contrib = (wm / pl) * (beta * (f * L.Le));
              const int j = queue_append(&cw->shadow);
              S.sh.path[j] = p;
              S.sh.ox[j] = x.x; S.sh.oy[j] = x.y; S.sh.oz[j] = x.z;
              S.sh.dx[j] = wl.x; S.sh.dy[j] = wl.y; S.sh.dz[j] = wl.z;
              S.sh.dist[j] = rr;
              S.sh.excl[j] = k;
              S.sh.cr[j] = contrib.x; S.sh.cg[j] = contrib.y; S.sh.cb[j] = contrib.z;
            }
          }
        }
        const float4 Us = rng(R.key, pix, sample, bounce, 1);
        const float U4[4] = {Us.x, Us.y, Us.z, Us.w};
        float3 wi, wgt;
        if (phase_sample(M, wo, U4, wi, wgt)) {
          beta = beta * wgt;
          if (beta.x > 0.f || beta.y > 0.f || beta.z > 0.f) {
            P.ps.pdf_prev[p] = phase_pdf_approx(M, wi, wo);
            P.ps.ox[p] = x.x; P.ps.oy[p] = x.y; P.ps.oz[p] = x.z;
            P.ps.dx[p] = wi.x; P.ps.dy[p] = wi.y; P.ps.dz[p] = wi.z;
            P.ps.br[p] = beta.x; P.ps.bg[p] = beta.y; P.ps.bb[p] = beta.z;
            P.ps.excl[p] = k;
            P.bounce[p] = bounce + 1;
            prepare_extend(P.ps, p, L, R.key, pix, sample, bounce + 1, x, wi);
            alive = true;
          }
        }
      }
      P.ps.lr[p] = Lr.x; P.ps.lg[p] = Lr.y; P.ps.lb[p] = Lr.z;
    }
    if (alive) S.live[nxt][queue_append(&cw->live[nxt])] = p;
    else S.retire[queue_append(&cw->retire)] = p;
  }
}

__global__ void __launch_bounds__(kTrBlock, kTrBlocksPerSM) k_b_shadow(BState S) {
  __shared__ int stk[kTrStack * kTrBlock];
  __shared__ unsigned long long tr_acc[kTrBlock];
  __shared__ int tr_owner[kTrBlock];
  const int count = S.ctl->shadow;
  const BPaths& P = S.P;
  // one ray per thread over a grid sized for the pool: the hardware spreads the blocks
  const int j = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (j >= count) return;
  const int p = S.sh.path[j];
  const TraceScene sc = S.scenes[P.req[p]];
  const Ray ray = make_ray(f3(S.sh.ox[j], S.sh.oy[j], S.sh.oz[j]), f3(S.sh.dx[j], S.sh.dy[j], S.sh.dz[j]));
  TrStats ts{0u, 0u, UGP_RAY_OK};
  const float tau = tr_optical_depth(sc, ray, 0.f, S.sh.dist[j], S.sh.excl[j], stk + threadIdx.x, kTrBlock,
                                     tr_acc + threadIdx.x, tr_owner + threadIdx.x, ts);
  const float T = fmaxf(0.f, 1.f - tau);
  if (T > 0.f) {
    P.ps.lr[p] += T * S.sh.cr[j];
    P.ps.lg[p] += T * S.sh.cg[j];
    P.ps.lb[p] += T * S.sh.cb[j];
  }
  unsigned long long* rays = S.ctl->rays;
  if (rays) {
    atomicAdd(rays + 1, 1ull);
    if (ts.st != UGP_RAY_OK) atomicAdd(rays + 2, 1ull);
  }
}

__global__ void __launch_bounds__(256) k_b_retire(BState S) {
  const int count = S.ctl->retire;
  const BPaths& P = S.P;
  for (int i = int(blockIdx.x * blockDim.x + threadIdx.x); i < count; i += int(gridDim.x * blockDim.x)) {
    const int p = S.retire[i];
    const int pix = P.pix[p];
    if (pix >= 0) {
      const int r = P.req[p];
      const BReq& R = S.reqs[r];
      const float v[3] = {P.ps.lr[p], P.ps.lg[p], P.ps.lb[p]};
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        atomicAdd(R.acc + 3 * size_t(pix) + ch, v[ch]);
        atomicAdd(R.acc2 + 3 * size_t(pix) + ch, v[ch] * v[ch]);
      }
      __threadfence();
      const unsigned long long d = atomicAdd(S.done + r, 1ull) + 1ull;
      if ((long long)d == R.paths) S.finish_ns[r] = umma::global_timer_ns();
    }
    S.stack[atomicAdd(&S.ctl->free_top, 1)] = p;
  }
}

// End of a wave: reset the per-wave counters and decide whether another wave runs.
__global__ void k_b_cond(BState S, cudaGraphConditionalHandle handle, int use_graph) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  BCtl& c = *S.ctl;
  const int cur = c.wave & 1, nxt = cur ^ 1;
  c.live[cur] = 0;
  c.shadow = 0;
  c.retire = 0;
  c.scan_next = 0;
  *S.dq.count = 0;
  c.wave += 1;
  int more = (c.live[nxt] > 0 || c.work_next < c.items_total) ? 1 : 0;
  if (more && c.wave >= c.max_waves) {
    c.status = 1;  // out of waves: the host reports UGP_ERR_ITER_LIMIT
    more = 0;
  }
  c.more = more;
  if (!more && c.rays && c.dense_err) {
    atomicAdd(c.rays + 2, c.dense_err);
    c.dense_err = 0ull;
  }
  if (use_graph) cudaGraphSetConditional(handle, unsigned(more));
}

// ------------------------------------------------------------------ workspace
struct BatchLayout {
  size_t ctl, reqs, scenes, done, finish, paths, live0, live1, retire, stack, shadow, dense, lists, total;
};

BatchLayout batch_layout(int max_req, int64_t pool) {
  BatchLayout L;
  size_t off = 0;
  const size_t col = align256(size_t(pool) * 4);
  L.ctl = off;     off += 256;
  L.reqs = off;    off += align256(sizeof(BReq) * size_t(max_req));
  L.scenes = off;  off += align256(sizeof(TraceScene) * size_t(max_req));
  L.done = off;    off += align256(8 * size_t(max_req));
  L.finish = off;  off += align256(8 * size_t(max_req));
  L.paths = off;   off += kPathCols * col;
  L.live0 = off;   off += col;
  L.live1 = off;   off += col;
  L.retire = off;  off += col;
  L.stack = off;   off += col;
  L.shadow = off;  off += 12 * col;
  L.dense = off;   off += dense_queue_bytes(pool);
  L.lists = off;   off += slot_list_bytes(pool);
  L.total = off;
  return L;
}

BState batch_state(char* ws, const BatchLayout& L, int64_t pool) {
  BState S;
  S.pool = pool;
  const size_t col = align256(size_t(pool) * 4);
  auto F = [&](size_t base, int k) { return reinterpret_cast<float*>(ws + base + k * col); };
  auto I = [&](size_t base, int k) { return reinterpret_cast<int*>(ws + base + k * col); };
  S.ctl = reinterpret_cast<BCtl*>(ws + L.ctl);
  S.reqs = reinterpret_cast<const BReq*>(ws + L.reqs);
  S.scenes = reinterpret_cast<const TraceScene*>(ws + L.scenes);
  S.done = reinterpret_cast<unsigned long long*>(ws + L.done);
  S.finish_ns = reinterpret_cast<unsigned long long*>(ws + L.finish);
  PathSoA& ps = S.P.ps;
  ps = PathSoA{F(L.paths, 0), F(L.paths, 1), F(L.paths, 2), F(L.paths, 3), F(L.paths, 4), F(L.paths, 5),
               F(L.paths, 6), F(L.paths, 7), F(L.paths, 8), F(L.paths, 9), F(L.paths, 10), F(L.paths, 11),
               F(L.paths, 12), I(L.paths, 13), I(L.paths, 14), F(L.paths, 15), F(L.paths, 16), I(L.paths, 17),
               F(L.paths, 18), F(L.paths, 19)};
  S.P.tu = F(L.paths, 20);
  S.P.req = I(L.paths, 21);
  S.P.pix = I(L.paths, 22);
  S.P.smp = I(L.paths, 23);
  S.P.bounce = I(L.paths, 24);
  S.live[0] = I(L.live0, 0);
  S.live[1] = I(L.live1, 0);
  S.retire = I(L.retire, 0);
  S.stack = I(L.stack, 0);
  S.sh = ShadowSoA{I(L.shadow, 0), F(L.shadow, 1), F(L.shadow, 2), F(L.shadow, 3), F(L.shadow, 4), F(L.shadow, 5),
                   F(L.shadow, 6), F(L.shadow, 7), I(L.shadow, 8), F(L.shadow, 9), F(L.shadow, 10),
                   F(L.shadow, 11)};
  S.dq = dense_queue_at(ws + L.dense, pool);
  S.dq.list = reinterpret_cast<const int*>(ws + L.lists);
  S.dq.scenes = S.scenes;
  return S;
}

int grid_of(const void* kernel, int block, int64_t n) {
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

// Persistent grid sizes of the wave kernels for a pool (computed before any stream capture).
struct WaveGrids {
  int regen, ext, shade, shadow, retire;
};
WaveGrids wave_grids(int64_t pool) {
  const int ext_need = int((pool + kFFBlock - 1) / kFFBlock), ext_cap = scan_grid((const void*)k_b_extend);
  return WaveGrids{grid_of((const void*)k_b_regen, 256, pool), ext_need < ext_cap ? ext_need : ext_cap,
                   grid_of((const void*)k_b_shade, 128, pool), int((pool + kTrBlock - 1) / kTrBlock),
                   grid_of((const void*)k_b_retire, 256, pool)};
}

// Launches one wave on `st` (also used while capturing the graph body).
ugp_status launch_wave(const BState& S, const WaveGrids& g, cudaGraphConditionalHandle h, int use_graph,
                       cudaStream_t st) {
  k_b_claim<<<1, 32, 0, st>>>(S);
  k_b_regen<<<g.regen, 256, 0, st>>>(S);
  k_b_extend<<<g.ext, kFFBlock, 0, st>>>(S);
  // every queued ray names its scene (S.dq.scenes), so the launch's own scene is unused
  ugp_status s = launch_dense(TraceScene{}, S.dq, 0, &S.ctl->dense_slots, S.pool, S.P.ps.prim, S.P.tu, S.P.ps.tsp,
                              nullptr, 0, nullptr, &S.ctl->dense_err, st);
  if (s != UGP_OK) return s;
  k_b_shade<<<g.shade, 128, 0, st>>>(S);
  k_b_shadow<<<g.shadow, kTrBlock, 0, st>>>(S);
  k_b_retire<<<g.retire, 256, 0, st>>>(S);
  k_b_cond<<<1, 32, 0, st>>>(S, h, use_graph);
  UGP_CUDA_CHECK(cudaGetLastError());
  return UGP_OK;
}
constexpr int kWaveKernels = 9;  // claim, regen, extend, the two finish passes, shade, shadow, retire, cond

// Instantiated graphs: one per (workspace, pool, device); the body reads everything else from
// the workspace, so a graph serves every batch that fits its workspace.
struct GraphEntry {
  const void* ws;
  int64_t pool;
  int max_req;
  int device;
  cudaGraphExec_t exec;
  cudaGraph_t graph;
};
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;

ugp_status get_graph(const BState& S, const void* ws, int64_t pool, int max_req, cudaGraphExec_t* out) {
  int dev = 0;
  UGP_CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (const GraphEntry& e : g_graphs)
    if (e.ws == ws && e.pool == pool && e.max_req == max_req && e.device == dev) {
      *out = e.exec;
      return UGP_OK;
    }
  static cudaStream_t cap_stream[64] = {};
  if (dev < 0 || dev >= 64) return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: device index out of range");
  if (!cap_stream[dev]) UGP_CUDA_CHECK(cudaStreamCreateWithFlags(&cap_stream[dev], cudaStreamNonBlocking));
  {
    const ugp_status ds = dense_prepare();
    if (ds != UGP_OK) return ds;
  }
  const WaveGrids wg = wave_grids(pool);
  cudaGraph_t g = nullptr;
  UGP_CUDA_CHECK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  UGP_CUDA_CHECK(cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  UGP_CUDA_CHECK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  prof_suspend(true);
  cudaError_t e = cudaStreamBeginCaptureToGraph(cap_stream[dev], body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal);
  ugp_status s = UGP_OK;
  if (e == cudaSuccess) {
    s = launch_wave(S, wg, h, 1, cap_stream[dev]);
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap_stream[dev], &captured);
    if (e2 != cudaSuccess && s == UGP_OK) s = cuda_fail(e2, "cudaStreamEndCapture");
  } else {
    s = cuda_fail(e, "cudaStreamBeginCaptureToGraph");
  }
  prof_suspend(false);
  if (s != UGP_OK) {
    cudaGraphDestroy(g);
    return s;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  g_graphs.push_back({ws, pool, max_req, dev, ex, g});
  *out = ex;
  return UGP_OK;
}

}  // namespace
}  // namespace ugp

using namespace ugp;

extern "C" size_t ugp_render_batch_workspace_size(int32_t max_requests, const ugp_batch_config* cfg) {
  if (!cfg || max_requests <= 0 || cfg->pool_log2 < 10 || cfg->pool_log2 > 24) return 0;
  return batch_layout(max_requests, int64_t(1) << cfg->pool_log2).total;
}

extern "C" ugp_status ugp_render_batch(int32_t n_req, const ugp_request* reqs, const ugp_batch_config* cfg,
                                       int32_t max_requests, void* workspace, size_t workspace_bytes,
                                       double* latency_ms_out, unsigned long long* ray_counts, void* stream_) {
  clear_error();
  if (!cfg) return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: NULL config");
  if (cfg->tile != 8 && cfg->tile != 16 && cfg->tile != 32)
    return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: tile must be 8, 16 or 32");
  if (cfg->pool_log2 < 10 || cfg->pool_log2 > 24)
    return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: pool_log2 must be in [10, 24]");
  if (n_req < 0 || n_req > max_requests) return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: bad request count");
  if (n_req > 0 && !reqs) return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: NULL request array");
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: workspace must be non-NULL and 256-byte aligned");
  const int64_t pool = int64_t(1) << cfg->pool_log2;
  const int T = cfg->tile, TP = T * T;
  const BatchLayout BL = batch_layout(max_requests, pool);
  if (workspace_bytes < BL.total)
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_render_batch: need %zu bytes, got %zu", BL.total, workspace_bytes);
  if (pool < TP) return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: pool smaller than one tile");
  cudaStream_t st = static_cast<cudaStream_t>(stream_);

  if (cfg->order != 0 && cfg->order != 1) return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: order must be 0 or 1");
  // service order: as given, or shortest first by the work estimate pixels x spp x (depth + 1)
  std::vector<int> order(size_t(n_req > 0 ? n_req : 0));
  for (int r = 0; r < n_req; ++r) order[size_t(r)] = r;
  if (cfg->order == 1) {
    auto work = [&](int r) {
      const ugp_request& q = reqs[r];
      return double(q.camera.width) * double(q.camera.height) * double(q.spp > 0 ? q.spp : 0) *
             double(q.max_depth + 1);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) < work(b); });
  }
  // host request table, in service order
  std::vector<BReq> hr(size_t(n_req > 0 ? n_req : 1));
  std::vector<TraceScene> hs(size_t(n_req > 0 ? n_req : 1));
  long long items = 0, max_depth = 0;
  for (int slot = 0; slot < n_req; ++slot) {
    const int r = order[size_t(slot)];
    const ugp_request& q = reqs[r];
    if (!valid_bvh(q.bvh)) return fail(UGP_ERR_NOT_BUILT, "ugp_render_batch: request %d: invalid BVH handle", r);
    if (!q.materials || !q.accum_rgb || !q.accum_sq_rgb)
      return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: request %d: NULL materials or accumulator", r);
    const ugp_materials& m = *q.materials;
    if (q.bvh->n_prims > 0 && (!m.sggx6 || !m.type || !m.albedo3 || !m.roughness || !m.emission3))
      return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: request %d: NULL material array", r);
    const int W = q.camera.width, H = q.camera.height;
    if (W <= 0 || H <= 0 || int64_t(W) * H > (int64_t(1) << 31) - 1)
      return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: request %d: bad image size", r);
    if (q.spp < 0 || q.max_depth < 0 || q.max_depth > 14)
      return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: request %d: spp >= 0 and max_depth in [0, 14]", r);
    if (!(q.camera.vfov_deg > 0.f && q.camera.vfov_deg < 180.f))
      return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch: request %d: vfov_deg must be in (0, 180)", r);
    BReq& b = hr[size_t(slot)];
    b.md = MatDev{m.sggx6, m.type, m.albedo3, m.roughness, m.emission3, m.disney9};
    b.L = lights_dev(&q.lights);
    const ugp_status cs = camera_dev(&q.camera, "ugp_render_batch", &b.cam);
    if (cs != UGP_OK) return cs;
    b.key = make_uint2(uint32_t(q.seed & 0xffffffffu), uint32_t(q.seed >> 32));
    b.spp = q.spp;
    b.depth = q.max_depth;
    b.nee = q.nee;
    b.spawn = q.spawn_mode;
    b.tiles_x = (W + T - 1) / T;
    b.n_tiles = b.tiles_x * ((H + T - 1) / T);
    b.item_begin = items;
    b.items = (long long)b.n_tiles * q.spp;
    b.paths = (long long)W * H * q.spp;
    b.acc = q.accum_rgb;
    b.acc2 = q.accum_sq_rgb;
    items += b.items;
    if (q.max_depth > max_depth) max_depth = q.max_depth;
    hs[size_t(slot)] = trace_scene(q.bvh);
  }
  // Bound on waves: every item is claimed within items / (pool / TP) + 1 claims, a claim per
  // wave at least once the pool drains, and a path lives at most max_depth + 1 waves.
  const long long per_wave = pool / TP;
  const long long bound = (items / per_wave + 2) * (max_depth + 2) + 16;
  const int max_waves = int(bound < (1 << 30) ? bound : (1 << 30));

  char* ws = static_cast<char*>(workspace);
  const BState S = batch_state(ws, BL, pool);
  if (n_req > 0) {
    UGP_CUDA_CHECK(cudaMemcpyAsync(ws + BL.reqs, hr.data(), sizeof(BReq) * size_t(n_req), cudaMemcpyHostToDevice, st));
    UGP_CUDA_CHECK(cudaMemcpyAsync(ws + BL.scenes, hs.data(), sizeof(TraceScene) * size_t(n_req),
                                   cudaMemcpyHostToDevice, st));
  }
  prof_begin(kStBatch, st);
  k_b_init<<<grid_of((const void*)k_b_init, 256, pool), 256, 0, st>>>(S, n_req, (unsigned long long)items, T, int(pool),
                                                                       max_waves, ray_counts);
  prof_end(kStBatch, st);
  UGP_CUDA_CHECK(cudaGetLastError());
  int waves_run = 0;
  if (items > 0) {
    if (cfg->use_graph) {
      cudaGraphExec_t ex = nullptr;
      ugp_status s = get_graph(S, workspace, pool, max_requests, &ex);
      if (s != UGP_OK) return s;
      prof_begin(kStBatch, st);
      UGP_CUDA_CHECK(cudaGraphLaunch(ex, st));
      prof_end(kStBatch, st, 0);
    } else {
      // host loop: waves in chunks, polling the device flag between chunks (a wave after the
      // last one finds no work and changes nothing)
      BCtl hc{};
      prof_begin(kStBatch, st);
      prof_suspend(true);
      ugp_status s = dense_prepare();
      const WaveGrids wg = wave_grids(pool);
      for (; s == UGP_OK;) {
        for (int w = 0; w < 8 && s == UGP_OK; ++w) s = launch_wave(S, wg, cudaGraphConditionalHandle{}, 0, st);
        if (s != UGP_OK) break;
        const cudaError_t e1 = cudaMemcpyAsync(&hc, S.ctl, sizeof(BCtl), cudaMemcpyDeviceToHost, st);
        const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamSynchronize(st) : e1;
        if (e2 != cudaSuccess) {
          s = cuda_fail(e2, "ugp_render_batch: polling the wave flag");
          break;
        }
        if (!hc.more) break;
      }
      prof_suspend(false);
      prof_end(kStBatch, st, 0);
      if (s != UGP_OK) return s;
    }
  }
  // results: status, waves and, when asked, per-request latencies (synchronises)
  BCtl hc{};
  UGP_CUDA_CHECK(cudaMemcpyAsync(&hc, S.ctl, sizeof(BCtl), cudaMemcpyDeviceToHost, st));
  std::vector<unsigned long long> fin(size_t(n_req > 0 ? n_req : 1));
  if (latency_ms_out && n_req > 0)
    UGP_CUDA_CHECK(cudaMemcpyAsync(fin.data(), S.finish_ns, 8 * size_t(n_req), cudaMemcpyDeviceToHost, st));
  UGP_CUDA_CHECK(cudaStreamSynchronize(st));
  waves_run = hc.wave;
  if (items > 0) add_launches(kStBatch, int64_t(cfg->use_graph ? waves_run : ((waves_run + 7) / 8) * 8) * kWaveKernels);
  if (latency_ms_out)
    for (int slot = 0; slot < n_req; ++slot) {
      const int r = order[size_t(slot)];
      const unsigned long long f = fin[size_t(slot)];
      latency_ms_out[r] = hr[size_t(slot)].paths == 0 ? 0.0 : (f > hc.start_ns ? 1e-6 * double(f - hc.start_ns) : -1.0);
    }
  if (hc.status != 0)
    return fail(UGP_ERR_ITER_LIMIT, "ugp_render_batch: stopped after %d waves with work left", waves_run);
  return UGP_OK;
}

namespace ugp {
namespace {

struct TuneEntry {
  int device, n_req, max_depth;
  long long probe_paths;
  ugp_batch_config best;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;

}  // namespace
}  // namespace ugp

extern "C" ugp_status ugp_render_batch_autotune(int32_t n_req, const ugp_request* reqs, int32_t probe_spp,
                                                int32_t pool_log2_min, int32_t pool_log2_max, int32_t use_graph,
                                                void* workspace, size_t workspace_bytes, float* scratch,
                                                size_t scratch_floats, ugp_batch_config* best_out, double* ms_out,
                                                void* stream_) {
  clear_error();
  if (!best_out || n_req <= 0 || !reqs || probe_spp <= 0 || pool_log2_min < 10 || pool_log2_max > 24 ||
      pool_log2_min > pool_log2_max || !scratch)
    return fail(UGP_ERR_INVALID_ARG, "ugp_render_batch_autotune: bad argument");
  // the probe: every request at min(spp, probe_spp) samples, accumulating into the scratch
  std::vector<ugp_request> probe(reqs, reqs + n_req);
  size_t need = 0;
  long long paths = 0;
  int max_depth = 0;
  for (ugp_request& q : probe) {
    const size_t px = size_t(q.camera.width > 0 ? q.camera.width : 0) * size_t(q.camera.height > 0 ? q.camera.height : 0);
    if (2 * 3 * px > need) need = 2 * 3 * px;
    if (q.spp > probe_spp) q.spp = probe_spp;
    paths += (long long)px * q.spp;
    if (q.max_depth > max_depth) max_depth = q.max_depth;
    q.accum_rgb = scratch;
    q.accum_sq_rgb = scratch + 3 * px;
  }
  if (scratch_floats < need)
    return fail(UGP_ERR_WORKSPACE_TOO_SMALL, "ugp_render_batch_autotune: scratch needs %zu floats", need);
  int dev = 0;
  UGP_CUDA_CHECK(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneEntry& e : g_tune)
      if (e.device == dev && e.n_req == n_req && e.max_depth == max_depth && e.probe_paths == paths &&
          e.best.pool_log2 >= pool_log2_min && e.best.pool_log2 <= pool_log2_max && e.best.use_graph == use_graph &&
          !ms_out) {
        *best_out = e.best;
        return UGP_OK;
      }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  cudaEvent_t e0, e1;
  UGP_CUDA_CHECK(cudaEventCreate(&e0));
  UGP_CUDA_CHECK(cudaEventCreate(&e1));
  const int tiles[3] = {8, 16, 32};
  double best_ms = 1e300;
  ugp_batch_config best{16, pool_log2_min, use_graph, 1};
  int k = 0;
  ugp_status s = UGP_OK;
  for (int lg = pool_log2_min; lg <= pool_log2_max && s == UGP_OK; ++lg) {
    for (int ti = 0; ti < 3 && s == UGP_OK; ++ti, ++k) {
      const ugp_batch_config cfg{tiles[ti], lg, use_graph, 1};
      if ((int64_t(1) << lg) < int64_t(tiles[ti]) * tiles[ti] ||
          workspace_bytes < ugp_render_batch_workspace_size(n_req, &cfg)) {
        if (ms_out) ms_out[k] = -1.0;
        continue;
      }
      // first run builds the graph for this pool size; the second is timed
      s = ugp_render_batch(n_req, probe.data(), &cfg, n_req, workspace, workspace_bytes, nullptr, nullptr, st);
      if (s != UGP_OK) break;
      cudaEventRecord(e0, st);
      s = ugp_render_batch(n_req, probe.data(), &cfg, n_req, workspace, workspace_bytes, nullptr, nullptr, st);
      cudaEventRecord(e1, st);
      if (s != UGP_OK) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms_out) ms_out[k] = ms;
      if (ms < best_ms) {
        best_ms = ms;
        best = cfg;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != UGP_OK) return s;
  *best_out = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.push_back({dev, n_req, max_depth, paths, best});
  return UGP_OK;
}
