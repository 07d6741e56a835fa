/*
 * ugp.h -- C ABI of the GB300 (sm_103a) Gaussian-primitive ray tracer.
 *
 * Implements the scene queries of "Unified Gaussian Primitives for Scene
 * Representation and Rendering" (Zhou, Wu, Yan; arXiv 2406.09733):
 * primitives are scaled anisotropic 3D Gaussians (Eq. 1, Eq. 2) truncated to
 * their k-sigma bounding ellipsoid (Eq. 4); light is attenuated by the linear
 * transmittance of Eq. 7 and scattered by whole primitives sampled from the
 * free-flight distribution of Eq. 8 (Sec. 5.2).
 *
 * Conventions shared by every entry point
 *  - Pointers are DEVICE pointers unless a comment says "host".  The caller
 *    owns all memory; the library never allocates device memory.  Arrays are
 *    dense, C-contiguous, structure-of-arrays: a "float3 array" of n elements
 *    is 3*n floats (x0,y0,z0,x1,...).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work is enqueued on it and the call returns without
 *    waiting, except where noted.  Argument errors are detected on the host
 *    before any launch and reported synchronously.
 *  - Rays are x_t = o + t d for t in [t0, t1]; d must be non-zero.  With a
 *    unit d, t is Euclidean distance.
 *  - Primitive indices in inputs and outputs are the caller's original
 *    indices (0 .. n_prims-1), never the internal leaf order.
 *  - Functions return a ugp_status; ugp_last_error() gives a thread-local
 *    message for the most recent failure on the calling thread.  No C++
 *    exception crosses this boundary.
 *  - Device loops are bounded.  A ray whose traversal hits a bound gets a
 *    non-zero per-ray status code (UGP_RAY_*) in status_out; the call itself
 *    still returns UGP_OK.
 */
#ifndef UGP_H_
#define UGP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ugp_status {
  UGP_OK = 0,
  UGP_ERR_INVALID_ARG = 1,          /* a pointer, size or value is out of range */
  UGP_ERR_WORKSPACE_TOO_SMALL = 2,  /* workspace_bytes < the *_workspace_size() query */
  UGP_ERR_CUDA = 3,                 /* a CUDA runtime call failed (see ugp_last_error) */
  UGP_ERR_ITER_LIMIT = 4,           /* reported by ugp_status_of_rays: some ray hit a loop bound */
  UGP_ERR_TIMEOUT = 5,              /* a bounded device wait gave up */
  UGP_ERR_NOT_BUILT = 6,            /* a NULL or released BVH handle */
  UGP_ERR_OVERFLOW = 7              /* reported by ugp_status_of_rays: a stack or buffer overflowed */
} ugp_status;

/* Per-ray status codes (uint8) written by the tracing entry points. */
enum {
  UGP_RAY_OK = 0,
  UGP_RAY_STACK_OVERFLOW = 1,   /* traversal stack full: result incomplete */
  UGP_RAY_BUFFER_OVERFLOW = 2,  /* reserved (the free-flight buffer falls back to binning) */
  UGP_RAY_ITER_LIMIT = 3,       /* free flight: collection-round bound reached */
  UGP_RAY_BAD_NODE = 4,         /* a node or leaf reference out of range (corrupt BVH) */
  UGP_RAY_SOLVE_LIMIT = 5       /* free flight: root solve did not converge in its bound */
};

/* Input primitives (Sec. 3.1, Eq. 1-2), device float32 arrays of n rows:
 *   mean3      mu              (n x 3)
 *   quat4      rotation R as a unit quaternion (w, x, y, z)   (n x 4); it is
 *              normalised by the library
 *   scale3     diagonal of S, all > 0                          (n x 3)
 *   magnitude  c of Eq. 1, >= 0                                (n)          */
typedef struct ugp_prims {
  int64_t n;
  const float* mean3;
  const float* quat4;
  const float* scale3;
  const float* magnitude;
} ugp_prims;

/* Opaque BVH handle.  The handle is a small host object; every array it
 * refers to lives in the caller's workspace, which must stay allocated and
 * unmodified for as long as the handle is used. */
typedef struct ugp_bvh ugp_bvh;

typedef struct ugp_bvh_info {
  int64_t n_prims;
  int64_t n_nodes;        /* internal binary nodes */
  float cutoff_k;         /* sqrt(-2 ln eps) of Eq. 4 */
  float bounds_lo[3];     /* bounds of all bounding boxes */
  float bounds_hi[3];
  size_t persistent_bytes;/* workspace bytes the built BVH keeps using */
  int64_t n_invalid;      /* primitives ignored as invalid (see ugp_build_bvh) */
} ugp_bvh_info;

/* Bytes of device workspace ugp_build_bvh needs for n_prims primitives
 * (the BVH itself plus build temporaries).  Needs a current CUDA device;
 * returns 0 if n_prims < 0 or the query fails. */
size_t ugp_build_bvh_workspace_size(int64_t n_prims);

/* Builds the acceleration structure over the primitives' bounding ellipsoids
 * (Eq. 4 with threshold cutoff_eps, in (0, 1); the paper uses 0.01).
 * Per primitive it precomputes the whitening matrix W = S^-1 R^T, so that
 * (RS)^-1 (x - mu) = W (x - mu), the normaliser g0 = c / ((2 pi)^{3/2} s_x s_y s_z)
 * of Eq. 1, and the bounding box of the k-ellipsoid.  The structure is a
 * binary BVH (the paper uses a kd-tree, Sec. 5.1; the exact order-free
 * sampling of ugp_sample_free_flight does not need non-overlapping nodes).
 *   prims       host pointer to the device SoA description above
 *   workspace   device buffer of at least ugp_build_bvh_workspace_size(n)
 *               bytes, 256-byte aligned; holds the BVH after the call
 *   out         host pointer; receives a new handle (free with ugp_bvh_release)
 * The call enqueues the build on `stream` and returns; the handle is usable
 * by later work on the same stream.  n_prims == 0 is allowed (every ray
 * escapes).  A primitive with a non-finite mean, a zero or non-finite
 * quaternion, a scale that is not finite and positive, or a magnitude that is
 * negative or not finite is ignored by every query (it is never hit); the
 * count is reported by ugp_bvh_get_info. */
ugp_status ugp_build_bvh(const ugp_prims* prims, float cutoff_eps, void* workspace,
                         size_t workspace_bytes, void* stream, ugp_bvh** out);

/* Frees the host handle (the workspace stays the caller's). NULL is ignored. */
void ugp_bvh_release(ugp_bvh* bvh);

/* Fills *out (host).  Synchronous: waits for the build stream, then copies
 * the scene bounds and the invalid-primitive count from the workspace. */
ugp_status ugp_bvh_get_info(const ugp_bvh* bvh, ugp_bvh_info* out);

/* Transmittance evaluation (Sec. 5.3, Eq. 7): for each ray r,
 *   T_out[r] = max(0, 1 - 1/2 sum_k I_k(max(t0, t_k-), min(t1, t_k+)))
 * where I_k is the closed-form ray integral of App. A over primitive k's
 * clipped bounding-ellipsoid interval.  Order-free; traversal stops once the
 * sum reaches 1 (T = 0).  Russian roulette is not applied (exact T).
 *   o3, d3        float3 arrays (n_rays)
 *   t0, t1        float arrays (n_rays), t0 <= t1
 *   exclude_prim  int32 array (n_rays) or NULL: primitive skipped by that
 *                 ray (the scattering primitive of Sec. 6), -1 for none
 *   T_out         float array (n_rays)
 *   status_out    uint8 array (n_rays) or NULL
 * n_rays == 0 is allowed. */
ugp_status ugp_trace_transmittance(const ugp_bvh* bvh, int64_t n_rays, const float* o3,
                                   const float* d3, const float* t0, const float* t1,
                                   const int32_t* exclude_prim, float* T_out,
                                   uint8_t* status_out, void* stream);

/* Free-flight distribution sampling (Sec. 5.2, Eq. 8-10), exact and
 * independent of traversal order.  With F(t) = 1/2 sum_k I_k(a_k, min(t, b_k))
 * over the clipped intervals [a_k, b_k]:
 *  - if F(t1) <= u the ray escapes: prim_out = -1, t_u_out = t1,
 *    t_spawn_out = t1;
 *  - otherwise t_u solves F(t_u) = u, and the primitive is drawn among those
 *    whose interval contains t_u with probability G_k(x_{t_u}) / sum_j G_j(x_{t_u})
 *    by an exponential race: candidate k gets E_k = -ln U_k, U_k = ((x0 >> 8) + 1) / 2^24
 *    where x = Philox4x32-10(counter (k, 0, 0, 0), key (bit pattern of u2, 0x2406C0DE)),
 *    and the smallest E_k / G_k(x_{t_u}) wins (ties: smaller index).
 *    t_spawn_out is the centre of the chosen primitive's clipped interval,
 *    where the paper spawns the scattered ray (Sec. 6).
 * The chosen primitive k has probability 1/2 I_k(a_k, min(b_k, t_sat)), the
 * saturating-distance clamp of Eq. 8.
 *   u, u2         float arrays (n_rays) of uniforms in [0, 1)
 *   prim_out      int32 array (n_rays); t_u_out, t_spawn_out float arrays
 *   workspace     device scratch of ugp_sample_free_flight_workspace_size(n_rays)
 *                 bytes (see below)
 *   other arguments as for ugp_trace_transmittance. */
ugp_status ugp_sample_free_flight(const ugp_bvh* bvh, int64_t n_rays, const float* o3,
                                  const float* d3, const float* t0, const float* t1,
                                  const float* u, const float* u2, const int32_t* exclude_prim,
                                  int32_t* prim_out, float* t_u_out, float* t_spawn_out,
                                  uint8_t* status_out, void* workspace, size_t workspace_bytes,
                                  void* stream);

/* Scratch bytes ugp_sample_free_flight needs for n_rays rays: the table of rays whose root
 * the first pass has bracketed (they are finished by the passes that follow it), the lists of
 * rays handed between those passes, and per ray a list of up to 256 primitive slots met by
 * the first pass (1100 bytes per ray in all), plus one 73,728-byte interval slot of the last
 * pass per 64 rays (4 to 2432 of them) and alignment.  The workspace must be 256-byte aligned
 * and is only used during the call's device work. */
size_t ugp_sample_free_flight_workspace_size(int64_t n_rays);

/* Free-flight sampling without any device allocation (no counterpart in the paper).
 * Same inputs, outputs and results as ugp_sample_free_flight, for callers that cannot
 * call cudaMalloc or hand the library a workspace -- for example code that runs while a
 * host application owns every device allocation, or a real-time loop that must not
 * touch the allocator.  The scratch queue lives in a fixed array of device memory inside
 * the library image, sized for UGP_NOALLOC_MAX_RAYS rays (about 9.7 MB); every GPU that
 * loads the library holds it until the process exits.  Without the per-ray slot lists of
 * the regular entry point, its warp pass finds dense intervals by traversal; the results
 * are the same.
 *  - n_rays above UGP_NOALLOC_MAX_RAYS is rejected with UGP_ERR_INVALID_ARG.
 *  - The first call on a device looks up the array's device address with that device
 *    current (cudaGetSymbolAddress); make that first call before any stream capture.
 *    The address is kept for the life of the process and is not valid after
 *    cudaDeviceReset of that device: do not call this entry point on a device that the
 *    process has reset.
 *  - Every call uses the same array and leaves its contents behind; the call clears the
 *    part that must start at zero on `stream`.  Calls whose device work overlaps (on
 *    different streams, or from several host threads) race on the array and must be
 *    serialised by the caller.
 *  - No cudaMalloc, cudaFree or allocating library routine is called. */
#define UGP_NOALLOC_MAX_RAYS 65536
ugp_status ugp_sample_free_flight_noalloc(const ugp_bvh* bvh, int64_t n_rays, const float* o3,
                                          const float* d3, const float* t0, const float* t1,
                                          const float* u, const float* u2,
                                          const int32_t* exclude_prim, int32_t* prim_out,
                                          float* t_u_out, float* t_spawn_out, uint8_t* status_out,
                                          void* stream);

/* Phase-function queries (Sec. 6: Eq. 12 with the SGGX visible normals of Eq. 11 and the
 * base BSDF; App. B for the pdf), for element-wise checks of the shading code.  Record i
 * has its own material (type 0, 1 or 3 as in ugp_materials; albedo3, roughness and sggx6
 * as there; disney9 (n x 9) may be NULL, then zeros) and unit directions wo3, wi3 (n x 3,
 * pointing away from the scattering point).  Outputs, per record:
 *   eval3_out           the phase function f_p(wi, wo) (Eq. 12): the closed form for
 *                       isotropic flakes with a Lambertian base, else the stochastic
 *                       estimate from the six uniforms u_eval6[6 i ..] (n x 6)
 *   pdf_out             the approximate pdf of App. B at wi
 *   sample_wi3_out      a direction sampled from wo with the four uniforms u_sample4
 *   sample_weight3_out  its weight f_p / pdf (zero when sample_ok_out[i] is 0)
 *   sample_ok_out       1 if the sample carries weight (uint8)
 * Uniforms lie in [0, 1).  All arrays are device arrays.  Errors: n < 0, or a NULL array
 * other than disney9, UGP_ERR_INVALID_ARG.  Asynchronous on `stream`. */
ugp_status ugp_phase_query(int64_t n, const uint8_t* type, const float* albedo3, const float* roughness,
                           const float* sggx6, const float* disney9, const float* wo3, const float* wi3,
                           const float* u_eval6, const float* u_sample4, float* eval3_out, float* pdf_out,
                           float* sample_wi3_out, float* sample_weight3_out, uint8_t* sample_ok_out,
                           void* stream);

/* The paper's own free-flight sampler (Sec. 5.1-5.2), a comparison variant of
 * ugp_sample_free_flight over an SAH kd-tree: front-to-back traversal, the CDF accumulated
 * primitive by primitive in each leaf's order, and in a leaf where the CDF reaches 1 the
 * paper's GPU partition of the ray-node interval into 8 equal bins, each classified again, with
 * the disambiguation of Eq. 10 in the bin where it reaches 1 (t_u solved in the bin, the
 * primitive drawn proportionally to I_k(bin start, t_u) among the intervals overlapping the
 * bin, using u2).  The rule depends on the tree and is biased where several primitives straddle
 * the saturating distance; ugp_sample_free_flight is exact.
 *
 * ugp_build_kdtree builds the tree on the device over the k-ellipsoid boxes of a built BVH's
 * primitives (binned surface-area heuristic, 8 planes per axis, traversal cost 1, intersection
 * cost 1.5; primitives straddling a plane go to both sides; at most 28 levels; leaves list
 * their primitives in ascending order).  It reads two counts per level back to the host, so it
 * returns after the build has finished on `stream`.  Workspace:
 * ugp_build_kdtree_workspace_size(n) bytes (256-byte aligned); the tree lives in its first part
 * and uses the BVH's records, so both must outlive the handle.  Errors: an invalid BVH,
 * UGP_ERR_NOT_BUILT; NULL or misaligned workspace, UGP_ERR_INVALID_ARG; more than 4 n
 * primitive references, UGP_ERR_WORKSPACE_TOO_SMALL.
 * ugp_kdtree_get_info: nodes, references, depth and root box (each output may be NULL).
 * ugp_kdtree_export copies the nodes (n_nodes x 4 int32 host array: interior (axis, plane as
 * float bits, left, right), leaf (3, count, first reference, 0)) and the references (n_refs
 * int32, as the caller's primitive indices) to host memory; synchronous.
 * ugp_sample_free_flight_kdtree: arguments as for ugp_sample_free_flight, without t_u and
 * workspace; t_spawn_out (may be NULL) receives the centre of the chosen primitive's clipped
 * interval.  Asynchronous on `stream`. */
typedef struct ugp_kdtree ugp_kdtree;
size_t ugp_build_kdtree_workspace_size(int64_t n_prims);
ugp_status ugp_build_kdtree(const ugp_bvh* bvh, void* workspace, size_t workspace_bytes, void* stream,
                            ugp_kdtree** out);
void ugp_kdtree_release(ugp_kdtree* kd);
ugp_status ugp_kdtree_get_info(const ugp_kdtree* kd, int64_t* n_nodes, int64_t* n_refs, int32_t* depth,
                               float* box6);
ugp_status ugp_kdtree_export(const ugp_kdtree* kd, int32_t* nodes4_host, int32_t* refs_host);
ugp_status ugp_sample_free_flight_kdtree(const ugp_kdtree* kd, int64_t n_rays, const float* o3, const float* d3,
                                         const float* t0, const float* t1, const float* u, const float* u2,
                                         const int32_t* exclude_prim, int32_t* prim_out, float* t_spawn_out,
                                         uint8_t* status_out, void* stream);

/* All clipped intervals along each ray (hit-set diagnostics).  For ray r,
 * count_out[r] receives the number of primitives whose k-ellipsoid interval
 * meets [t0, t1] (Eq. 4 cut-off, the same test as the queries above); the
 * first min(count, cap) of them, in traversal order, are written to
 * ids_out[r*cap + j], a_out[r*cap + j], b_out[r*cap + j] (the clipped
 * interval [a, b]).
 *   cap         >= 0; ids_out, a_out, b_out hold n_rays*cap elements (may be
 *               NULL when cap == 0)
 *   count_out   int32 array (n_rays)
 *   other arguments as for ugp_trace_transmittance. */
ugp_status ugp_collect_hits(const ugp_bvh* bvh, int64_t n_rays, const float* o3, const float* d3,
                            const float* t0, const float* t1, const int32_t* exclude_prim,
                            int32_t cap, int32_t* ids_out, float* a_out, float* b_out,
                            int32_t* count_out, uint8_t* status_out, void* stream);

/* Radiance-field forward render (Sec. 7, Eq. rf): the primitives as an emitting,
 * non-scattering medium, rendered deterministically.  For ray r, with F the free-flight CDF
 * of Eq. 8 over [t0, t1] and t_sat its root at 1 (the saturating distance; t_sat = t1 when
 * F(t1) <= 1):
 *   rgb_out[3r + c] = sum_k 1/2 I_k(a_k, min(b_k, t_sat)) emission3[3k + c]
 *                     + (F(t1) <= 1 ? 1 - F(t1) : 0) background3[c]
 * summed over the primitives whose clipped interval [a_k, b_k] meets [t0, t_sat].
 *   emission3    device float array (n_prims x 3), indexed by the caller's primitive index
 *   background3  HOST pointer to 3 floats, or NULL for black
 *   rgb_out      device float array (n_rays x 3)
 *   status_out   device uint8 array (n_rays) or NULL: the free-flight pass's status, else
 *                the traversal's (UGP_RAY_*)
 *   workspace    device scratch of ugp_render_radiance_field_workspace_size(n_rays) bytes,
 *                256-byte aligned
 *   other arguments as for ugp_trace_transmittance (rays are not clipped at an excluded
 *   primitive here).
 * Asynchronous on `stream`.  Errors: UGP_ERR_NOT_BUILT for an invalid handle;
 * UGP_ERR_INVALID_ARG for a NULL array, a misaligned workspace or n_rays outside
 * [0, 2^31 - 1]; UGP_ERR_WORKSPACE_TOO_SMALL. */
size_t ugp_render_radiance_field_workspace_size(int64_t n_rays);
ugp_status ugp_render_radiance_field(const ugp_bvh* bvh, int64_t n_rays, const float* o3, const float* d3,
                                     const float* t0, const float* t1, const float* emission3,
                                     const float* background3, float* rgb_out, uint8_t* status_out,
                                     void* workspace, size_t workspace_bytes, void* stream);

/* Exponential-transmittance variant (appendix "Sampling Exponential Transmittance Gaussians
 * via Analog Decomposition Tracking").  The primitives are read as the extinction coefficient
 * sigma_t(x) = sum_k G_k(x) of the classical exponential model (Eq. exp_ff) instead of the
 * linear model of Eq. 7, each contribution clipped to its k-ellipsoid as in Sec. 4.1.
 *
 * ugp_sample_free_flight_exponential: analog decomposition tracking.  Every primitive k whose
 * clipped interval [a_k, b_k] meets [t0, t1] draws a collision depth E_k = -ln U_k, with U_k =
 * ((x0 >> 8) + 1) / 2^24 and x0 the first word of Philox4x32-10 under key (bits of u[r],
 * 0x2406DEC0) and counter (k, 0, 0, 0).  If E_k < I_k(a_k, b_k) it collides at t_k with
 * I_k(a_k, t_k) = E_k; the nearest collision is the sample (equal distances: the lower index).
 *   u          device float array (n_rays): the ray's uniform in [0, 1) (keys the E_k)
 *   prim_out   device int32 array (n_rays): the colliding primitive, -1 if none collides
 *   t_out      device float array (n_rays): its collision distance, t1 on escape
 *   status_out device uint8 array (n_rays) or NULL: UGP_RAY_OK, UGP_RAY_STACK_OVERFLOW or
 *              UGP_RAY_BAD_NODE
 *   other arguments as for ugp_trace_transmittance.  Escape has probability
 *   exp(-sum_k I_k(a_k, b_k)).
 *
 * ugp_trace_transmittance_exponential: T_out[r] = exp(-sum_k I_k(a_k, b_k)) over [t0, t1]
 * (0 once the sum passes 112, where float32 exp underflows); arguments as for
 * ugp_trace_transmittance.
 *
 * Both: one thread per ray, no workspace, asynchronous on `stream`.  Errors: UGP_ERR_NOT_BUILT
 * for an invalid handle; UGP_ERR_INVALID_ARG for a NULL array or n_rays outside
 * [0, (2^31 - 1) * 128]. */
ugp_status ugp_sample_free_flight_exponential(const ugp_bvh* bvh, int64_t n_rays, const float* o3, const float* d3,
                                              const float* t0, const float* t1, const float* u,
                                              const int32_t* exclude_prim, int32_t* prim_out, float* t_out,
                                              uint8_t* status_out, void* stream);
ugp_status ugp_trace_transmittance_exponential(const ugp_bvh* bvh, int64_t n_rays, const float* o3,
                                               const float* d3, const float* t0, const float* t1,
                                               const int32_t* exclude_prim, float* T_out, uint8_t* status_out,
                                               void* stream);

/* ------------------------------------------------------------------ rendering
 * Per-primitive appearance (Sec. 6), device arrays in the caller's order:
 *   sggx6      SGGX matrix S (Sxx, Syy, Szz, Sxy, Sxz, Syz), positive definite (n x 6)
 *   type       0 Lambertian base, 1 GGX base, 2 emissive (pure emitter),
 *              3 Disney principled base (Sec. 6, 12 parameters)             (n, uint8)
 *   albedo3    Lambertian rho, the GGX base's Schlick F0, or the Disney base
 *              colour                                                        (n x 3)
 *   roughness  GGX alpha in (0, 1]                                          (n)
 *   emission3  radiance of emissive primitives (isotropic)                  (n x 3)
 *   disney9    Disney parameters of type-3 primitives, each in [0, 1]: metallic,
 *              subsurface, specular, specular tint, roughness, sheen, sheen tint,
 *              clearcoat, clearcoat gloss (n x 9); read only for type 3.  May be
 *              NULL: type-3 primitives then take the published defaults (0, 0, 0.5,
 *              0, 0.5, 0, 0.5, 0, 1). */
typedef struct ugp_materials {
  const float* sggx6;
  const uint8_t* type;
  const float* albedo3;
  const float* roughness;
  const float* emission3;
  const float* disney9;
} ugp_materials;

/* Codebook-quantised primitive records (the random-access compression the paper combines
 * with its level-of-detail scheme).  A record is 24 bytes: the mean (3 float) and magnitude
 * (float) exact, then 16-bit codes of four attribute groups, each the index of the nearest of
 * 4096 entries of its codebook: scale (as log s, 3 values), rotation (unit quaternion with
 * w >= 0, 4), SGGX (6), material (albedo 3, roughness, emission 3, Disney 9: 16), and the
 * material type in the top 4 bits of the last code.  Layout of record i (little endian):
 *   bytes 0-11 mean, 12-15 magnitude, 16-17 scale code, 18-19 rotation code, 20-21 SGGX
 *   code, 22-23 material code | type << 12.
 * The codebook is 4096 x 29 floats (row k: log scale 3, quaternion 4, SGGX 6, material 16).
 *
 * ugp_codebook_encode fits the four codebooks to the caller's primitives by `iters` Lloyd
 * iterations on the device (every primitive to its nearest entry by squared distance, ties to
 * the lower index; every entry with primitives to their mean, summed in 64-bit fixed point so
 * that the fit is reproducible), entries starting at the primitives of index floor(k n / 4096);
 * then writes the codebook (ugp_codebook_size() bytes, 16-byte aligned) and n records (24 n
 * bytes, 4-byte aligned).  prims and materials as for ugp_build_bvh and ugp_render
 * (disney9 may be NULL: zeros).  Workspace: ugp_codebook_workspace_size(n) bytes, 256-byte
 * aligned.  Errors: n not in [1, 2^30], iters not in [0, 100], a NULL or misaligned array,
 * UGP_ERR_INVALID_ARG; a short workspace, UGP_ERR_WORKSPACE_TOO_SMALL.
 *
 * ugp_codebook_decode expands n records into the arrays of ugp_prims and ugp_materials
 * (scale = exp of the entry, quaternion normalised; disney9 may be NULL to skip it).  Each
 * record is decoded on its own (random access).  Asynchronous on `stream`. */
size_t ugp_codebook_size(void);
size_t ugp_codebook_workspace_size(int64_t n_prims);
ugp_status ugp_codebook_encode(const ugp_prims* prims, const ugp_materials* materials, int32_t iters,
                               void* codebook, void* records, void* workspace, size_t workspace_bytes,
                               void* stream);
ugp_status ugp_codebook_decode(int64_t n, const void* records, const void* codebook, float* mean3,
                               float* quat4, float* scale3, float* magnitude, float* sggx6, uint8_t* type,
                               float* albedo3, float* roughness, float* emission3, float* disney9,
                               void* stream);

/* Pinhole camera (host struct).  Pixel (px, py), row 0 at the top, is sampled at
 * (px + jx, py + jy) with a Philox jitter (bounce 15, slot 0). */
typedef struct ugp_camera {
  float eye[3], look[3], up[3];
  float vfov_deg;
  int32_t width, height;
} ugp_camera;

/* Lights (host struct): an optional one-sided parallelogram area light
 * {corner + a e1 + b e2, a, b in [0, 1]} emitting quad_Le towards e1 x e2, and a
 * constant background radiance bg seen by rays that escape without reaching the light. */
typedef struct ugp_lights {
  int32_t has_quad;
  float quad_corner[3], quad_e1[3], quad_e2[3], quad_Le[3];
  float bg[3];
} ugp_lights;

/* ------------------------------------------------------------------ learned guide
 * A learned proposal for scattering directions. Sec. 6 allows any sampling technique that
 * is combined by MIS with the approximate phase pdf p~ of App. B; this one is a small MLP
 * that maps a scattering vertex (position x, outgoing direction wo) to a mixture of
 * UGP_GUIDE_LOBES von Mises-Fisher lobes q(wi). The paper fixes none of its details; the
 * network is:
 *   input   64 features: x normalised to [0,1]^3 over [pos_lo, pos_hi] (clamped), with
 *           sin/cos(2^l pi x), l = 0..5 (36); the polar angles (theta, phi) of wo in radians,
 *           with sin/cos(2^l angle), l = 0..3 (16); the raw (x, y, z, theta / pi,
 *           phi / (2 pi) + 1/2) (5); zeros (7)
 *   layers  four 64 x 64 ReLU layers and a 64 -> 40 head with biases, on the tensor cores:
 *           weights and layer inputs rounded to BF16 (nearest even), FP32 sums and biases
 *   head    lobe j = outputs 5j..5j+4 = (m (3), s, a): mu_j = m / |m|,
 *           kappa_j = min(kappa_max, kappa_min + softplus(s)), pi = softmax(a)
 *   q(wi) = sum_j pi_j kappa_j / (2 pi (1 - e^{-2 kappa_j})) e^{kappa_j (mu_j . wi - 1)}
 * Training minimises the mean over samples of -(L / p) ln q(wi), with L the incident-
 * radiance estimate along wi and p the pdf wi was drawn with, by Adam on FP32 master weights.
 * Parameters (FP32, UGP_GUIDE_NPARAMS): for l = 0..3, W_l (64 x 64, row-major [out][in]) then
 * b_l (64); then the head W_4 (40 x 64) and b_4 (40).
 * Mixture arrays ("mix") hold 40 floats per row: per lobe mu_x, mu_y, mu_z, kappa, pi. */
#define UGP_GUIDE_LOBES 8
#define UGP_GUIDE_WIDTH 64
#define UGP_GUIDE_OUT 40
#define UGP_GUIDE_NPARAMS 19240

typedef struct ugp_guide {
  float* params;   /* device, UGP_GUIDE_NPARAMS FP32 master weights */
  float* adam_m;   /* device, UGP_GUIDE_NPARAMS Adam first moments (zero before the first step) */
  float* adam_v;   /* device, UGP_GUIDE_NPARAMS Adam second moments (zero before the first step) */
  int64_t step;    /* Adam steps taken; ugp_guide_adam_step increments it */
  float lr, beta1, beta2, eps;   /* Adam hyper-parameters (e.g. 1e-3, 0.9, 0.99, 1e-8) */
  float pos_lo[3], pos_hi[3];    /* input normalisation box, pos_hi > pos_lo */
  float kappa_min, kappa_max;    /* lobe sharpness range, 0 < kappa_min <= kappa_max */
  int32_t train_target;  /* training from render logs: 0 incident radiance L_i (weight L_i / p),
                            1 its product with the phase function (weight f_p L_i / p: the
                            radiance the path gathered after the vertex over the throughput
                            before it), whose minimiser is q proportional to f_p L_i */
} ugp_guide;

/* Bytes of the scratch every guide call takes (packed BF16 weights, per-block gradient
 * partials, an error word). The first 256 bytes must be zero before first use
 * (ugp_guide_reset_workspace); the guide calls never clear them. */
size_t ugp_guide_workspace_size(void);
ugp_status ugp_guide_reset_workspace(void* workspace, void* stream);
/* UGP_OK, or UGP_ERR_TIMEOUT if a bounded tensor-core wait of an earlier guide call on this
 * workspace gave up (its outputs are then invalid). Synchronises `stream`. */
ugp_status ugp_guide_check(const void* workspace, void* stream);

/* Forward pass for n vertices (x3, wo3: float3 arrays). Writes, where not NULL, the head
 * outputs head_out (n x 40) and the mixture mix_out (n x 40). Asynchronous. */
ugp_status ugp_guide_forward(const ugp_guide* g, int64_t n, const float* x3, const float* wo3, float* head_out,
                             float* mix_out, void* workspace, size_t workspace_bytes, void* stream);
/* Mixture density of each row of mix at the unit direction wi3[row]. */
ugp_status ugp_guide_mixture_pdf(int64_t n, const float* mix, const float* wi3, float* pdf_out, void* stream);
/* One direction per row from uniforms u3[row] = (lobe choice, u1, u2): the lobe is the first
 * whose cumulative pi exceeds the lobe choice; 1 - mu.wi = -ln(v + (1 - v) e^{-2 kappa}) / kappa
 * with v = 1 - u1; azimuth 2 pi u2 about mu. pdf_out (may be NULL) receives q(wi). */
ugp_status ugp_guide_mixture_sample(int64_t n, const float* mix, const float* u3, float* wi_out, float* pdf_out,
                                    void* stream);
/* Gradient of the mean loss over n samples (x3, wo3, wi3: float3 arrays; weight[n] = L / p)
 * into grad_out (device, UGP_GUIDE_NPARAMS floats) and the mean loss into loss_out (device
 * float, may be NULL). The sum over samples is in a fixed order (deterministic). Asynchronous. */
ugp_status ugp_guide_grad(const ugp_guide* g, int64_t n, const float* x3, const float* wo3, const float* wi3,
                          const float* weight, float* grad_out, float* loss_out, void* workspace,
                          size_t workspace_bytes, void* stream);
/* One Adam step with the gradient grad (device): params, adam_m, adam_v in place, bias
 * corrections 1 - beta^t with t = g->step + 1; then g->step = t (host field). */
ugp_status ugp_guide_adam_step(ugp_guide* g, const float* grad, void* stream);

/* Render parameters (host struct).
 *   spp, spp_begin  samples [spp_begin, spp_begin + spp) of every pixel (resumable)
 *   max_depth       at most max_depth scattering vertices per path (>= 0)
 *   nee             1: light sampling with balance-heuristic MIS (Table 1), 0: none
 *   seed            Philox key (low, high 32 bits)
 *   spawn_mode      0: scattered rays start at the centre of the chosen primitive's
 *                   clipped interval (Sec. 6), 1: at x_{t_u}
 *   guide           NULL: phase sampling. Otherwise each scattering vertex draws its
 *                   direction from the guide with probability guide_alpha in (0, 1), else by
 *                   phase sampling, and weights it by the balance heuristic over both
 *                   techniques with p~ (one-sample MIS; unbiased for any guide). The
 *                   mixture pdf alpha q + (1 - alpha) p~ is the MIS partner of light sampling.
 *   guide_log       1: record every scattering vertex of this call for training
 *                   (ugp_guide_train_from_render); requires spp == 1 and a guide
 *   guide_min_roughness  vertices whose base is glossier (GGX alpha, or the Disney
 *                   specular's max(1e-3, roughness^2), below this value) scatter by phase
 *                   sampling alone even with a guide (0: every vertex mixes in the guide)
 *   emitters        NULL, or a device table from ugp_build_emitter_table for this BVH and
 *                   these materials: each scattering vertex then also samples a point of an
 *                   emissive primitive (light sampling, balanced against phase sampling). A
 *                   table built for another primitive count is ignored. With nee = 1 and an
 *                   area light as well, a vertex takes one light sample of each (two shadow
 *                   rays), each balanced against phase sampling alone (the two light kinds do
 *                   not overlap). */
typedef struct ugp_render_params {
  int32_t spp, spp_begin, max_depth, nee;
  uint64_t seed;
  int32_t spawn_mode, guide_log;
  const ugp_guide* guide;
  float guide_alpha;
  float guide_min_roughness;
  const void* emitters;
} ugp_render_params;

/* Light sampling toward emissive primitives (the paper finds its emitters by phase sampling
 * only). Emitter j is chosen with probability pi_j proportional to its power c_j mean(L_e,j),
 * and a point y from its Gaussian restricted to the k-ellipsoid. The free flight from a vertex
 * x picks j at distance t with density 1/2 G_j(x + t w) below the saturating distance (Eq. 8),
 * so one sample estimates the emitter's direct contribution by
 *   1/2 c_j m L_e,j f_p(w) 1[T(x, y) > 0] / (|y - x|^2 pi_j),  m = P(chi_3 <= k),
 * weighted by the balance heuristic 2 r_c^2 pi_j / (2 r_c^2 pi_j + c_j m p(w)) against phase
 * sampling (r_c: distance from x to the emitter's mean; a path that reaches the emitter by
 * phase sampling takes the complement). Philox slots 8 (choice, radius, direction) and 9-10
 * (stochastic phase evaluation).
 * ugp_emitter_table_size: bytes of the table for n_prims primitives (76 per primitive plus
 *   alignment), 0 for n_prims outside [0, 2^31 - 1].
 * ugp_build_emitter_table: fills `table` (device, 256-byte aligned, caller-owned) from the BVH
 *   and the materials' type and emission3 arrays; asynchronous on `stream`; rebuild after
 *   changing either. Errors: UGP_ERR_NOT_BUILT for an invalid handle, UGP_ERR_INVALID_ARG for
 *   a NULL or misaligned argument, UGP_ERR_WORKSPACE_TOO_SMALL. */
size_t ugp_emitter_table_size(int64_t n_prims);
ugp_status ugp_build_emitter_table(const ugp_bvh* bvh, const ugp_materials* materials, void* table,
                                   size_t table_bytes, void* stream);

/* Workspace bytes ugp_render needs for a width x height image (path state, queues and
 * per-path primitive-slot lists, 1284 bytes per pixel, plus one 73,728-byte interval slot of the
 * free-flight finish per 64 pixels, at most 2432 of them, plus alignment). */
size_t ugp_render_workspace_size(int32_t width, int32_t height);
/* Workspace bytes of a guided render of up to max_depth scattering vertices: the plain
 * workspace, the per-path mixtures (160 bytes per pixel), the training log (88 bytes per
 * pixel and vertex) and the guide's packed weights. */
size_t ugp_render_guided_workspace_size(int32_t width, int32_t height, int32_t max_depth);

/* Path-traces the image with the volumetric path tracer of Table 1 (right column)
 * as a wavefront: per bounce, an extend pass (free-flight sampling,
 * ugp_sample_free_flight), a shade pass (emission, light sampling, phase
 * sampling) and a shadow pass (ugp_trace_transmittance), with live paths
 * compacted between bounces.  Random numbers are Philox4x32-10 with counter
 * (pixel, sample, 16 * bounce + slot, 0); slots: 0 free flight, 1 phase
 * sampling, 2 guide (lobe choice, technique choice, two for the lobe), 3 light point,
 * 4-5 stochastic phase evaluation of the light sample, 6-7 stochastic phase evaluation
 * of a guide sample.
 *   accum_rgb, accum_sq_rgb  device float arrays (height x width x 3) to which the
 *                per-pixel sums of sample values and of their squares are ADDED
 *   ray_counts   device uint64[3] or NULL: [0] += free-flight queries,
 *                [1] += shadow queries, [2] += queries with a non-zero ray status
 * Asynchronous on `stream`. */
ugp_status ugp_render(const ugp_bvh* bvh, const ugp_materials* materials, const ugp_camera* camera,
                      const ugp_lights* lights, const ugp_render_params* params, float* accum_rgb,
                      float* accum_sq_rgb, void* workspace, size_t workspace_bytes,
                      unsigned long long* ray_counts, void* stream);

/* Trains the guide on the vertices logged by the last ugp_render call with guide_log = 1 on
 * `render_ws` (same width, height and max_depth). For every logged vertex the incident
 * radiance L along its sampled direction is the radiance the path gathered after the vertex
 * divided by the path throughput after it (per channel, luminance-weighted); vertices with
 * L > 0 are the training samples, with weight L / p. If there are more than max_samples, a
 * deterministic hash keeps about max_samples of them. They are visited in minibatches of
 * `minibatch` rows, one ugp_guide_grad + ugp_guide_adam_step each: one pass over the samples,
 * or min_steps minibatches taken cyclically when that is more. Writes the number of samples
 * used and the mean loss of the last minibatch (host, may be NULL). Synchronises. */
ugp_status ugp_guide_train_from_render(ugp_guide* g, const void* render_ws, size_t render_ws_bytes, int32_t width,
                                       int32_t height, int32_t max_depth, int64_t max_samples, int32_t minibatch,
                                       int32_t min_steps, void* guide_ws, size_t guide_ws_bytes,
                                       int64_t* n_samples_out, float* mean_loss_out, void* stream);

/* ------------------------------------------------------------------ batched serving
 * Many independent render requests (own scene, camera, lights, image size, spp and depth)
 * served together. The paper has no counterpart: it is the serving form of ugp_render.
 * Work items are (request, sample, square tile of `tile` x `tile` pixels), taken in request
 * order from one atomic counter into a shared pool of 2^pool_log2 paths: every wave fills the
 * free pool slots with camera paths of new items, then extends, finishes, shades and
 * shadow-traces every live path in its own request's scene, and retires the paths that
 * ended into their request's image. A path draws exactly the Philox numbers ugp_render
 * draws for that request (counter (pixel, sample, 16 * bounce + slot, 0), key = the
 * request's seed), so each image equals ugp_render's up to the order of the per-pixel sums.
 * With use_graph = 1 the waves run inside one CUDA graph launch (a conditional while-node
 * whose body is one wave; the graph is instantiated once per workspace and pool size and
 * reused); with use_graph = 0 the host launches the waves and polls a device flag. */
typedef struct ugp_request {
  const ugp_bvh* bvh;              /* built scene of the request */
  const ugp_materials* materials;  /* host struct of device arrays, as for ugp_render */
  ugp_camera camera;               /* image of camera.width x camera.height pixels */
  ugp_lights lights;
  int32_t spp;                     /* samples 0 .. spp-1 of every pixel */
  int32_t max_depth;               /* scattering vertices per path, 0..14 */
  int32_t nee, spawn_mode;         /* as in ugp_render_params */
  uint64_t seed;                   /* Philox key */
  float* accum_rgb;                /* device, height x width x 3: per-pixel sums ADDED */
  float* accum_sq_rgb;             /* device, same layout: sums of squares ADDED */
} ugp_request;

typedef struct ugp_batch_config {
  int32_t tile;       /* side of a work item's pixel tile: 8, 16 or 32 */
  int32_t pool_log2;  /* paths in flight: 2^pool_log2, 10..24 */
  int32_t use_graph;  /* 1: one CUDA graph launch with a device-side loop; 0: host loop */
  int32_t order;      /* service order: 0 as given, 1 shortest first (pixels x spp x (depth + 1)) */
} ugp_batch_config;

/* Workspace bytes for batches of up to max_requests requests with this config (path pool,
 * queues, request table); 0 for a bad argument. */
size_t ugp_render_batch_workspace_size(int32_t max_requests, const ugp_batch_config* cfg);
/* Renders the n_req requests (host array) with a workspace sized for max_requests. Waits for
 * the batch to finish. latency_ms_out (host, n_req doubles, may be NULL) receives each
 * request's completion time after the batch started (device %globaltimer; 0 for a request
 * with no paths). ray_counts as for ugp_render. UGP_ERR_ITER_LIMIT if the device-side wave
 * bound was reached with work left (never expected). A graph built for a workspace must not
 * be launched concurrently from two streams. */
ugp_status ugp_render_batch(int32_t n_req, const ugp_request* reqs, const ugp_batch_config* cfg,
                            int32_t max_requests, void* workspace, size_t workspace_bytes, double* latency_ms_out,
                            unsigned long long* ray_counts, void* stream);

/* Autotuner of the batch configuration: renders a probe of the batch (every request at
 * min(spp, probe_spp) samples, accumulating into `scratch`, which must hold
 * 6 x (largest width x height) floats) with every candidate tile in {8, 16, 32} and pool in
 * 2^[pool_log2_min, pool_log2_max] whose workspace fits `workspace_bytes`, each once to build
 * its graph and once timed (CUDA events), and returns the fastest in best_out. ms_out (host,
 * 3 x (pool_log2_max - pool_log2_min + 1) doubles, pool-major, -1 for skipped candidates,
 * may be NULL) receives the probe times. Results are cached per device and batch shape
 * (request count, deepest request, probe paths) and reused when ms_out is NULL.
 * Synchronises. */
ugp_status ugp_render_batch_autotune(int32_t n_req, const ugp_request* reqs, int32_t probe_spp, int32_t pool_log2_min,
                                     int32_t pool_log2_max, int32_t use_graph, void* workspace,
                                     size_t workspace_bytes, float* scratch, size_t scratch_floats,
                                     ugp_batch_config* best_out, double* ms_out, void* stream);

/* Optional traversal statistics: when `counters` is a device pointer to 12
 * zero-initialised uint64, later tracing calls on any stream add (atomically)
 *   [0] nodes loaded, [1] primitive records loaded, [2] rays traced,
 *   [3] per-thread traversal passes, [4] free-flight rays handed to the finish passes
 *   (whose node and record loads are added to [0] and [1]), [5] free-flight rays the
 *   finish's first pass handed to its second (more intervals than 16 lanes hold, or an
 *   overflowed slot list)
 * for free-flight and transmittance queries (standalone, and the renderer's extend
 * pass), and the first five quantities at [6..10] for the renderer's shadow rays;
 * [11] is reserved.  NULL turns counting off (the default).  Host-side
 * setting, not thread safe against concurrent tracing calls. */
ugp_status ugp_set_trace_counters(unsigned long long* counters);

/* ------------------------------------------------------------------ measurement
 * Kernel timing without synchronisation: after ugp_profile_begin, every kernel the
 * library launches is bracketed by a pair of CUDA events recorded on the launch
 * stream (host-side event objects, created on first use and reused).  Stages:
 *   0 BVH build (all its kernels, the radix sort included), 1 camera rays,
 *   2 extend (free flight, per thread), 3 shade, 4 shadow (transmittance),
 *   5 accumulate, 6 standalone queries (ugp_trace_transmittance,
 *   ugp_sample_free_flight), 7 finish of free flight (the bracketed rays), 8 learned guide
 *   (packing, forward, gradient, Adam, training-set selection), 9 batched serving (one pair
 *   around each batch's graph launch or wave loop; graph launches add their kernels to the
 *   counts after the batch).
 * ugp_profile_end waits for the recorded events, writes the summed milliseconds and
 * launch counts per stage (arrays of UGP_PROFILE_STAGES, host) and stops recording.
 * At most max_records event pairs are kept; later launches are counted but not timed
 * (ugp_profile_end returns UGP_ERR_OVERFLOW then).  Not thread safe. */
#define UGP_PROFILE_STAGES 10
ugp_status ugp_profile_begin(int32_t max_records);
ugp_status ugp_profile_end(double* ms_out, int64_t* launches_out);

/* Number of kernels the library has launched since it was loaded (its own kernels and
 * the radix-sort kernels of the BVH build). */
int64_t ugp_launch_count(void);

/* Static description of a status code. */
const char* ugp_status_string(ugp_status s);
/* Thread-local message of the last failing call on this thread ("" if none). */
const char* ugp_last_error(void);
/* Library version string. */
const char* ugp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* UGP_H_ */
