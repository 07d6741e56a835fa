"""ctypes front end of the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, brute-force C++
statement of what the Gaussian-primitive path tracer computes (Eq. 1-10, the
appendices, and the path-tracing loop of Table 1), in double precision.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library; the
two meet only in the seeded input generators of
``paper_2406_09733_gb300.scenes``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_LIB = None

f32p = C.POINTER(C.c_float)
f64p = C.POINTER(C.c_double)
i32p = C.POINTER(C.c_int32)
u32p = C.POINTER(C.c_uint32)
u8p = C.POINTER(C.c_uint8)


class OrcScene(C.Structure):
    _fields_ = [("n", C.c_int64), ("mean3", f32p), ("quat4", f32p), ("scale3", f32p),
                ("magnitude", f32p), ("sggx6", f32p), ("type", u8p), ("albedo3", f32p),
                ("roughness", f32p), ("emission3", f32p), ("disney9", f32p)]


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_prim_setup.argtypes = [C.POINTER(OrcScene), C.c_double, f64p, f64p, f64p]
        L.orc_prim_integral.argtypes = [C.POINTER(OrcScene), C.c_int64, f32p, f32p, C.c_double,
                                        C.c_double]
        L.orc_prim_integral.restype = C.c_double
        L.orc_hits.argtypes = [C.POINTER(OrcScene), C.c_double, f32p, f32p, C.c_float, C.c_float,
                               C.c_int32, i32p, f64p, f64p, f64p, f64p, C.c_int64]
        L.orc_hits.restype = C.c_int64
        L.orc_transmittance.argtypes = [C.POINTER(OrcScene), C.c_double, C.c_int64, f32p, f32p,
                                        f32p, f32p, i32p, f64p, f64p, i32p]
        L.orc_sample_free_flight.argtypes = [C.POINTER(OrcScene), C.c_double, C.c_int64, f32p,
                                             f32p, f32p, f32p, i32p, f32p, f32p, i32p, f64p,
                                             f64p, f64p, i32p, f64p]
        L.orc_race_exponential.argtypes = [C.c_double, C.c_int32]
        L.orc_radiance_field.argtypes = [C.POINTER(OrcScene), C.c_double, C.c_int64, f32p, f32p, f32p, f32p,
                                         f32p, f64p, C.c_double, f64p, f64p, f64p]
        L.orc_race_exponential.restype = C.c_double
        L.orc_sample_free_flight_exponential.argtypes = [C.POINTER(OrcScene), C.c_double, C.c_int64, f32p, f32p,
                                                         f32p, f32p, i32p, f32p, i32p, f64p, f64p, f64p, f64p,
                                                         f64p, f64p]
        L.orc_transmittance_exponential.argtypes = [C.POINTER(OrcScene), C.c_double, C.c_int64, f32p, f32p,
                                                    f32p, f32p, i32p, f64p, f64p]
        L.orc_band_rays.argtypes = [C.POINTER(OrcScene), C.c_double, C.c_int64, f32p, f32p, f32p, f32p, C.c_double,
                                    i32p]
        L.orc_sample_free_flight_paper_rule.argtypes = [C.POINTER(OrcScene), C.c_double, C.c_int64, f32p, f32p,
                                                        f32p, f32p, f32p, f32p, i32p]
        L.orc_kd_sample_tree.argtypes = [C.POINTER(OrcScene), C.c_double, i32p, C.c_int64, i32p, C.c_int64, f32p,
                                         C.c_int32, C.c_int64, f32p, f32p, f32p, f32p, f32p, f32p, i32p, f64p]
        L.orc_kd_sample_free_flight.argtypes = [C.POINTER(OrcScene), C.c_double, C.c_int64, f32p, f32p, f32p, f32p,
                                                f32p, f32p, i32p, f64p, C.POINTER(C.c_int64),
                                                C.POINTER(C.c_int64)]
        L.orc_decomposition_exponential.argtypes = [C.c_double, C.c_int32]
        L.orc_decomposition_exponential.restype = C.c_double
        L.orc_prim_quadratic.argtypes = [C.POINTER(OrcScene), C.c_int64, f32p, f32p, f64p]
        L.orc_erfinv.argtypes = [C.c_double]
        L.orc_erfinv.restype = C.c_double
        _post_load(L)
        _LIB = L
    return _LIB


def _post_load(L):
    """Hook for the argtypes of the phase, render and guide modules (filled below)."""
    for fn in _REGISTRY:
        fn(L)


_REGISTRY = []


def _ptr(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(t)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class _SceneRef:
    """Keeps the numpy arrays behind an OrcScene alive."""

    def __init__(self, scene):
        self.arrs = dict(
            mean=_c(scene.mean, np.float32), quat=_c(scene.quat, np.float32),
            scale=_c(scene.scale, np.float32), mag=_c(scene.magnitude, np.float32),
            sggx=_c(scene.sggx, np.float32), type=_c(scene.mtype, np.uint8),
            albedo=_c(scene.albedo, np.float32), rough=_c(scene.roughness, np.float32),
            emit=_c(scene.emission, np.float32))
        dis = getattr(scene, "disney", None)
        if dis is not None:
            self.arrs["disney"] = _c(dis, np.float32)
        a = self.arrs
        self.s = OrcScene(scene.n, _ptr(a["mean"], f32p), _ptr(a["quat"], f32p),
                          _ptr(a["scale"], f32p), _ptr(a["mag"], f32p), _ptr(a["sggx"], f32p),
                          _ptr(a["type"], u8p), _ptr(a["albedo"], f32p), _ptr(a["rough"], f32p),
                          _ptr(a["emit"], f32p), _ptr(a["disney"], f32p) if dis is not None else None)

    @property
    def ref(self):
        return C.byref(self.s)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, u32p), _ptr(k, u32p), _ptr(out, u32p))
    return out


def prim_setup(scene, eps=0.01):
    n = scene.n
    W = np.zeros((n, 9))
    g0 = np.zeros(n)
    aabb = np.zeros((n, 6))
    sr = _SceneRef(scene)
    lib().orc_prim_setup(sr.ref, eps, _ptr(W, f64p), _ptr(g0, f64p), _ptr(aabb, f64p))
    return W.reshape(n, 3, 3), g0, aabb


def prim_integral(scene, i, o, d, ta, tb) -> float:
    sr = _SceneRef(scene)
    o = _c(o, np.float32)
    d = _c(d, np.float32)
    return float(lib().orc_prim_integral(sr.ref, int(i), _ptr(o, f32p), _ptr(d, f32p), float(ta),
                                         float(tb)))


def hits(scene, o, d, t0, t1, exclude=-1, eps=0.01, cap=4096, _sr=None):
    sr = _sr or _SceneRef(scene)
    o = _c(o, np.float32)
    d = _c(d, np.float32)
    ids = np.zeros(cap, np.int32)
    a, b, d2, hI = (np.zeros(cap) for _ in range(4))
    m = lib().orc_hits(sr.ref, eps, _ptr(o, f32p), _ptr(d, f32p), float(t0), float(t1),
                       int(exclude), _ptr(ids, i32p), _ptr(a, f64p), _ptr(b, f64p),
                       _ptr(d2, f64p), _ptr(hI, f64p), cap)
    m = min(int(m), cap)
    return dict(ids=ids[:m], a=a[:m], b=b[:m], d2=d2[:m], half_I=hI[:m])


def transmittance(scene, rays, exclude=None, eps=0.01):
    sr = _SceneRef(scene)
    n = rays.n
    o, d = _c(rays.o, np.float32), _c(rays.d, np.float32)
    t0, t1 = _c(rays.t0, np.float32), _c(rays.t1, np.float32)
    ex = None if exclude is None else _c(exclude, np.int32)
    T = np.zeros(n)
    tau = np.zeros(n)
    nh = np.zeros(n, np.int32)
    lib().orc_transmittance(sr.ref, eps, n, _ptr(o, f32p), _ptr(d, f32p), _ptr(t0, f32p),
                            _ptr(t1, f32p), _ptr(ex, i32p), _ptr(T, f64p), _ptr(tau, f64p),
                            _ptr(nh, i32p))
    return T, tau, nh


def sample_free_flight(scene, rays, u, u2, exclude=None, eps=0.01):
    sr = _SceneRef(scene)
    n = rays.n
    o, d = _c(rays.o, np.float32), _c(rays.d, np.float32)
    t0, t1 = _c(rays.t0, np.float32), _c(rays.t1, np.float32)
    u = _c(u, np.float32)
    u2 = _c(u2, np.float32)
    ex = None if exclude is None else _c(exclude, np.int32)
    prim = np.zeros(n, np.int32)
    tu, ts, fe = np.zeros(n), np.zeros(n), np.zeros(n)
    na = np.zeros(n, np.int32)
    mg = np.zeros(n)
    lib().orc_sample_free_flight(sr.ref, eps, n, _ptr(o, f32p), _ptr(d, f32p), _ptr(t0, f32p),
                                 _ptr(t1, f32p), _ptr(ex, i32p), _ptr(u, f32p), _ptr(u2, f32p),
                                 _ptr(prim, i32p), _ptr(tu, f64p), _ptr(ts, f64p), _ptr(fe, f64p),
                                 _ptr(na, i32p), _ptr(mg, f64p))
    return dict(prim=prim, t_u=tu, t_spawn=ts, F_end=fe, n_active=na, race_margin=mg)


def radiance_field(scene, rays, emission, background=(0.0, 0.0, 0.0), eps=0.01, t_shift_ulps=0.0):
    """Radiance-field render of Sec. 7 (Eq. rf): per ray the RGB sum of 1/2 I_k clipped at the
    saturating distance times primitive k's emission (indexed by primitive), plus the
    unsaturated remainder times the background. t_shift_ulps moves the saturating distance by
    that many float32 ulps of itself (for tolerance bounds). Returns (rgb (n, 3), t_sat (n,),
    F_end (n,))."""
    sr = _SceneRef(scene)
    n = rays.n
    o, d = _c(rays.o, np.float32), _c(rays.d, np.float32)
    t0, t1 = _c(rays.t0, np.float32), _c(rays.t1, np.float32)
    em = _c(emission, np.float32)
    bg = _c(np.asarray(background, np.float64), np.float64)
    rgb, ts, fe = np.zeros((n, 3)), np.zeros(n), np.zeros(n)
    lib().orc_radiance_field(sr.ref, eps, n, _ptr(o, f32p), _ptr(d, f32p), _ptr(t0, f32p), _ptr(t1, f32p),
                             _ptr(em, f32p), _ptr(bg, f64p), float(t_shift_ulps), _ptr(rgb, f64p), _ptr(ts, f64p),
                             _ptr(fe, f64p))
    return rgb, ts, fe


def sample_free_flight_exponential(scene, rays, u, exclude=None, eps=0.01):
    """Analog decomposition tracking of the exponential variant (sigma_t = sum_k G_k): per ray
    the nearest per-primitive exponential collision, keyed by the uniform u. Returns a dict of
    prim (-1: escape), t (t1 on escape), t_second (next-nearest collision, inf if none), margin
    (min relative gap between a primitive's variate and its optical depth), amp and G_t of the
    chosen primitive (I = amp [erf(tau_t) - erf(tau_a)], G at t) and depth (sum_k I_k)."""
    sr = _SceneRef(scene)
    n = rays.n
    o, d = _c(rays.o, np.float32), _c(rays.d, np.float32)
    t0, t1 = _c(rays.t0, np.float32), _c(rays.t1, np.float32)
    u = _c(u, np.float32)
    ex = None if exclude is None else _c(exclude, np.int32)
    prim = np.zeros(n, np.int32)
    t, t2, mg, amp, G, depth = (np.zeros(n) for _ in range(6))
    lib().orc_sample_free_flight_exponential(sr.ref, eps, n, _ptr(o, f32p), _ptr(d, f32p), _ptr(t0, f32p),
                                             _ptr(t1, f32p), _ptr(ex, i32p), _ptr(u, f32p), _ptr(prim, i32p),
                                             _ptr(t, f64p), _ptr(t2, f64p), _ptr(mg, f64p), _ptr(amp, f64p),
                                             _ptr(G, f64p), _ptr(depth, f64p))
    return dict(prim=prim, t=t, t_second=t2, margin=mg, amp=amp, G_t=G, depth=depth)


def transmittance_exponential(scene, rays, exclude=None, eps=0.01):
    """exp(-sum_k I_k) over each ray's [t0, t1]; returns (T, optical depth)."""
    sr = _SceneRef(scene)
    n = rays.n
    o, d = _c(rays.o, np.float32), _c(rays.d, np.float32)
    t0, t1 = _c(rays.t0, np.float32), _c(rays.t1, np.float32)
    ex = None if exclude is None else _c(exclude, np.int32)
    T, depth = np.zeros(n), np.zeros(n)
    lib().orc_transmittance_exponential(sr.ref, eps, n, _ptr(o, f32p), _ptr(d, f32p), _ptr(t0, f32p),
                                        _ptr(t1, f32p), _ptr(ex, i32p), _ptr(T, f64p), _ptr(depth, f64p))
    return T, depth


def sample_free_flight_paper_rule(scene, rays, u, u2, eps=0.01):
    """Free-flight sampling with the paper's own disambiguation rule (pick proportional to
    I_k(s0, t_u) in the segment where F reaches 1): a diagnostic of that rule's bias, not a
    parity target. Returns the primitive per ray (-1: escape)."""
    sr = _SceneRef(scene)
    n = rays.n
    o, d = _c(rays.o, np.float32), _c(rays.d, np.float32)
    t0, t1 = _c(rays.t0, np.float32), _c(rays.t1, np.float32)
    u, u2 = _c(u, np.float32), _c(u2, np.float32)
    prim = np.zeros(n, np.int32)
    lib().orc_sample_free_flight_paper_rule(sr.ref, eps, n, _ptr(o, f32p), _ptr(d, f32p), _ptr(t0, f32p),
                                            _ptr(t1, f32p), _ptr(u, f32p), _ptr(u2, f32p), _ptr(prim, i32p))
    return prim


def kd_sample_tree(scene, nodes4, refs, box6, rays, u, u2, nbins=8, eps=0.01):
    """The paper's sampler over a given kd-tree (nodes4 (m, 4) int32, refs int32 primitive indices,
    box6 the root box), with an ambiguous leaf cut into nbins equal bins of its ray interval (the
    paper's GPU partition; 0: exact segments). Returns (prim, start of the disambiguated segment
    or NaN)."""
    sr = _SceneRef(scene)
    n = rays.n
    o, d, t0, t1 = (_c(x, np.float32) for x in (rays.o, rays.d, rays.t0, rays.t1))
    nodes4 = _c(nodes4, np.int32)
    refs = _c(refs, np.int32)
    box6 = _c(box6, np.float32)
    u, u2 = _c(u, np.float32), _c(u2, np.float32)
    prim = np.zeros(n, np.int32)
    amb = np.zeros(n)
    lib().orc_kd_sample_tree(sr.ref, eps, _ptr(nodes4, i32p), nodes4.shape[0], _ptr(refs, i32p), refs.size,
                             _ptr(box6, f32p), int(nbins), n, _ptr(o, f32p), _ptr(d, f32p), _ptr(t0, f32p),
                             _ptr(t1, f32p), _ptr(u, f32p), _ptr(u2, f32p), _ptr(prim, i32p), _ptr(amb, f64p))
    return prim, amb


def kd_sample_free_flight(scene, rays, u, u2, eps=0.01):
    """The paper's own free-flight sampler over an SAH kd-tree (Sec. 5.2): per-leaf accumulation in
    front-to-back order and its disambiguation rule. A diagnostic, not a parity target. Returns a
    dict of prim (-1: escape), ambiguous_start (start of the ambiguous segment used, NaN if none),
    nodes and prims (kd-tree nodes visited and primitives tested)."""
    sr = _SceneRef(scene)
    n = rays.n
    o, d = _c(rays.o, np.float32), _c(rays.d, np.float32)
    t0, t1 = _c(rays.t0, np.float32), _c(rays.t1, np.float32)
    u, u2 = _c(u, np.float32), _c(u2, np.float32)
    prim = np.zeros(n, np.int32)
    amb = np.zeros(n)
    nodes, prims = np.zeros(n, np.int64), np.zeros(n, np.int64)
    i64p = C.POINTER(C.c_int64)
    lib().orc_kd_sample_free_flight(sr.ref, eps, n, _ptr(o, f32p), _ptr(d, f32p), _ptr(t0, f32p), _ptr(t1, f32p),
                                    _ptr(u, f32p), _ptr(u2, f32p), _ptr(prim, i32p), _ptr(amb, f64p),
                                    nodes.ctypes.data_as(i64p), prims.ctypes.data_as(i64p))
    return dict(prim=prim, ambiguous_start=amb, nodes=nodes, prims=prims)


def band_rays(scene, rays, rel=1e-5, eps=0.01):
    """Boolean per ray: its hit set is decided at rounding level (a primitive whose whitened
    closest approach is within rel of the cut-off k inside [t0, t1], or an ellipsoid end point
    within rel (t1 - t0) of t0 or t1)."""
    sr = _SceneRef(scene)
    n = rays.n
    o, d = _c(rays.o, np.float32), _c(rays.d, np.float32)
    t0, t1 = _c(rays.t0, np.float32), _c(rays.t1, np.float32)
    flag = np.zeros(n, np.int32)
    lib().orc_band_rays(sr.ref, eps, n, _ptr(o, f32p), _ptr(d, f32p), _ptr(t0, f32p), _ptr(t1, f32p), float(rel),
                        _ptr(flag, i32p))
    return flag.astype(bool)


def decomposition_exponential(u: float, k: int) -> float:
    """The collision depth E_k = -ln U_k of primitive k for the ray uniform u."""
    return float(lib().orc_decomposition_exponential(float(np.float32(u)), int(k)))


def race_exponential(u2: float, k: int) -> float:
    """The race variate E_k = -ln U_k of primitive k for the uniform u2 (free-flight choice)."""
    return float(lib().orc_race_exponential(float(np.float32(u2)), int(k)))


def prim_quadratic(scene, i, o, d, _sr=None):
    """(A, t*, d2) of App. A for primitive i along the ray (o, d), unclipped."""
    sr = _sr or _SceneRef(scene)
    o = _c(o, np.float32)
    d = _c(d, np.float32)
    out = np.zeros(3)
    lib().orc_prim_quadratic(sr.ref, int(i), _ptr(o, f32p), _ptr(d, f32p), _ptr(out, f64p))
    return out


def erfinv(y: float) -> float:
    return float(lib().orc_erfinv(float(y)))


# ------------------------------------------------------------------ appearance and rendering
def _register_phase(L):
    d = f64p
    L.orc_sggx_eval.argtypes = [d, C.c_int64, d, d, d]
    L.orc_sggx_dvis.argtypes = [d, d, C.c_int64, d, d]
    L.orc_sggx_sample_vndf.argtypes = [d, d, C.c_int64, d, d]
    L.orc_sggx_roughen.argtypes = [d, C.c_double, d]
    L.orc_base_bsdf.argtypes = [C.c_int, d, C.c_double, C.c_int64, d, d, d, d]
    L.orc_ggx_sample_vn.argtypes = [C.c_double, d, d, C.c_int64, d, d]
    L.orc_micro_sample.argtypes = [C.c_double, d, C.c_int64, d, d]
    L.orc_phase_eval.argtypes = [C.c_int, d, C.c_double, d, d, C.c_int64, d, d, C.c_int, d]
    L.orc_phase_sample.argtypes = [C.c_int, d, C.c_double, d, d, C.c_int64, d, d, d, i32p]
    L.orc_phase_pdf_approx.argtypes = [C.c_int, d, C.c_double, d, d, C.c_int64, d, d]
    L.orc_disney_f.argtypes = [d, d, C.c_int64, d, d, d, d]
    L.orc_disney_f_diffuse.argtypes = [d, d, C.c_int64, d, d, d, d]
    L.orc_disney_pdf.argtypes = [d, d, d, d, C.c_int64, d, d]
    L.orc_disney_sample.argtypes = [d, d, d, d, C.c_int64, d, d, d, i32p]
    L.orc_gtr1_D.argtypes = [C.c_double, C.c_double]
    L.orc_gtr1_D.restype = C.c_double
    L.orc_phase_eval_disney.argtypes = [d, d, d, d, C.c_int64, d, d, d]
    L.orc_phase_sample_disney.argtypes = [d, d, d, d, C.c_int64, d, d, d, i32p]
    L.orc_phase_pdf_approx_disney.argtypes = [d, d, d, d, C.c_int64, d, d]
    L.orc_render.argtypes = [C.POINTER(OrcScene), C.POINTER(OrcCamera), C.POINTER(OrcLights),
                             C.POINTER(OrcParams), C.c_int64, C.c_int64, d, d,
                             C.POINTER(C.c_int64)]
    L.orc_sample_in_ellipsoid.argtypes = [C.POINTER(OrcScene), C.c_int64, C.c_double, C.c_int64, d, d]
    L.orc_emitter_nee.argtypes = [C.POINTER(OrcScene), C.c_double, d, d, C.c_int32, C.c_int32, d, C.c_double, d,
                                  C.c_int64, C.c_uint64, d, d]
    L.orc_chi3_cdf.argtypes = [C.c_double]
    L.orc_chi3_cdf.restype = C.c_double


_REGISTRY.append(_register_phase)


class OrcCamera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class OrcLights(C.Structure):
    _fields_ = [("has_quad", C.c_int32), ("corner", C.c_float * 3), ("e1", C.c_float * 3),
                ("e2", C.c_float * 3), ("Le", C.c_float * 3), ("bg", C.c_float * 3)]


class OrcGuideCfg(C.Structure):
    _fields_ = [("pos_lo", C.c_double * 3), ("pos_hi", C.c_double * 3), ("kappa_min", C.c_double),
                ("kappa_max", C.c_double), ("round_bf16", C.c_int32)]


class OrcParams(C.Structure):
    _fields_ = [("spp", C.c_int32), ("spp_begin", C.c_int32), ("max_depth", C.c_int32),
                ("seed", C.c_uint64), ("cutoff_eps", C.c_double), ("nee", C.c_int32),
                ("spawn_mode", C.c_int32), ("guide", f32p), ("guide_cfg", OrcGuideCfg),
                ("guide_alpha", C.c_double), ("nee_emitters", C.c_int32), ("accel", C.c_int32),
                ("guide_min_roughness", C.c_double), ("crop_x0", C.c_int32), ("crop_x1", C.c_int32)]


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def sggx_eval(S6, w):
    S6, w = _d(S6), _d(w).reshape(-1, 3)
    n = w.shape[0]
    sig, D = np.zeros(n), np.zeros(n)
    lib().orc_sggx_eval(_ptr(S6, f64p), n, _ptr(w, f64p), _ptr(sig, f64p), _ptr(D, f64p))
    return sig, D


def sggx_dvis(S6, wo, nrm):
    S6, wo, nrm = _d(S6), _d(wo), _d(nrm).reshape(-1, 3)
    out = np.zeros(nrm.shape[0])
    lib().orc_sggx_dvis(_ptr(S6, f64p), _ptr(wo, f64p), nrm.shape[0], _ptr(nrm, f64p), _ptr(out, f64p))
    return out


def sggx_sample_vndf(S6, wo, U2):
    S6, wo, U2 = _d(S6), _d(wo), _d(U2).reshape(-1, 2)
    out = np.zeros((U2.shape[0], 3))
    lib().orc_sggx_sample_vndf(_ptr(S6, f64p), _ptr(wo, f64p), U2.shape[0], _ptr(U2, f64p), _ptr(out, f64p))
    return out


def sggx_roughen(S6, alpha):
    S6 = _d(S6)
    out = np.zeros(6)
    lib().orc_sggx_roughen(_ptr(S6, f64p), float(alpha), _ptr(out, f64p))
    return out


def base_bsdf(mtype, albedo, alpha, wi, wo, nrm):
    albedo, wi, wo, nrm = _d(albedo), _d(wi).reshape(-1, 3), _d(wo), _d(nrm)
    out = np.zeros((wi.shape[0], 3))
    lib().orc_base_bsdf(int(mtype), _ptr(albedo, f64p), float(alpha), wi.shape[0], _ptr(wi, f64p),
                        _ptr(wo, f64p), _ptr(nrm, f64p), _ptr(out, f64p))
    return out


def ggx_sample_vn(alpha, wo, nrm, U2):
    wo, nrm, U2 = _d(wo), _d(nrm), _d(U2).reshape(-1, 2)
    out = np.zeros((U2.shape[0], 3))
    lib().orc_ggx_sample_vn(float(alpha), _ptr(wo, f64p), _ptr(nrm, f64p), U2.shape[0], _ptr(U2, f64p),
                            _ptr(out, f64p))
    return out


def micro_sample(alpha, h, U2):
    h, U2 = _d(h), _d(U2).reshape(-1, 2)
    out = np.zeros((U2.shape[0], 3))
    lib().orc_micro_sample(float(alpha), _ptr(h, f64p), U2.shape[0], _ptr(U2, f64p), _ptr(out, f64p))
    return out


def phase_eval(mtype, albedo, alpha, S6, wo, wi, U6=None, mode=0):
    albedo, S6, wo, wi = _d(albedo), _d(S6), _d(wo), _d(wi).reshape(-1, 3)
    n = wi.shape[0]
    U6 = np.zeros((n, 6)) if U6 is None else _d(U6).reshape(n, 6)
    out = np.zeros((n, 3))
    lib().orc_phase_eval(int(mtype), _ptr(albedo, f64p), float(alpha), _ptr(S6, f64p), _ptr(wo, f64p), n,
                         _ptr(wi, f64p), _ptr(U6, f64p), int(mode), _ptr(out, f64p))
    return out


# Disney principled base (Sec. 6): dis = (metallic, subsurface, specular, specular tint, roughness,
# sheen, sheen tint, clearcoat, clearcoat gloss), C the base colour.
def disney_f(C, dis, wi, wo, nrm):
    """Cosine-weighted base BSDF f <n.wi> for directions wi (n x 3)."""
    wi = _d(wi).reshape(-1, 3)
    out = np.zeros_like(wi)
    lib().orc_disney_f(_ptr(_d(C), f64p), _ptr(_d(dis), f64p), wi.shape[0], _ptr(wi, f64p), _ptr(_d(wo), f64p),
                       _ptr(_d(nrm), f64p), _ptr(out, f64p))
    return out


def disney_f_diffuse(C, dis, wi, wo, nrm):
    """The diffuse, subsurface and sheen part of the base, times <n.wi>, for directions wi (n x 3)."""
    wi = _d(wi).reshape(-1, 3)
    out = np.zeros_like(wi)
    lib().orc_disney_f_diffuse(_ptr(_d(C), f64p), _ptr(_d(dis), f64p), wi.shape[0], _ptr(wi, f64p),
                               _ptr(_d(wo), f64p), _ptr(_d(nrm), f64p), _ptr(out, f64p))
    return out


def disney_pdf(C, dis, wo, nrm, wi):
    wi = _d(wi).reshape(-1, 3)
    out = np.zeros(wi.shape[0])
    lib().orc_disney_pdf(_ptr(_d(C), f64p), _ptr(_d(dis), f64p), _ptr(_d(wo), f64p), _ptr(_d(nrm), f64p),
                         wi.shape[0], _ptr(wi, f64p), _ptr(out, f64p))
    return out


def disney_sample(C, dis, wo, nrm, U2):
    """(wi, weight, ok) of the base sampler from two uniforms per sample."""
    U = _d(U2).reshape(-1, 2)
    n = U.shape[0]
    wi, w = np.zeros((n, 3)), np.zeros((n, 3))
    ok = np.zeros(n, np.int32)
    lib().orc_disney_sample(_ptr(_d(C), f64p), _ptr(_d(dis), f64p), _ptr(_d(wo), f64p), _ptr(_d(nrm), f64p), n,
                            _ptr(U, f64p), _ptr(wi, f64p), _ptr(w, f64p), _ptr(ok, i32p))
    return wi, w, ok.astype(bool)


def gtr1_D(a, c):
    return float(lib().orc_gtr1_D(float(a), float(c)))


def phase_eval_disney(C, dis, S6, wo, wi, U6):
    wi = _d(wi).reshape(-1, 3)
    n = wi.shape[0]
    out = np.zeros((n, 3))
    lib().orc_phase_eval_disney(_ptr(_d(C), f64p), _ptr(_d(dis), f64p), _ptr(_d(S6), f64p), _ptr(_d(wo), f64p), n,
                                _ptr(wi, f64p), _ptr(_d(U6).reshape(n, 6), f64p), _ptr(out, f64p))
    return out


def phase_sample_disney(C, dis, S6, wo, U4):
    U = _d(U4).reshape(-1, 4)
    n = U.shape[0]
    wi, w = np.zeros((n, 3)), np.zeros((n, 3))
    ok = np.zeros(n, np.int32)
    lib().orc_phase_sample_disney(_ptr(_d(C), f64p), _ptr(_d(dis), f64p), _ptr(_d(S6), f64p), _ptr(_d(wo), f64p), n,
                                  _ptr(U, f64p), _ptr(wi, f64p), _ptr(w, f64p), _ptr(ok, i32p))
    return wi, w, ok.astype(bool)


def phase_pdf_approx_disney(C, dis, S6, wo, wi):
    wi = _d(wi).reshape(-1, 3)
    out = np.zeros(wi.shape[0])
    lib().orc_phase_pdf_approx_disney(_ptr(_d(C), f64p), _ptr(_d(dis), f64p), _ptr(_d(S6), f64p), _ptr(_d(wo), f64p),
                                      wi.shape[0], _ptr(wi, f64p), _ptr(out, f64p))
    return out


def phase_sample(mtype, albedo, alpha, S6, wo, U4):
    albedo, S6, wo, U4 = _d(albedo), _d(S6), _d(wo), _d(U4).reshape(-1, 4)
    n = U4.shape[0]
    wi, w = np.zeros((n, 3)), np.zeros((n, 3))
    ok = np.zeros(n, np.int32)
    lib().orc_phase_sample(int(mtype), _ptr(albedo, f64p), float(alpha), _ptr(S6, f64p), _ptr(wo, f64p), n,
                           _ptr(U4, f64p), _ptr(wi, f64p), _ptr(w, f64p), _ptr(ok, i32p))
    return wi, w, ok.astype(bool)


def phase_pdf_approx(mtype, albedo, alpha, S6, wo, wi):
    albedo, S6, wo, wi = _d(albedo), _d(S6), _d(wo), _d(wi).reshape(-1, 3)
    out = np.zeros(wi.shape[0])
    lib().orc_phase_pdf_approx(int(mtype), _ptr(albedo, f64p), float(alpha), _ptr(S6, f64p), _ptr(wo, f64p),
                               wi.shape[0], _ptr(wi, f64p), _ptr(out, f64p))
    return out


def render(scene, spp, max_depth=4, seed=0, spp_begin=0, cutoff_eps=0.01, nee=1, spawn_mode=0,
           pixels=None, threads=None, guide=None, guide_alpha=0.5, nee_emitters=0, accel=False,
           guide_min_roughness=0.0, rect=None):
    """Per-pixel sums of sample values and squares, shape (H, W, 3) each, plus query counts.

    ``pixels`` = (p_begin, p_end) renders only that row-major pixel range (others stay zero).
    ``rect`` = (x0, y0, w, h) renders only that rectangle of pixels (instead of ``pixels``).
    ``guide`` = (params, GuideConfig) renders with the learned guide by one-sample MIS.
    ``nee_emitters`` = 1 adds next-event estimation toward emissive primitives (with MIS).
    ``accel`` finds each ray's intervals with a BVH instead of testing every primitive: the same
    intervals and results, for timing large scenes.
    """
    cam, li = scene.camera, scene.lights
    W, H = cam.width, cam.height
    c = OrcCamera((C.c_float * 3)(*cam.eye), (C.c_float * 3)(*cam.look), (C.c_float * 3)(*cam.up),
                  cam.vfov_deg, W, H)
    l = OrcLights(int(li.has_quad), (C.c_float * 3)(*li.quad_corner), (C.c_float * 3)(*li.quad_e1),
                  (C.c_float * 3)(*li.quad_e2), (C.c_float * 3)(*li.quad_Le), (C.c_float * 3)(*li.bg))
    gp = None
    gcfg = OrcGuideCfg()
    if guide is not None:
        gp = _c(guide[0], np.float32)
        gcfg = _guide_cfg(guide[1])
    p = OrcParams(int(spp), int(spp_begin), int(max_depth), int(seed), float(cutoff_eps), int(nee),
                  int(spawn_mode), _ptr(gp, f32p), gcfg, float(guide_alpha), int(nee_emitters), int(bool(accel)),
                  float(guide_min_roughness), 0, 0)
    acc = np.zeros((H, W, 3))
    acc2 = np.zeros((H, W, 3))
    counts = (C.c_int64 * 2)(0, 0)
    pb, pe = (0, W * H) if pixels is None else pixels
    if rect is not None:
        x0, y0, rw, rh = (int(v) for v in rect)
        if not (0 <= x0 and 0 <= y0 and rw > 0 and rh > 0 and x0 + rw <= W and y0 + rh <= H):
            raise ValueError(f"rect {rect} outside the {W}x{H} image")
        pb, pe = y0 * W, (y0 + rh) * W
        p.crop_x0, p.crop_x1 = x0, x0 + rw
    sr = _SceneRef(scene)
    if threads:
        set_num_threads(threads)
    lib().orc_render(sr.ref, C.byref(c), C.byref(l), C.byref(p), int(pb), int(pe), _ptr(acc, f64p),
                     _ptr(acc2, f64p), counts)
    return acc, acc2, (int(counts[0]), int(counts[1]))


def sample_in_ellipsoid(scene, i, U3, eps=0.01):
    """Points of primitive i drawn from its Gaussian restricted to the k-ellipsoid (n x 3 uniforms)."""
    U = _d(U3).reshape(-1, 3)
    y = np.zeros_like(U)
    lib().orc_sample_in_ellipsoid(_SceneRef(scene).ref, int(i), float(eps), U.shape[0], _ptr(U, f64p), _ptr(y, f64p))
    return y


def emitter_nee(scene, x, wo, mtype, albedo, alpha, S6, n, seed=0, exclude=-1, eps=0.01):
    """Mean and standard error (per RGB channel) of n one-sample light estimates toward the
    scene's emissive primitives at vertex x (outgoing wo, the given material), without MIS."""
    sm, sq = np.zeros(3), np.zeros(3)
    lib().orc_emitter_nee(_SceneRef(scene).ref, float(eps), _ptr(_d(x), f64p), _ptr(_d(wo), f64p), int(exclude),
                          int(mtype), _ptr(_d(albedo), f64p), float(alpha), _ptr(_d(S6), f64p), int(n), int(seed),
                          _ptr(sm, f64p), _ptr(sq, f64p))
    mean = sm / n
    return mean, np.sqrt(np.maximum(sq / n - mean ** 2, 0.0) / n)


def chi3_cdf(r: float) -> float:
    return float(lib().orc_chi3_cdf(float(r)))


# ------------------------------------------------------------------ learned guide
def _register_guide(L):
    d = f64p
    L.orc_guide_nparams.restype = C.c_int64
    L.orc_bf16_round.argtypes = [C.c_int64, d, d]
    L.orc_guide_encode.argtypes = [C.POINTER(OrcGuideCfg), C.c_int64, f32p, f32p, d]
    L.orc_guide_forward.argtypes = [C.POINTER(OrcGuideCfg), f32p, C.c_int64, f32p, f32p, d, d]
    L.orc_mixture_pdf.argtypes = [C.c_int64, d, d, d]
    L.orc_mixture_sample.argtypes = [C.c_int64, d, d, d, d]
    L.orc_mixture_loss_grad.argtypes = [C.POINTER(OrcGuideCfg), d, d, C.c_double, d]
    L.orc_mixture_loss_grad.restype = C.c_double
    L.orc_guide_loss_grad.argtypes = [C.POINTER(OrcGuideCfg), f32p, C.c_int64, f32p, f32p, f32p, f32p, d]
    L.orc_guide_loss_grad.restype = C.c_double
    L.orc_adam_step.argtypes = [C.c_int64, d, d, d, d, C.c_int64, C.c_double, C.c_double, C.c_double,
                                C.c_double]


_REGISTRY.append(_register_guide)


def _guide_cfg(cfg, round_bf16=None):
    """OrcGuideCfg from an object with pos_lo, pos_hi, kappa_min, kappa_max (and round_bf16)."""
    rb = getattr(cfg, "round_bf16", 1) if round_bf16 is None else round_bf16
    return OrcGuideCfg((C.c_double * 3)(*cfg.pos_lo), (C.c_double * 3)(*cfg.pos_hi), float(cfg.kappa_min),
                       float(cfg.kappa_max), int(rb))


def guide_nparams() -> int:
    return int(lib().orc_guide_nparams())


def bf16_round(x):
    x = _d(x)
    out = np.zeros_like(x)
    lib().orc_bf16_round(x.size, _ptr(x, f64p), _ptr(out, f64p))
    return out


def guide_encode(cfg, x3, wo3, round_bf16=None):
    x3, wo3 = _c(x3, np.float32).reshape(-1, 3), _c(wo3, np.float32).reshape(-1, 3)
    n = x3.shape[0]
    out = np.zeros((n, 64))
    g = _guide_cfg(cfg, round_bf16)
    lib().orc_guide_encode(C.byref(g), n, _ptr(x3, f32p), _ptr(wo3, f32p), _ptr(out, f64p))
    return out


def guide_forward(cfg, params, x3, wo3, round_bf16=None):
    """(Y, mix): head outputs (n, 40) and mixture (n, 8, 5) = per lobe (mu xyz, kappa, pi)."""
    params = _c(params, np.float32)
    x3, wo3 = _c(x3, np.float32).reshape(-1, 3), _c(wo3, np.float32).reshape(-1, 3)
    n = x3.shape[0]
    Y = np.zeros((n, 40))
    mix = np.zeros((n, 40))
    g = _guide_cfg(cfg, round_bf16)
    lib().orc_guide_forward(C.byref(g), _ptr(params, f32p), n, _ptr(x3, f32p), _ptr(wo3, f32p), _ptr(Y, f64p),
                            _ptr(mix, f64p))
    return Y, mix.reshape(n, 8, 5)


def mixture_pdf(mix, wi3):
    mix = _d(mix).reshape(-1, 40)
    wi3 = _d(wi3).reshape(-1, 3)
    out = np.zeros(mix.shape[0])
    lib().orc_mixture_pdf(mix.shape[0], _ptr(mix, f64p), _ptr(wi3, f64p), _ptr(out, f64p))
    return out


def mixture_sample(mix, U3):
    mix = _d(mix).reshape(-1, 40)
    U3 = _d(U3).reshape(-1, 3)
    n = mix.shape[0]
    wi, pdf = np.zeros((n, 3)), np.zeros(n)
    lib().orc_mixture_sample(n, _ptr(mix, f64p), _ptr(U3, f64p), _ptr(wi, f64p), _ptr(pdf, f64p))
    return wi, pdf


def mixture_loss_grad(cfg, Y, wi, w):
    Y, wi = _d(Y), _d(wi)
    dY = np.zeros(40)
    g = _guide_cfg(cfg)
    loss = lib().orc_mixture_loss_grad(C.byref(g), _ptr(Y, f64p), _ptr(wi, f64p), float(w), _ptr(dY, f64p))
    return float(loss), dY


def guide_loss_grad(cfg, params, x3, wo3, wi3, weight, round_bf16=None):
    """(mean loss, gradient of the mean loss over the flat parameters)."""
    params = _c(params, np.float32)
    x3, wo3, wi3 = (_c(a, np.float32).reshape(-1, 3) for a in (x3, wo3, wi3))
    weight = _c(weight, np.float32)
    grad = np.zeros(guide_nparams())
    g = _guide_cfg(cfg, round_bf16)
    loss = lib().orc_guide_loss_grad(C.byref(g), _ptr(params, f32p), x3.shape[0], _ptr(x3, f32p), _ptr(wo3, f32p),
                                     _ptr(wi3, f32p), _ptr(weight, f32p), _ptr(grad, f64p))
    return float(loss), grad


def adam_step(theta, m, v, g, t, lr=1e-3, b1=0.9, b2=0.99, eps=1e-8):
    """One Adam step in place on FP64 copies; returns (theta, m, v)."""
    theta, m, v, g = _d(theta).copy(), _d(m).copy(), _d(v).copy(), _d(g)
    lib().orc_adam_step(theta.size, _ptr(theta, f64p), _ptr(m, f64p), _ptr(v, f64p), _ptr(g, f64p), int(t),
                        float(lr), float(b1), float(b2), float(eps))
    return theta, m, v
