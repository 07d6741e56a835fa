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
                ("roughness", f32p), ("emission3", f32p)]


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
                                             f64p, f64p, i32p]
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
        a = self.arrs
        self.s = OrcScene(scene.n, _ptr(a["mean"], f32p), _ptr(a["quat"], f32p),
                          _ptr(a["scale"], f32p), _ptr(a["mag"], f32p), _ptr(a["sggx"], f32p),
                          _ptr(a["type"], u8p), _ptr(a["albedo"], f32p), _ptr(a["rough"], f32p),
                          _ptr(a["emit"], f32p))

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
    lib().orc_sample_free_flight(sr.ref, eps, n, _ptr(o, f32p), _ptr(d, f32p), _ptr(t0, f32p),
                                 _ptr(t1, f32p), _ptr(ex, i32p), _ptr(u, f32p), _ptr(u2, f32p),
                                 _ptr(prim, i32p), _ptr(tu, f64p), _ptr(ts, f64p), _ptr(fe, f64p),
                                 _ptr(na, i32p))
    return dict(prim=prim, t_u=tu, t_spawn=ts, F_end=fe, n_active=na)


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
