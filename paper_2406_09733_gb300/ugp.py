"""Thin Python binding of the ugp C ABI (``include/ugp.h``).

Argument marshalling only: tensors are checked for device, dtype and
contiguity, outputs are allocated with torch, and raw device pointers plus the
current CUDA stream are handed to ``libugp.so``.  Every step of the hot path
runs in the library's CUDA kernels; there is no fallback of any kind, and
loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

_LIB = None
vp = C.c_void_p


class UgpPrims(C.Structure):
    _fields_ = [("n", C.c_int64), ("mean3", vp), ("quat4", vp), ("scale3", vp), ("magnitude", vp)]


class UgpBvhInfo(C.Structure):
    _fields_ = [("n_prims", C.c_int64), ("n_nodes", C.c_int64), ("cutoff_k", C.c_float),
                ("bounds_lo", C.c_float * 3), ("bounds_hi", C.c_float * 3),
                ("persistent_bytes", C.c_size_t), ("n_invalid", C.c_int64)]


class UgpMaterials(C.Structure):
    _fields_ = [("sggx6", vp), ("type", vp), ("albedo3", vp), ("roughness", vp), ("emission3", vp),
                ("disney9", vp)]


class UgpCamera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class UgpLights(C.Structure):
    _fields_ = [("has_quad", C.c_int32), ("quad_corner", C.c_float * 3), ("quad_e1", C.c_float * 3),
                ("quad_e2", C.c_float * 3), ("quad_Le", C.c_float * 3), ("bg", C.c_float * 3)]


class UgpGuide(C.Structure):
    _fields_ = [("params", vp), ("adam_m", vp), ("adam_v", vp), ("step", C.c_int64), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("pos_lo", C.c_float * 3),
                ("pos_hi", C.c_float * 3), ("kappa_min", C.c_float), ("kappa_max", C.c_float),
                ("train_target", C.c_int32)]


class UgpRenderParams(C.Structure):
    _fields_ = [("spp", C.c_int32), ("spp_begin", C.c_int32), ("max_depth", C.c_int32),
                ("nee", C.c_int32), ("seed", C.c_uint64), ("spawn_mode", C.c_int32),
                ("guide_log", C.c_int32), ("guide", C.POINTER(UgpGuide)), ("guide_alpha", C.c_float),
                ("guide_min_roughness", C.c_float), ("emitters", C.c_void_p)]


class UgpError(RuntimeError):
    pass


RAY_OK, RAY_STACK_OVERFLOW, RAY_BUFFER_OVERFLOW, RAY_ITER_LIMIT, RAY_BAD_NODE, RAY_SOLVE_LIMIT = 0, 1, 2, 3, 4, 5


def lib():
    """Loads ``libugp.so`` (built in-tree by ``build.build()``)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.LIB):
            raise UgpError(f"CUDA library not built: {_build.LIB} is missing "
                           "(run __graft_entry__.build())")
        L = C.CDLL(_build.LIB)
        L.ugp_status_string.restype = C.c_char_p
        L.ugp_status_string.argtypes = [C.c_int]
        L.ugp_last_error.restype = C.c_char_p
        L.ugp_version.restype = C.c_char_p
        L.ugp_build_bvh_workspace_size.restype = C.c_size_t
        L.ugp_build_bvh_workspace_size.argtypes = [C.c_int64]
        L.ugp_build_bvh.restype = C.c_int
        L.ugp_build_bvh.argtypes = [C.POINTER(UgpPrims), C.c_float, vp, C.c_size_t, vp,
                                    C.POINTER(vp)]
        L.ugp_bvh_release.argtypes = [vp]
        L.ugp_bvh_release.restype = None
        L.ugp_bvh_get_info.restype = C.c_int
        L.ugp_bvh_get_info.argtypes = [vp, C.POINTER(UgpBvhInfo)]
        L.ugp_trace_transmittance.restype = C.c_int
        L.ugp_trace_transmittance.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp]
        L.ugp_sample_free_flight.restype = C.c_int
        L.ugp_sample_free_flight.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                             vp, vp, C.c_size_t, vp]
        L.ugp_sample_free_flight_workspace_size.restype = C.c_size_t
        L.ugp_sample_free_flight_workspace_size.argtypes = [C.c_int64]
        L.ugp_collect_hits.restype = C.c_int
        L.ugp_collect_hits.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, C.c_int32, vp, vp, vp,
                                       vp, vp, vp]
        L.ugp_render_workspace_size.restype = C.c_size_t
        L.ugp_render_workspace_size.argtypes = [C.c_int32, C.c_int32]
        L.ugp_render.restype = C.c_int
        L.ugp_render.argtypes = [vp, C.POINTER(UgpMaterials), C.POINTER(UgpCamera),
                                 C.POINTER(UgpLights), C.POINTER(UgpRenderParams), vp, vp, vp,
                                 C.c_size_t, vp, vp]
        L.ugp_profile_begin.restype = C.c_int
        L.ugp_profile_begin.argtypes = [C.c_int32]
        L.ugp_profile_end.restype = C.c_int
        L.ugp_profile_end.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.ugp_launch_count.restype = C.c_int64
        L.ugp_render_radiance_field_workspace_size.restype = C.c_size_t
        L.ugp_render_radiance_field_workspace_size.argtypes = [C.c_int64]
        L.ugp_render_radiance_field.restype = C.c_int
        L.ugp_render_radiance_field.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, C.POINTER(C.c_float), vp, vp, vp,
                                                C.c_size_t, vp]
        L.ugp_emitter_table_size.restype = C.c_size_t
        L.ugp_emitter_table_size.argtypes = [C.c_int64]
        L.ugp_build_emitter_table.restype = C.c_int
        L.ugp_build_emitter_table.argtypes = [vp, vp, vp, C.c_size_t, vp]
        L.ugp_sample_free_flight_exponential.restype = C.c_int
        L.ugp_sample_free_flight_exponential.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.ugp_trace_transmittance_exponential.restype = C.c_int
        L.ugp_trace_transmittance_exponential.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp]
        L.ugp_build_kdtree_workspace_size.restype = C.c_size_t
        L.ugp_build_kdtree_workspace_size.argtypes = [C.c_int64]
        L.ugp_build_kdtree.restype = C.c_int
        L.ugp_build_kdtree.argtypes = [vp, vp, C.c_size_t, vp, C.POINTER(vp)]
        L.ugp_kdtree_release.restype = None
        L.ugp_kdtree_release.argtypes = [vp]
        L.ugp_kdtree_get_info.restype = C.c_int
        L.ugp_kdtree_get_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                          C.POINTER(C.c_float)]
        L.ugp_kdtree_export.restype = C.c_int
        L.ugp_kdtree_export.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.ugp_sample_free_flight_kdtree.restype = C.c_int
        L.ugp_sample_free_flight_kdtree.argtypes = [vp, C.c_int64] + [vp] * 10 + [vp]
        L.ugp_codebook_size.restype = C.c_size_t
        L.ugp_codebook_size.argtypes = []
        L.ugp_codebook_workspace_size.restype = C.c_size_t
        L.ugp_codebook_workspace_size.argtypes = [C.c_int64]
        L.ugp_codebook_encode.restype = C.c_int
        L.ugp_codebook_encode.argtypes = [C.POINTER(UgpPrims), C.POINTER(UgpMaterials), C.c_int32, vp, vp, vp,
                                          C.c_size_t, vp]
        L.ugp_codebook_decode.restype = C.c_int
        L.ugp_codebook_decode.argtypes = [C.c_int64] + [vp] * 13
        L.ugp_phase_query.restype = C.c_int
        L.ugp_phase_query.argtypes = [C.c_int64] + [vp] * 15
        L.ugp_set_trace_counters.restype = C.c_int
        L.ugp_set_trace_counters.argtypes = [vp]
        for fn in _EXTRA:
            fn(L)
        _LIB = L
    return _LIB


_EXTRA = []


def _check(status: int, what: str):
    if status != 0:
        L = lib()
        raise UgpError(f"{what}: {L.ugp_status_string(status).decode()} "
                       f"({L.ugp_last_error().decode()})")


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev(t, dtype, name, shape_last=None, n=None, device=None, cuda=True):
    """Checks a tensor handed to the library: dtype, contiguous; with `shape_last`, shape
    (rows, shape_last); with `n`, exactly n rows (n elements for a flat array); with `device`,
    that device; with `cuda`, a CUDA tensor. The kernels index every per-ray array up to n, so a
    short array would be read past its end on the device."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_last is not None and (t.dim() != 2 or t.shape[1] != shape_last):
        raise ValueError(f"{name} must have shape (n, {shape_last})")
    if n is not None:
        rows = t.shape[0] if shape_last is not None else t.numel()
        if rows != n:
            raise ValueError(f"{name} must hold {n} {'rows' if shape_last is not None else 'elements'}, got {rows}")
    if device is not None and t.device != torch.device(device):
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if cuda and not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    return t


def _rays(o, d, t0, t1, exclude=None, **more):
    """Validates a batch of rays (o, d: (n, 3); t0, t1 and the optional per-ray arrays: n
    elements, all float32 except `exclude` (int32), all on o's device). Returns n."""
    _dev(o, torch.float32, "o", 3, cuda=False)
    n = int(o.shape[0])
    checks = [(d, torch.float32, "d", 3), (t0, torch.float32, "t0", None), (t1, torch.float32, "t1", None),
              (exclude, torch.int32, "exclude", None)] + [(t, torch.float32, nm, None) for nm, t in more.items()]
    for t, dt, nm, last in checks:           # sizes and devices first, so that a short array is
        _dev(t, dt, nm, last, n=n, device=o.device, cuda=False)   # named even on a host tensor
    _dev(o, torch.float32, "o", 3)
    for t, dt, nm, last in checks:
        _dev(t, dt, nm, last)
    return n


def _workspace(workspace, nbytes, device):
    """The caller's workspace after the same checks as every other device argument (a uint8 CUDA
    tensor on `device`), or a new one when none is given or it is too small."""
    if workspace is not None:
        _dev(workspace, torch.uint8, "workspace", device=device)
        if workspace.numel() >= nbytes:
            return workspace
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Bvh:
    """A built BVH: the library handle plus the workspace tensor that holds it."""

    def __init__(self, handle: int, workspace: torch.Tensor, n: int, inputs):
        self.handle = handle
        self.workspace = workspace
        self.n = n
        self._inputs = inputs  # keep the primitive arrays alive while the build runs

    def info(self) -> dict:
        inf = UgpBvhInfo()
        _check(lib().ugp_bvh_get_info(C.c_void_p(self.handle), C.byref(inf)), "ugp_bvh_get_info")
        return dict(n_prims=inf.n_prims, n_nodes=inf.n_nodes, cutoff_k=inf.cutoff_k,
                    bounds_lo=list(inf.bounds_lo), bounds_hi=list(inf.bounds_hi),
                    persistent_bytes=inf.persistent_bytes, n_invalid=inf.n_invalid)

    def release(self):
        if self.handle:
            lib().ugp_bvh_release(C.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def build_bvh_workspace_size(n: int) -> int:
    return int(lib().ugp_build_bvh_workspace_size(int(n)))


def build_bvh(mean, quat, scale, magnitude, cutoff_eps: float = 0.01, stream=None, workspace=None) -> Bvh:
    """Builds the BVH; `workspace` (uint8 CUDA tensor) is reused when given and large enough."""
    n = int(mean.shape[0])
    _dev(mean, torch.float32, "mean", 3)
    _dev(quat, torch.float32, "quat", 4, n=n, device=mean.device)
    _dev(scale, torch.float32, "scale", 3, n=n, device=mean.device)
    _dev(magnitude, torch.float32, "magnitude", n=n, device=mean.device)
    ws_bytes = build_bvh_workspace_size(n)
    if ws_bytes == 0:
        raise UgpError("ugp_build_bvh_workspace_size failed")
    if workspace is not None:
        _dev(workspace, torch.uint8, "workspace", device=mean.device)
        if workspace.numel() < ws_bytes:
            raise ValueError(f"workspace needs {ws_bytes} bytes")
        ws = workspace
    else:
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=mean.device)
    prims = UgpPrims(n, _p(mean), _p(quat), _p(scale), _p(magnitude))
    h = vp()
    _check(lib().ugp_build_bvh(C.byref(prims), float(cutoff_eps), _p(ws), ws_bytes,
                               C.c_void_p(_stream(stream)), C.byref(h)), "ugp_build_bvh")
    return Bvh(h.value, ws, n, (mean, quat, scale, magnitude))


def trace_transmittance(bvh: Bvh, o, d, t0, t1, exclude=None, stream=None):
    n = _rays(o, d, t0, t1, exclude)
    T = torch.empty(n, dtype=torch.float32, device=o.device)
    st = torch.empty(n, dtype=torch.uint8, device=o.device)
    _check(lib().ugp_trace_transmittance(C.c_void_p(bvh.handle), n, _p(o), _p(d), _p(t0), _p(t1),
                                         _p(exclude), _p(T), _p(st), C.c_void_p(_stream(stream))),
           "ugp_trace_transmittance")
    return T, st


def sample_free_flight(bvh: Bvh, o, d, t0, t1, u, u2, exclude=None, stream=None, workspace=None):
    n = _rays(o, d, t0, t1, exclude, u=u, u2=u2)
    nb = int(lib().ugp_sample_free_flight_workspace_size(n))
    workspace = _workspace(workspace, nb, o.device)
    prim = torch.empty(n, dtype=torch.int32, device=o.device)
    tu = torch.empty(n, dtype=torch.float32, device=o.device)
    tsp = torch.empty(n, dtype=torch.float32, device=o.device)
    st = torch.empty(n, dtype=torch.uint8, device=o.device)
    _check(lib().ugp_sample_free_flight(C.c_void_p(bvh.handle), n, _p(o), _p(d), _p(t0), _p(t1),
                                        _p(u), _p(u2), _p(exclude), _p(prim), _p(tu), _p(tsp),
                                        _p(st), _p(workspace), workspace.numel(),
                                        C.c_void_p(_stream(stream))),
           "ugp_sample_free_flight")
    return prim, tu, tsp, st


def render_radiance_field(bvh: Bvh, o, d, t0, t1, emission, background=None, stream=None, workspace=None):
    """Radiance-field forward render (Sec. 7, Eq. rf): per ray the emission-weighted 1/2 I of
    every primitive clipped at the saturating distance, plus the unsaturated remainder times
    the background. Returns (rgb (n, 3), status (n,))."""
    n = _rays(o, d, t0, t1)
    nb = int(lib().ugp_render_radiance_field_workspace_size(n))
    workspace = _workspace(workspace, nb, o.device)
    _dev(emission, torch.float32, "emission", 3, n=bvh.n, device=o.device)
    rgb = torch.empty((n, 3), dtype=torch.float32, device=o.device)
    st = torch.empty(n, dtype=torch.uint8, device=o.device)
    bg = None if background is None else (C.c_float * 3)(*[float(x) for x in background])
    _check(lib().ugp_render_radiance_field(C.c_void_p(bvh.handle), n, _p(o), _p(d), _p(t0), _p(t1), _p(emission),
                                           bg, _p(rgb), _p(st), _p(workspace), workspace.numel(),
                                           C.c_void_p(_stream(stream))),
           "ugp_render_radiance_field")
    return rgb, st


def sample_free_flight_exponential(bvh: Bvh, o, d, t0, t1, u, exclude=None, stream=None):
    """Exponential variant by analog decomposition tracking (sigma_t = sum_k G_k): per ray the
    nearest per-primitive exponential collision keyed by the uniform u. Returns (prim (-1:
    escape), t (t1 on escape), status)."""
    n = _rays(o, d, t0, t1, exclude, u=u)
    prim = torch.empty(n, dtype=torch.int32, device=o.device)
    t = torch.empty(n, dtype=torch.float32, device=o.device)
    st = torch.empty(n, dtype=torch.uint8, device=o.device)
    _check(lib().ugp_sample_free_flight_exponential(C.c_void_p(bvh.handle), n, _p(o), _p(d), _p(t0), _p(t1), _p(u),
                                                    _p(exclude), _p(prim), _p(t), _p(st),
                                                    C.c_void_p(_stream(stream))),
           "ugp_sample_free_flight_exponential")
    return prim, t, st


def trace_transmittance_exponential(bvh: Bvh, o, d, t0, t1, exclude=None, stream=None):
    """exp(-sum_k I_k) over each ray's [t0, t1] (exponential variant). Returns (T, status)."""
    n = _rays(o, d, t0, t1, exclude)
    T = torch.empty(n, dtype=torch.float32, device=o.device)
    st = torch.empty(n, dtype=torch.uint8, device=o.device)
    _check(lib().ugp_trace_transmittance_exponential(C.c_void_p(bvh.handle), n, _p(o), _p(d), _p(t0), _p(t1),
                                                     _p(exclude), _p(T), _p(st), C.c_void_p(_stream(stream))),
           "ugp_trace_transmittance_exponential")
    return T, st


def phase_query(mtype, albedo3, roughness, sggx6, wo3, wi3, u_eval6, u_sample4, disney9=None, stream=None):
    """Phase-function queries on independent records (Sec. 6, App. B): returns (eval (n, 3),
    App. B pdf (n,), sampled wi (n, 3), sample weight (n, 3), sample ok (n,) uint8)."""
    _dev(mtype, torch.uint8, "type", cuda=False)
    n, dev = int(mtype.numel()), mtype.device
    for t, nm, last in ((albedo3, "albedo3", 3), (roughness, "roughness", None), (sggx6, "sggx6", 6),
                        (disney9, "disney9", 9), (wo3, "wo3", 3), (wi3, "wi3", 3), (u_eval6, "u_eval6", 6),
                        (u_sample4, "u_sample4", 4)):
        _dev(t, torch.float32, nm, last, n=n, device=dev)
    _dev(mtype, torch.uint8, "type")
    ev = torch.empty((n, 3), dtype=torch.float32, device=dev)
    pdf = torch.empty(n, dtype=torch.float32, device=dev)
    swi = torch.empty((n, 3), dtype=torch.float32, device=dev)
    sw = torch.empty((n, 3), dtype=torch.float32, device=dev)
    ok = torch.empty(n, dtype=torch.uint8, device=dev)
    _check(lib().ugp_phase_query(n, _p(mtype), _p(albedo3), _p(roughness), _p(sggx6), _p(disney9), _p(wo3),
                                 _p(wi3), _p(u_eval6), _p(u_sample4), _p(ev), _p(pdf), _p(swi), _p(sw), _p(ok),
                                 C.c_void_p(_stream(stream))), "ugp_phase_query")
    return ev, pdf, swi, sw, ok


class KdTree:
    """The paper's SAH kd-tree over a built BVH's primitives (the comparison sampler's structure)."""

    def __init__(self, bvh: Bvh, stream=None):
        nb = int(lib().ugp_build_kdtree_workspace_size(int(bvh.n)))
        if nb == 0:
            raise UgpError("ugp_build_kdtree_workspace_size failed")
        self.bvh = bvh
        self.workspace = torch.empty(nb, dtype=torch.uint8, device=bvh.workspace.device)
        h = vp()
        _check(lib().ugp_build_kdtree(C.c_void_p(bvh.handle), _p(self.workspace), nb, C.c_void_p(_stream(stream)),
                                      C.byref(h)), "ugp_build_kdtree")
        self.handle = h.value

    def info(self) -> dict:
        nn, nr, dp = C.c_int64(), C.c_int64(), C.c_int32()
        box = (C.c_float * 6)()
        _check(lib().ugp_kdtree_get_info(C.c_void_p(self.handle), C.byref(nn), C.byref(nr), C.byref(dp), box),
               "ugp_kdtree_get_info")
        return dict(n_nodes=nn.value, n_refs=nr.value, depth=dp.value, box=list(box))

    def export(self):
        """(nodes (m, 4) int32, refs int32 primitive indices, root box (6,) float32) on the host."""
        import numpy as np
        inf = self.info()
        nodes = np.zeros((inf["n_nodes"], 4), np.int32)
        refs = np.zeros(inf["n_refs"], np.int32)
        i32 = C.POINTER(C.c_int32)
        _check(lib().ugp_kdtree_export(C.c_void_p(self.handle), nodes.ctypes.data_as(i32), refs.ctypes.data_as(i32)),
               "ugp_kdtree_export")
        return nodes, refs, np.array(inf["box"], np.float32)

    def sample_free_flight(self, o, d, t0, t1, u, u2, exclude=None, stream=None):
        """(prim (-1: escape), t_spawn, status) of the paper's sampler."""
        n = _rays(o, d, t0, t1, exclude, u=u, u2=u2)
        prim = torch.empty(n, dtype=torch.int32, device=o.device)
        tsp = torch.empty(n, dtype=torch.float32, device=o.device)
        st = torch.empty(n, dtype=torch.uint8, device=o.device)
        _check(lib().ugp_sample_free_flight_kdtree(C.c_void_p(self.handle), n, _p(o), _p(d), _p(t0), _p(t1), _p(u),
                                                   _p(u2), _p(exclude), _p(prim), _p(tsp), _p(st),
                                                   C.c_void_p(_stream(stream))), "ugp_sample_free_flight_kdtree")
        return prim, tsp, st

    def release(self):
        if getattr(self, "handle", 0):
            lib().ugp_kdtree_release(C.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


CODEBOOK_ENTRIES, CODEBOOK_FEATURES, RECORD_BYTES = 4096, 29, 24


def codebook_encode(mean, quat, scale, magnitude, mats: "Materials", iters: int = 8, stream=None):
    """Codebook-quantised records of a scene: returns (codebook (4096, 29) float32, records
    (n, 24) uint8)."""
    n = int(mean.shape[0])
    dev = mean.device
    _dev(mean, torch.float32, "mean", 3)
    _dev(quat, torch.float32, "quat", 4, n=n, device=dev)
    _dev(scale, torch.float32, "scale", 3, n=n, device=dev)
    _dev(magnitude, torch.float32, "magnitude", n=n, device=dev)
    if mats.n != n or mats.device != dev:
        raise ValueError("materials must describe the same primitives on the same device")
    book = torch.empty((CODEBOOK_ENTRIES, CODEBOOK_FEATURES), dtype=torch.float32, device=dev)
    rec = torch.empty((n, RECORD_BYTES), dtype=torch.uint8, device=dev)
    ws = torch.empty(max(int(lib().ugp_codebook_workspace_size(n)), 256), dtype=torch.uint8, device=dev)
    prims = UgpPrims(n, _p(mean), _p(quat), _p(scale), _p(magnitude))
    _check(lib().ugp_codebook_encode(C.byref(prims), C.byref(mats.c), int(iters), _p(book), _p(rec), _p(ws),
                                     ws.numel(), C.c_void_p(_stream(stream))), "ugp_codebook_encode")
    return book, rec


def codebook_decode(records, codebook, disney=True, stream=None):
    """Decodes records into a dict of the scene arrays (mean, quat, scale, magnitude, sggx, mtype,
    albedo, roughness, emission, disney)."""
    _dev(records, torch.uint8, "records", RECORD_BYTES)
    n, dev = int(records.shape[0]), records.device
    _dev(codebook, torch.float32, "codebook", CODEBOOK_FEATURES, n=CODEBOOK_ENTRIES, device=dev)
    f = lambda *shape: torch.empty(shape, dtype=torch.float32, device=dev)
    out = dict(mean=f(n, 3), quat=f(n, 4), scale=f(n, 3), magnitude=f(n), sggx=f(n, 6),
               mtype=torch.empty(n, dtype=torch.uint8, device=dev), albedo=f(n, 3), roughness=f(n),
               emission=f(n, 3), disney=f(n, 9) if disney else None)
    _check(lib().ugp_codebook_decode(n, _p(records), _p(codebook), _p(out["mean"]), _p(out["quat"]),
                                     _p(out["scale"]), _p(out["magnitude"]), _p(out["sggx"]), _p(out["mtype"]),
                                     _p(out["albedo"]), _p(out["roughness"]), _p(out["emission"]),
                                     _p(out["disney"]), C.c_void_p(_stream(stream))), "ugp_codebook_decode")
    return out


def collect_hits(bvh: Bvh, o, d, t0, t1, cap: int, exclude=None, stream=None):
    """All clipped intervals per ray: (ids, a, b) of shape (n, cap), count (n,), status."""
    n = _rays(o, d, t0, t1, exclude)
    ids = torch.full((n, cap), -1, dtype=torch.int32, device=o.device)
    a = torch.zeros((n, cap), dtype=torch.float32, device=o.device)
    b = torch.zeros((n, cap), dtype=torch.float32, device=o.device)
    cnt = torch.empty(n, dtype=torch.int32, device=o.device)
    st = torch.empty(n, dtype=torch.uint8, device=o.device)
    _check(lib().ugp_collect_hits(C.c_void_p(bvh.handle), n, _p(o), _p(d), _p(t0), _p(t1),
                                  _p(exclude), int(cap), _p(ids), _p(a), _p(b), _p(cnt), _p(st),
                                  C.c_void_p(_stream(stream))), "ugp_collect_hits")
    return ids, a, b, cnt, st


class Materials:
    """Device copies of the per-primitive appearance arrays (kept alive with the struct).
    ``disney9`` ((n, 9) float32 or None) holds the Disney parameters of type-3 primitives."""

    def __init__(self, sggx6, mtype, albedo3, roughness, emission3, disney9=None):
        _dev(sggx6, torch.float32, "sggx6", 6)
        n, dev = int(sggx6.shape[0]), sggx6.device
        _dev(mtype, torch.uint8, "type", n=n, device=dev)
        _dev(albedo3, torch.float32, "albedo3", 3, n=n, device=dev)
        _dev(roughness, torch.float32, "roughness", n=n, device=dev)
        _dev(emission3, torch.float32, "emission3", 3, n=n, device=dev)
        _dev(disney9, torch.float32, "disney9", 9, n=n, device=dev)
        self.n, self.device = n, dev
        self.tensors = (sggx6, mtype, albedo3, roughness, emission3, disney9)
        self.c = UgpMaterials(*[_p(t) for t in self.tensors])


def camera_struct(eye, look, up, vfov_deg, width, height) -> UgpCamera:
    return UgpCamera((C.c_float * 3)(*eye), (C.c_float * 3)(*look), (C.c_float * 3)(*up),
                     float(vfov_deg), int(width), int(height))


def lights_struct(has_quad=False, corner=(0, 0, 0), e1=(0, 0, 0), e2=(0, 0, 0), Le=(0, 0, 0),
                  bg=(0, 0, 0)) -> UgpLights:
    f3 = lambda v: (C.c_float * 3)(*v)
    return UgpLights(int(bool(has_quad)), f3(corner), f3(e1), f3(e2), f3(Le), f3(bg))


def scene_to_device(scene, device="cuda", cutoff_eps: float = 0.01):
    """Uploads a ``scenes.Scene`` and builds its BVH: returns (bvh, materials, camera, lights)."""
    t = lambda a: torch.from_numpy(__import__("numpy").ascontiguousarray(a)).to(device)
    bvh = build_bvh(t(scene.mean), t(scene.quat), t(scene.scale), t(scene.magnitude), cutoff_eps)
    dis = getattr(scene, "disney", None)
    mats = Materials(t(scene.sggx), t(scene.mtype), t(scene.albedo), t(scene.roughness), t(scene.emission),
                     None if dis is None else t(dis))
    cam = scene.camera
    li = scene.lights
    return (bvh, mats, camera_struct(cam.eye, cam.look, cam.up, cam.vfov_deg, cam.width, cam.height),
            lights_struct(li.has_quad, li.quad_corner, li.quad_e1, li.quad_e2, li.quad_Le, li.bg))


def render_workspace_size(width: int, height: int) -> int:
    return int(lib().ugp_render_workspace_size(int(width), int(height)))


class Renderer:
    """Reusable render workspace for one image size."""

    def __init__(self, width: int, height: int, device="cuda"):
        self.width, self.height = int(width), int(height)
        nb = render_workspace_size(self.width, self.height)
        if nb == 0:
            raise UgpError("bad image size")
        self.workspace = torch.empty(nb, dtype=torch.uint8, device=device)
        self.guided_depth = None

    def render(self, bvh: Bvh, mats: Materials, camera: UgpCamera, lights: UgpLights, spp: int,
               max_depth: int, seed: int = 0, spp_begin: int = 0, nee: bool = True, spawn_mode: int = 0,
               accum=None, accum_sq=None, ray_counts=None, stream=None, guide=None, guide_alpha: float = 0.5,
               guide_log: bool = False, emitters=None, guide_min_roughness: float = 0.0):
        """Adds spp samples per pixel into accum / accum_sq ((H, W, 3) float32, created if None).

        With ``guide`` (a ``Guide``) the renderer samples directions by one-sample MIS between
        the guide and phase sampling; ``guide_log`` records the vertices for ``Guide.train_from``.
        ``emitters`` (from ``build_emitter_table``) adds light sampling of emissive primitives.
        """
        dev = self.workspace.device
        shape = (self.height, self.width, 3)
        if accum is None:
            accum = torch.zeros(shape, dtype=torch.float32, device=dev)
        if accum_sq is None:
            accum_sq = torch.zeros(shape, dtype=torch.float32, device=dev)
        _dev(accum, torch.float32, "accum", device=dev)
        _dev(accum_sq, torch.float32, "accum_sq", device=dev)
        if tuple(accum.shape) != shape or tuple(accum_sq.shape) != shape:
            raise ValueError(f"accumulators must have shape {shape}")
        if ray_counts is not None:
            _dev(ray_counts, torch.int64, "ray_counts", n=3, device=dev)
        _check_scene(bvh, mats, dev)
        if emitters is not None:
            _dev(emitters, torch.uint8, "emitters", device=dev)
        if camera.width != self.width or camera.height != self.height:
            raise ValueError("camera size does not match the renderer")
        prm = UgpRenderParams(int(spp), int(spp_begin), int(max_depth), int(bool(nee)), int(seed),
                              int(spawn_mode), int(bool(guide_log)),
                              C.pointer(guide.c) if guide is not None else None, float(guide_alpha),
                              float(guide_min_roughness),
                              emitters.data_ptr() if emitters is not None else None)
        if guide is not None:
            need = guided_workspace_size(self.width, self.height, max_depth)
            if self.workspace.numel() < need:
                self.workspace = torch.empty(need, dtype=torch.uint8, device=dev)
            self.guided_depth = int(max_depth)
        _check(lib().ugp_render(C.c_void_p(bvh.handle), C.byref(mats.c), C.byref(camera),
                                C.byref(lights), C.byref(prm), _p(accum), _p(accum_sq),
                                _p(self.workspace), self.workspace.numel(), _p(ray_counts),
                                C.c_void_p(_stream(stream))), "ugp_render")
        return accum, accum_sq


def _check_scene(bvh: Bvh, mats: "Materials", device):
    """The materials must describe the BVH's primitives and sit on the render's device."""
    if mats.n != bvh.n:
        raise ValueError(f"materials hold {mats.n} primitives, the BVH {bvh.n}")
    if mats.device != torch.device(device) or bvh.workspace.device != torch.device(device):
        raise ValueError(f"scene arrays must be on {device}")


def build_emitter_table(bvh: Bvh, mats, stream=None):
    """Device table for light sampling of the emissive primitives of ``bvh`` with materials
    ``mats`` (a ``Materials``): pass it to ``Renderer.render(emitters=...)``."""
    _check_scene(bvh, mats, bvh.workspace.device)
    nb = int(lib().ugp_emitter_table_size(int(bvh.n)))
    table = torch.empty(max(nb, 256), dtype=torch.uint8, device=bvh.workspace.device)
    _check(lib().ugp_build_emitter_table(C.c_void_p(bvh.handle), C.byref(mats.c), _p(table), table.numel(),
                                         C.c_void_p(_stream(stream))), "ugp_build_emitter_table")
    return table


def set_trace_counters(counters=None):
    """Turns traversal statistics on (a CUDA int64 tensor of 12 zeros) or off (None)."""
    if counters is not None:
        _dev(counters, torch.int64, "counters")
        if counters.numel() < 12:
            raise ValueError("counters needs 12 elements")
    _check(lib().ugp_set_trace_counters(_p(counters)), "ugp_set_trace_counters")


PROFILE_STAGES = ("build", "camera", "extend", "shade", "shadow", "accumulate", "query", "dense", "guide")


def profile_begin(max_records: int = 1 << 16):
    """Starts event timing of every library kernel launch (no synchronisation)."""
    _check(lib().ugp_profile_begin(int(max_records)), "ugp_profile_begin")


def profile_end():
    """Stops timing; returns {stage: (milliseconds, launches)} (waits for the recorded events)."""
    ms = (C.c_double * len(PROFILE_STAGES))()
    nl = (C.c_int64 * len(PROFILE_STAGES))()
    _check(lib().ugp_profile_end(ms, nl), "ugp_profile_end")
    return {name: (ms[i], nl[i]) for i, name in enumerate(PROFILE_STAGES)}


def launch_count() -> int:
    return int(lib().ugp_launch_count())


def version() -> str:
    return lib().ugp_version().decode()


# ------------------------------------------------------------------ learned guide
GUIDE_NPARAMS = 19240


def _register_guide(L):
    L.ugp_guide_workspace_size.restype = C.c_size_t
    L.ugp_guide_workspace_size.argtypes = []
    L.ugp_guide_reset_workspace.restype = C.c_int
    L.ugp_guide_reset_workspace.argtypes = [vp, vp]
    L.ugp_guide_check.restype = C.c_int
    L.ugp_guide_check.argtypes = [vp, vp]
    L.ugp_guide_forward.restype = C.c_int
    L.ugp_guide_forward.argtypes = [C.POINTER(UgpGuide), C.c_int64, vp, vp, vp, vp, vp, C.c_size_t, vp]
    L.ugp_guide_mixture_pdf.restype = C.c_int
    L.ugp_guide_mixture_pdf.argtypes = [C.c_int64, vp, vp, vp, vp]
    L.ugp_guide_mixture_sample.restype = C.c_int
    L.ugp_guide_mixture_sample.argtypes = [C.c_int64, vp, vp, vp, vp, vp]
    L.ugp_guide_grad.restype = C.c_int
    L.ugp_guide_grad.argtypes = [C.POINTER(UgpGuide), C.c_int64, vp, vp, vp, vp, vp, vp, vp, C.c_size_t, vp]
    L.ugp_guide_adam_step.restype = C.c_int
    L.ugp_guide_adam_step.argtypes = [C.POINTER(UgpGuide), vp, vp]
    L.ugp_guide_train_from_render.restype = C.c_int
    L.ugp_guide_train_from_render.argtypes = [C.POINTER(UgpGuide), vp, C.c_size_t, C.c_int32, C.c_int32, C.c_int32,
                                              C.c_int64, C.c_int32, C.c_int32, vp, C.c_size_t, C.POINTER(C.c_int64),
                                              C.POINTER(C.c_float), vp]
    L.ugp_render_guided_workspace_size.restype = C.c_size_t
    L.ugp_render_guided_workspace_size.argtypes = [C.c_int32, C.c_int32, C.c_int32]


_EXTRA.append(_register_guide)


def guided_workspace_size(width: int, height: int, max_depth: int) -> int:
    return int(lib().ugp_render_guided_workspace_size(int(width), int(height), int(max_depth)))


class Guide:
    """The learned vMF-mixture guide: FP32 master weights, Adam moments and a workspace, all on
    the device; the C struct points at them."""

    def __init__(self, params, pos_lo=(0.0, 0.0, 0.0), pos_hi=(1.0, 1.0, 1.0), kappa_min=0.1, kappa_max=1e4,
                 lr=1e-3, beta1=0.9, beta2=0.99, eps=1e-8, device="cuda", train_target=0):
        p = torch.as_tensor(params, dtype=torch.float32).to(device).contiguous().clone()
        if p.numel() != GUIDE_NPARAMS:
            raise ValueError(f"guide needs {GUIDE_NPARAMS} parameters")
        self.params = p
        self.adam_m = torch.zeros_like(p)
        self.adam_v = torch.zeros_like(p)
        self.workspace = torch.empty(int(lib().ugp_guide_workspace_size()), dtype=torch.uint8, device=device)
        _check(lib().ugp_guide_reset_workspace(_p(self.workspace), C.c_void_p(_stream())), "ugp_guide_reset_workspace")
        self.c = UgpGuide(_p(self.params), _p(self.adam_m), _p(self.adam_v), 0, float(lr), float(beta1), float(beta2),
                          float(eps), (C.c_float * 3)(*pos_lo), (C.c_float * 3)(*pos_hi), float(kappa_min),
                          float(kappa_max), int(train_target))

    @property
    def step(self) -> int:
        return int(self.c.step)

    def check(self, stream=None):
        _check(lib().ugp_guide_check(_p(self.workspace), C.c_void_p(_stream(stream))), "ugp_guide_check")

    def forward(self, x3, wo3, head=True, mix=True, stream=None):
        """(head outputs (n, 40), mixtures (n, 40)) for vertices x3, wo3 ((n, 3) float32)."""
        n = int(x3.shape[0])
        dev = self.params.device
        _dev(x3, torch.float32, "x3", 3, device=dev)
        _dev(wo3, torch.float32, "wo3", 3, n=n, device=dev)
        Y = torch.empty((n, 40), dtype=torch.float32, device=x3.device) if head else None
        M = torch.empty((n, 40), dtype=torch.float32, device=x3.device) if mix else None
        _check(lib().ugp_guide_forward(C.byref(self.c), n, _p(x3), _p(wo3), _p(Y), _p(M), _p(self.workspace),
                                       self.workspace.numel(), C.c_void_p(_stream(stream))), "ugp_guide_forward")
        return Y, M

    def grad(self, x3, wo3, wi3, weight, stream=None):
        """(gradient of the mean loss (GUIDE_NPARAMS,), mean loss (1,)) on the device."""
        n = int(x3.shape[0])
        dev = self.params.device
        for t, nm in ((x3, "x3"), (wo3, "wo3"), (wi3, "wi3")):
            _dev(t, torch.float32, nm, 3, n=n, device=dev)
        _dev(weight, torch.float32, "weight", n=n, device=dev)
        g = torch.empty(GUIDE_NPARAMS, dtype=torch.float32, device=self.params.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.params.device)
        _check(lib().ugp_guide_grad(C.byref(self.c), n, _p(x3), _p(wo3), _p(wi3), _p(weight), _p(g), _p(loss),
                                    _p(self.workspace), self.workspace.numel(), C.c_void_p(_stream(stream))),
               "ugp_guide_grad")
        return g, loss

    def adam_step(self, grad, stream=None):
        _dev(grad, torch.float32, "grad", n=GUIDE_NPARAMS, device=self.params.device)
        _check(lib().ugp_guide_adam_step(C.byref(self.c), _p(grad), C.c_void_p(_stream(stream))), "ugp_guide_adam_step")

    def train_from(self, renderer: "Renderer", max_samples: int = 1 << 20, minibatch: int = 1 << 16,
                   min_steps: int = 0, stream=None):
        """Adam over the vertices the renderer's last logged call recorded: one pass in minibatches,
        or min_steps minibatches (cycling) if that is more. Returns (samples used, mean loss of the
        last minibatch); synchronises."""
        ns = C.c_int64(0)
        ml = C.c_float(0)
        _check(lib().ugp_guide_train_from_render(C.byref(self.c), _p(renderer.workspace), renderer.workspace.numel(),
                                                 renderer.width, renderer.height, renderer.guided_depth,
                                                 int(max_samples), int(minibatch), int(min_steps), _p(self.workspace),
                                                 self.workspace.numel(), C.byref(ns), C.byref(ml),
                                                 C.c_void_p(_stream(stream))), "ugp_guide_train_from_render")
        return int(ns.value), float(ml.value)


def mixture_pdf(mix, wi3, stream=None):
    n = int(mix.shape[0])
    _dev(mix, torch.float32, "mix", 40)
    _dev(wi3, torch.float32, "wi3", 3, n=n, device=mix.device)
    out = torch.empty(n, dtype=torch.float32, device=mix.device)
    _check(lib().ugp_guide_mixture_pdf(n, _p(mix), _p(wi3), _p(out), C.c_void_p(_stream(stream))),
           "ugp_guide_mixture_pdf")
    return out


def mixture_sample(mix, u3, stream=None):
    n = int(mix.shape[0])
    _dev(mix, torch.float32, "mix", 40)
    _dev(u3, torch.float32, "u3", 3, n=n, device=mix.device)
    wi = torch.empty((n, 3), dtype=torch.float32, device=mix.device)
    pdf = torch.empty(n, dtype=torch.float32, device=mix.device)
    _check(lib().ugp_guide_mixture_sample(n, _p(mix), _p(u3), _p(wi), _p(pdf), C.c_void_p(_stream(stream))),
           "ugp_guide_mixture_sample")
    return wi, pdf


# ------------------------------------------------------------------ batched serving
class UgpRequest(C.Structure):
    _fields_ = [("bvh", vp), ("materials", C.POINTER(UgpMaterials)), ("camera", UgpCamera), ("lights", UgpLights),
                ("spp", C.c_int32), ("max_depth", C.c_int32), ("nee", C.c_int32), ("spawn_mode", C.c_int32),
                ("seed", C.c_uint64), ("accum_rgb", vp), ("accum_sq_rgb", vp)]


class UgpBatchConfig(C.Structure):
    _fields_ = [("tile", C.c_int32), ("pool_log2", C.c_int32), ("use_graph", C.c_int32), ("order", C.c_int32)]


def _register_batch(L):
    L.ugp_render_batch_workspace_size.restype = C.c_size_t
    L.ugp_render_batch_workspace_size.argtypes = [C.c_int32, C.POINTER(UgpBatchConfig)]
    L.ugp_render_batch.restype = C.c_int
    L.ugp_render_batch.argtypes = [C.c_int32, C.POINTER(UgpRequest), C.POINTER(UgpBatchConfig), C.c_int32, vp,
                                   C.c_size_t, C.POINTER(C.c_double), vp, vp]
    L.ugp_render_batch_autotune.restype = C.c_int
    L.ugp_render_batch_autotune.argtypes = [C.c_int32, C.POINTER(UgpRequest), C.c_int32, C.c_int32, C.c_int32,
                                            C.c_int32, vp, C.c_size_t, vp, C.c_size_t, C.POINTER(UgpBatchConfig),
                                            C.POINTER(C.c_double), vp]


_EXTRA.append(_register_batch)


class Request:
    """One render request of a batch; accumulators are created if not given."""

    def __init__(self, bvh: Bvh, mats: Materials, camera: UgpCamera, lights: UgpLights, spp: int, max_depth: int,
                 seed: int = 0, nee: bool = True, spawn_mode: int = 0, accum=None, accum_sq=None, device="cuda"):
        shape = (camera.height, camera.width, 3)
        self.accum = accum if accum is not None else torch.zeros(shape, dtype=torch.float32, device=device)
        self.accum_sq = accum_sq if accum_sq is not None else torch.zeros(shape, dtype=torch.float32, device=device)
        for t, nm in ((self.accum, "accum"), (self.accum_sq, "accum_sq")):
            _dev(t, torch.float32, nm, device=self.accum.device)
            if tuple(t.shape) != shape:
                raise ValueError(f"{nm} must have shape {shape}")
        _check_scene(bvh, mats, self.accum.device)
        self.bvh, self.mats = bvh, mats
        self.c = UgpRequest(C.c_void_p(bvh.handle).value, C.pointer(mats.c), camera, lights, int(spp), int(max_depth),
                            int(bool(nee)), int(spawn_mode), int(seed), _p(self.accum).value,
                            _p(self.accum_sq).value)


def batch_workspace_size(max_requests: int, tile: int, pool_log2: int) -> int:
    cfg = UgpBatchConfig(int(tile), int(pool_log2), 1, 1)
    return int(lib().ugp_render_batch_workspace_size(int(max_requests), C.byref(cfg)))


class BatchRenderer:
    """Serves batches of render requests in one wavefront over a shared path pool (one CUDA graph
    launch per batch). The workspace is sized for `max_requests` and the largest pool used."""

    def __init__(self, max_requests: int, pool_log2: int = 20, tile: int = 16, use_graph: bool = True,
                 shortest_first: bool = True, device="cuda"):
        self.max_requests = int(max_requests)
        self.cfg = UgpBatchConfig(int(tile), int(pool_log2), int(bool(use_graph)), int(bool(shortest_first)))
        self.device = device
        self.workspace = None
        self._ensure(int(pool_log2))

    def _ensure(self, pool_log2):
        nb = batch_workspace_size(self.max_requests, self.cfg.tile, pool_log2)
        if nb == 0:
            raise UgpError("bad batch configuration")
        if self.workspace is None or self.workspace.numel() < nb:
            self.workspace = torch.empty(nb, dtype=torch.uint8, device=self.device)

    def render(self, requests, ray_counts=None, stream=None):
        """Renders all requests; returns the per-request completion times in ms (numpy array)."""
        import numpy as np
        n = len(requests)
        if n > self.max_requests:
            raise ValueError("more requests than the workspace was sized for")
        arr = (UgpRequest * max(n, 1))(*[r.c for r in requests])
        lat = (C.c_double * max(n, 1))()
        if ray_counts is not None:
            _dev(ray_counts, torch.int64, "ray_counts", n=3, device=self.workspace.device)
        self._ensure(self.cfg.pool_log2)
        _check(lib().ugp_render_batch(n, arr, C.byref(self.cfg), self.max_requests, _p(self.workspace),
                                      self.workspace.numel(), lat, _p(ray_counts), C.c_void_p(_stream(stream))),
               "ugp_render_batch")
        return np.array(lat[:n])

    def autotune(self, requests, probe_spp: int = 1, pool_log2_range=(18, 22), stream=None):
        """Picks tile and pool size on a probe of `requests`; sets and returns the config and the
        table of probe times {(tile, pool_log2): ms}."""
        lo, hi = pool_log2_range
        n = len(requests)
        for lg in range(lo, hi + 1):
            nb = batch_workspace_size(max(n, self.max_requests), 8, lg)
            if self.workspace is None or self.workspace.numel() < nb:
                self.workspace = torch.empty(nb, dtype=torch.uint8, device=self.device)
        px = max(r.c.camera.width * r.c.camera.height for r in requests)
        scratch = torch.zeros(6 * px, dtype=torch.float32, device=self.device)
        arr = (UgpRequest * n)(*[r.c for r in requests])
        best = UgpBatchConfig()
        ms = (C.c_double * (3 * (hi - lo + 1)))()
        _check(lib().ugp_render_batch_autotune(n, arr, int(probe_spp), int(lo), int(hi), self.cfg.use_graph,
                                               _p(self.workspace), self.workspace.numel(), _p(scratch),
                                               scratch.numel(), C.byref(best), ms, C.c_void_p(_stream(stream))),
               "ugp_render_batch_autotune")
        table = {}
        k = 0
        for lg in range(lo, hi + 1):
            for t in (8, 16, 32):
                table[(t, lg)] = ms[k]
                k += 1
        self.cfg = UgpBatchConfig(best.tile, best.pool_log2, best.use_graph, self.cfg.order)
        return (best.tile, best.pool_log2), table
