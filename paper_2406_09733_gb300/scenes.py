"""Seeded synthetic inputs: scenes of Gaussian primitives, cameras, lights and query rays.

Both the CUDA path and the CPU oracle are fed from this module, and nothing else
is shared between them.  It only *draws* inputs; it holds none of the rendering
method's arithmetic (no integrals, no transmittance, no sampling of the light
transport).  Every array it returns is plain float32 / uint8 numpy data in the
layout of the C ABI (structure of arrays, one row per primitive).

Recipes (the paper's own scenes are purchased assets and datasets that are not
available; these generators stand in for them):

* ``tiny_scene``  -- 1,000 random anisotropic Gaussians in the unit cube, the
  analogue of the "1K random Gaussians" convergence study (Sec. 5.2, Fig. 7).
  Peak density rho ~ U[0.5, 5] is turned into the magnitude c of Eq. 1 by
  c = rho (2 pi)^{3/2} s_x s_y s_z, i.e. rho is the value of G at the mean.
* ``room_scene``  -- a procedural room of surface splats and volumetric
  aggregates shaped like the paper's large scenes (Sec. 9, Table 3): 70 %
  surface-like primitives (one scale 1/100 of the others) on planes, spheres
  and boxes, 30 % isotropic primitives in Gaussian clusters.  Tangential
  splat scales follow the mesh-conversion rule of Sec. 7.1,
  s_t = sqrt(eps * k * A / n) with eps = 0.01 and k = 16.  Surface
  magnitudes make a normal-incidence ray through the centre reach an optical
  depth of 1.5 (c = 3 * 2 pi s_x s_y); aggregate primitives get a
  through-centre depth drawn from U[0.05, 0.5] (c = 4 pi depth s^2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MAT_DIFFUSE = 0
MAT_GGX = 1
MAT_EMISSIVE = 2
MAT_DISNEY = 3


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


@dataclass
class Camera:
    eye: tuple
    look: tuple
    up: tuple
    vfov_deg: float
    width: int
    height: int


@dataclass
class Lights:
    """One optional one-sided rectangular area light plus a constant background."""
    has_quad: bool = False
    quad_corner: tuple = (0.0, 0.0, 0.0)
    quad_e1: tuple = (0.0, 0.0, 0.0)
    quad_e2: tuple = (0.0, 0.0, 0.0)
    quad_Le: tuple = (0.0, 0.0, 0.0)
    bg: tuple = (0.0, 0.0, 0.0)


@dataclass
class Scene:
    mean: np.ndarray          # (N,3) float32
    quat: np.ndarray          # (N,4) float32, (w,x,y,z), unit length
    scale: np.ndarray         # (N,3) float32, > 0
    magnitude: np.ndarray     # (N,)  float32, c of Eq. 1
    sggx: np.ndarray          # (N,6) float32, (Sxx,Syy,Szz,Sxy,Sxz,Syz)
    mtype: np.ndarray         # (N,)  uint8, MAT_*
    albedo: np.ndarray        # (N,3) float32
    roughness: np.ndarray     # (N,)  float32, GGX alpha
    emission: np.ndarray      # (N,3) float32
    camera: Camera = None
    lights: Lights = field(default_factory=Lights)
    # (N,9) float32 Disney parameters of MAT_DISNEY primitives (metallic, subsurface, specular,
    # specular tint, roughness, sheen, sheen tint, clearcoat, clearcoat gloss), or None
    disney: np.ndarray = None

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.mean[idx], self.quat[idx], self.scale[idx], self.magnitude[idx],
                     self.sggx[idx], self.mtype[idx], self.albedo[idx], self.roughness[idx],
                     self.emission[idx], self.camera, self.lights,
                     None if self.disney is None else self.disney[idx])


def random_disney_params(rng: np.random.Generator, n: int) -> np.ndarray:
    """n parameter sets of the Disney base: metallic, subsurface, specular, specular tint,
    sheen, sheen tint and clearcoat gloss uniform in [0, 1], roughness uniform in [0.3, 0.9],
    clearcoat uniform in [0, 1] on half of the sets and 0 on the rest."""
    d = rng.random((n, 9))
    d[:, 4] = rng.uniform(0.3, 0.9, n)
    d[:, 7] *= rng.random(n) < 0.5
    return d


def with_disney(scene: Scene, frac: float, seed: int = 0) -> Scene:
    """The scene with a random fraction `frac` of its non-emissive primitives turned into Disney
    primitives (base colour = their albedo) with random parameters."""
    rng = _rng(seed)
    mtype = scene.mtype.copy()
    cand = np.flatnonzero(mtype != MAT_EMISSIVE)
    pick = cand[rng.random(cand.size) < frac]
    mtype[pick] = MAT_DISNEY
    dis = np.zeros((scene.n, 9))
    dis[pick] = random_disney_params(rng, pick.size)
    return Scene(scene.mean, scene.quat, scene.scale, scene.magnitude, scene.sggx, mtype, scene.albedo,
                 scene.roughness, scene.emission, scene.camera, scene.lights, _f32(dis))


def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed unit quaternions (Shoemake, Graphics Gems III), (w,x,y,z)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = b * np.sin(2 * np.pi * u3)
    w = b * np.cos(2 * np.pi * u3)
    return np.stack([w, x, y, z], axis=1)


def frame_to_quaternion(t1: np.ndarray, t2: np.ndarray, nrm: np.ndarray) -> np.ndarray:
    """Quaternions (w,x,y,z) of rotation matrices whose columns are (t1, t2, nrm)."""
    m = np.stack([t1, t2, nrm], axis=2)          # (n,3,3), columns are the frame axes
    n = m.shape[0]
    q = np.zeros((n, 4))
    tr = m[:, 0, 0] + m[:, 1, 1] + m[:, 2, 2]
    # Branch on the largest diagonal term for a well conditioned extraction.
    cases = np.argmax(np.stack([tr, m[:, 0, 0], m[:, 1, 1], m[:, 2, 2]], axis=1), axis=1)
    for c in range(4):
        s = cases == c
        if not np.any(s):
            continue
        mm = m[s]
        if c == 0:
            r = np.sqrt(1.0 + tr[s]) * 2
            q[s] = np.stack([0.25 * r, (mm[:, 2, 1] - mm[:, 1, 2]) / r,
                             (mm[:, 0, 2] - mm[:, 2, 0]) / r, (mm[:, 1, 0] - mm[:, 0, 1]) / r], 1)
        elif c == 1:
            r = np.sqrt(1.0 + mm[:, 0, 0] - mm[:, 1, 1] - mm[:, 2, 2]) * 2
            q[s] = np.stack([(mm[:, 2, 1] - mm[:, 1, 2]) / r, 0.25 * r,
                             (mm[:, 0, 1] + mm[:, 1, 0]) / r, (mm[:, 0, 2] + mm[:, 2, 0]) / r], 1)
        elif c == 2:
            r = np.sqrt(1.0 + mm[:, 1, 1] - mm[:, 0, 0] - mm[:, 2, 2]) * 2
            q[s] = np.stack([(mm[:, 0, 2] - mm[:, 2, 0]) / r, (mm[:, 0, 1] + mm[:, 1, 0]) / r,
                             0.25 * r, (mm[:, 1, 2] + mm[:, 2, 1]) / r], 1)
        else:
            r = np.sqrt(1.0 + mm[:, 2, 2] - mm[:, 0, 0] - mm[:, 1, 1]) * 2
            q[s] = np.stack([(mm[:, 1, 0] - mm[:, 0, 1]) / r, (mm[:, 0, 2] + mm[:, 2, 0]) / r,
                             (mm[:, 1, 2] + mm[:, 2, 1]) / r, 0.25 * r], 1)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sggx_from_frame(t1, t2, nrm, r):
    """SGGX matrix S = n n^T + r^2 (t1 t1^T + t2 t2^T): a surface-like flake distribution."""
    S = (nrm[:, :, None] * nrm[:, None, :]
         + (r ** 2) * (t1[:, :, None] * t1[:, None, :] + t2[:, :, None] * t2[:, None, :]))
    return np.stack([S[:, 0, 0], S[:, 1, 1], S[:, 2, 2], S[:, 0, 1], S[:, 0, 2], S[:, 1, 2]], 1)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def tiny_scene(n: int = 1000, seed: int = 0, width: int = 128, height: int = 128,
               emissive_radiance: float = 10.0) -> Scene:
    """1,000 random Gaussians in [0,1]^3 (peak density, Lambertian, S = I, primitive 0 emissive)."""
    rng = _rng(seed)
    mean = rng.random((n, 3))
    scale = np.exp(rng.uniform(np.log(0.01), np.log(0.05), size=(n, 3)))
    quat = random_quaternions(rng, n)
    rho = rng.uniform(0.5, 5.0, size=n)
    magnitude = rho * (2 * np.pi) ** 1.5 * scale.prod(axis=1)
    albedo = rng.uniform(0.2, 0.8, size=(n, 3))
    sggx = np.tile(np.array([1, 1, 1, 0, 0, 0], dtype=np.float64), (n, 1))
    mtype = np.full(n, MAT_DIFFUSE, dtype=np.uint8)
    emission = np.zeros((n, 3))
    mtype[0] = MAT_EMISSIVE
    emission[0] = emissive_radiance
    rough = np.full(n, 0.3)
    cam = Camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 40.0, width, height)
    return Scene(_f32(mean), _f32(quat), _f32(scale), _f32(magnitude), _f32(sggx), mtype,
                 _f32(albedo), _f32(rough), _f32(emission), cam, Lights())


def _sample_plane(rng, m, origin, e1, e2):
    u, v = rng.random(m), rng.random(m)
    p = origin[None] + u[:, None] * e1[None] + v[:, None] * e2[None]
    nrm = np.cross(e1, e2)
    nrm = nrm / np.linalg.norm(nrm)
    return p, np.tile(nrm, (m, 1))


def _sample_sphere(rng, m, c, r):
    z = rng.uniform(-1, 1, m)
    phi = rng.uniform(0, 2 * np.pi, m)
    s = np.sqrt(1 - z * z)
    nrm = np.stack([s * np.cos(phi), s * np.sin(phi), z], 1)
    return c[None] + r * nrm, nrm


def _tangent_frame(rng, nrm):
    a = rng.normal(size=nrm.shape)
    t1 = a - (a * nrm).sum(1, keepdims=True) * nrm
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(nrm, t1)
    return t1, t2


def room_scene(n: int = 1_000_000, seed: int = 0, width: int = 1024, height: int = 1024,
               near_specular_frac: float = 0.0, lighting: str = "A",
               n_small_emitters: int = 12000, n_clusters: int = 300) -> Scene:
    """Procedural room of surface splats and aggregate clusters (mixed materials).

    lighting "A": one 0.3 x 0.3 quad light below the ceiling (L_e = 20) plus
    background radiance 0.2.  lighting "B": ``n_small_emitters`` small emissive
    aggregate primitives, no quad, black background.  ``n_clusters`` sets how many
    aggregate clusters share the 30 % aggregate primitives (smaller scenes keep the
    per-cluster density of the 1M scene with n_clusters = 300 * n / 1e6).
    """
    rng = _rng(seed)
    n_surf = int(round(0.7 * n))
    n_aggr = n - n_surf

    # --- shapes: 5 room planes (open towards -z), 12 spheres, 8 axis-aligned boxes -------------
    shapes = []   # (kind, params, area, material index)
    o = np.zeros(3)
    X, Y, Z = np.eye(3)
    shapes.append(("plane", (o, Z, X), 1.0))                    # floor y = 0, normal +y
    shapes.append(("plane", (Y.copy(), X, Z), 1.0))             # ceiling y = 1, normal -y
    shapes.append(("plane", (Z.copy(), X, Y), 1.0))             # back wall z = 1, normal -z
    shapes.append(("plane", (o, Y, Z), 1.0))                    # left wall x = 0, normal +x
    shapes.append(("plane", (X.copy(), Z, Y), 1.0))             # right wall x = 1, normal -x
    for _ in range(12):
        r = rng.uniform(0.05, 0.15)
        c = rng.uniform(0.2, 0.8, 3)
        shapes.append(("sphere", (c, r), 4 * np.pi * r * r))
    for _ in range(8):
        e = rng.uniform(0.05, 0.2)
        lo = rng.uniform(0.05, 0.95 - e, 3)
        lo[1] = 0.0                                              # boxes stand on the floor
        shapes.append(("box", (lo, e), 6 * e * e))
    areas = np.array([s[2] for s in shapes])
    counts = np.floor(n_surf * areas / areas.sum()).astype(np.int64)
    counts[0] += n_surf - counts.sum()

    # Per-shape materials: room planes diffuse or glossy, other shapes from the 50/40/10 mix.
    n_shapes = len(shapes)
    u = rng.random(n_shapes)
    shape_type = np.where(u < 0.5, MAT_DIFFUSE, np.where(u < 0.9, MAT_GGX, MAT_EMISSIVE))
    shape_type[:5] = np.where(rng.random(5) < 0.7, MAT_DIFFUSE, MAT_GGX)
    shape_albedo = rng.uniform(0.2, 0.8, (n_shapes, 3))
    shape_rough = rng.uniform(0.05, 0.5, n_shapes)
    near_spec = rng.random(n_shapes) < near_specular_frac
    shape_rough[near_spec] = 0.02
    shape_type[near_spec] = MAT_GGX
    colour = rng.uniform(0.3, 1.0, (n_shapes, 3))
    shape_emit = rng.uniform(0.5, 5.0, (n_shapes, 1)) * colour

    P, N_, T1, T2, S_t, SID = [], [], [], [], [], []
    for sid, (kind, prm, area) in enumerate(shapes):
        m = int(counts[sid])
        if m == 0:
            continue
        if kind == "plane":
            p, nrm = _sample_plane(rng, m, *prm)
        elif kind == "sphere":
            p, nrm = _sample_sphere(rng, m, *prm)
        else:
            lo, e = prm
            face = rng.integers(0, 6, m)
            axis, side = face // 2, face % 2
            uv = rng.random((m, 2)) * e
            p = np.tile(lo, (m, 1)).astype(np.float64)
            nrm = np.zeros((m, 3))
            for ax in range(3):
                s_ax = axis == ax
                others = [a for a in range(3) if a != ax]
                p[s_ax, ax] += side[s_ax] * e
                p[s_ax, others[0]] += uv[s_ax, 0]
                p[s_ax, others[1]] += uv[s_ax, 1]
                nrm[s_ax, ax] = np.where(side[s_ax] == 1, 1.0, -1.0)
        t1, t2 = _tangent_frame(rng, nrm)
        s_t = np.sqrt(0.01 * 16.0 * area / m)
        P.append(p); N_.append(nrm); T1.append(t1); T2.append(t2)
        S_t.append(np.full(m, s_t)); SID.append(np.full(m, sid))
    p = np.concatenate(P); nrm = np.concatenate(N_); t1 = np.concatenate(T1); t2 = np.concatenate(T2)
    s_t = np.concatenate(S_t); sid = np.concatenate(SID)
    surf_scale = np.stack([s_t, s_t, 0.01 * s_t], 1)
    surf_quat = frame_to_quaternion(t1, t2, nrm)
    surf_mag = 3.0 * 2 * np.pi * s_t * s_t
    surf_sggx = _sggx_from_frame(t1, t2, nrm, 0.01)

    # --- aggregates: 300 Gaussian clusters of isotropic primitives ------------------------------
    n_cl = max(1, int(n_clusters))
    centres = rng.uniform(0.1, 0.9, (n_cl, 3))
    cl = rng.integers(0, n_cl, n_aggr)
    ap = centres[cl] + rng.normal(scale=0.03, size=(n_aggr, 3))
    s_a = np.exp(rng.uniform(np.log(0.003), np.log(0.01), n_aggr))
    depth = rng.uniform(0.05, 0.5, n_aggr)
    a_mag = 4 * np.pi * depth * s_a * s_a
    u = rng.random(n_cl)
    cl_type = np.where(u < 0.5, MAT_DIFFUSE, np.where(u < 0.9, MAT_GGX, MAT_EMISSIVE))
    cl_albedo = rng.uniform(0.2, 0.8, (n_cl, 3))
    cl_rough = rng.uniform(0.05, 0.5, n_cl)
    cl_emit = rng.uniform(0.5, 5.0, (n_cl, 1)) * rng.uniform(0.3, 1.0, (n_cl, 3))

    mean = np.concatenate([p, ap])
    scale = np.concatenate([surf_scale, np.stack([s_a] * 3, 1)])
    quat = np.concatenate([surf_quat, random_quaternions(rng, n_aggr)])
    mag = np.concatenate([surf_mag, a_mag])
    sggx = np.concatenate([surf_sggx, np.tile([1.0, 1, 1, 0, 0, 0], (n_aggr, 1))])
    mtype = np.concatenate([shape_type[sid], cl_type[cl]]).astype(np.uint8)
    albedo = np.concatenate([shape_albedo[sid], cl_albedo[cl]])
    rough = np.concatenate([shape_rough[sid], cl_rough[cl]])
    emission = np.concatenate([shape_emit[sid], cl_emit[cl]])
    emission[mtype != MAT_EMISSIVE] = 0.0

    lights = Lights()
    if lighting == "A":
        lights = Lights(True, (0.35, 0.98, 0.35), (0.3, 0.0, 0.0), (0.0, 0.0, 0.3),
                        (20.0, 20.0, 20.0), (0.2, 0.2, 0.2))   # e1 x e2 points down (-y)
    elif lighting == "B":
        k = min(n_small_emitters, n_aggr)
        pick = n_surf + rng.choice(n_aggr, size=k, replace=False)
        mtype[pick] = MAT_EMISSIVE
        emission[pick] = rng.uniform(2.0, 20.0, (k, 1)) * rng.uniform(0.5, 1.0, (k, 3))
    else:
        raise ValueError(f"unknown lighting {lighting!r}")

    cam = Camera((0.5, 0.5, -0.8), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, width, height)
    return Scene(_f32(mean), _f32(quat), _f32(scale), _f32(mag), _f32(sggx), mtype,
                 _f32(albedo), _f32(rough), _f32(emission), cam, lights)


@dataclass
class Rays:
    o: np.ndarray    # (n,3) float32
    d: np.ndarray    # (n,3) float32, unit
    t0: np.ndarray   # (n,) float32
    t1: np.ndarray   # (n,) float32

    @property
    def n(self) -> int:
        return int(self.o.shape[0])


def random_rays(n: int, seed: int = 1, inside_frac: float = 0.25, finite_frac: float = 0.25,
                centre=(0.5, 0.5, 0.5), radius: float = 1.5) -> Rays:
    """Query rays through the unit cube.

    Most rays start on a sphere around the cube and aim at a uniform point
    inside it; ``inside_frac`` of them start inside the cube (so intervals are
    clipped at t0), and ``finite_frac`` end inside it (clipped at t1).
    """
    rng = _rng(seed)
    c = np.asarray(centre, dtype=np.float64)
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    o = c + radius * dirs
    target = rng.random((n, 3))
    inside = rng.random(n) < inside_frac
    o[inside] = rng.random((int(inside.sum()), 3))
    d = target - o
    bad = np.linalg.norm(d, axis=1) < 1e-3
    d[bad] = rng.normal(size=(int(bad.sum()), 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d = _f32(d)
    # renormalise in float32 so the direction stored is unit to float32 rounding
    d = _f32(d / np.linalg.norm(d.astype(np.float64), axis=1, keepdims=True))
    t0 = np.zeros(n)
    t1 = np.full(n, 4.0)
    fin = rng.random(n) < finite_frac
    t1[fin] = rng.uniform(0.2, 2.0, int(fin.sum()))
    return Rays(_f32(o), d, _f32(t0), _f32(t1))


def uniforms24(rng_or_seed, shape) -> np.ndarray:
    """Uniforms on the 2^-24 grid in [0,1): exactly representable in float32 and float64."""
    rng = _rng(rng_or_seed) if isinstance(rng_or_seed, (int, np.integer)) else rng_or_seed
    k = rng.integers(0, 1 << 24, size=shape, dtype=np.int64)
    return _f32(k.astype(np.float64) * (2.0 ** -24))


# ------------------------------------------------------------------ learned guide inputs
GUIDE_LOBES = 8
GUIDE_WIDTH = 64
GUIDE_OUT = 5 * GUIDE_LOBES
GUIDE_LAYERS = 4
# Flat parameter vector: for l = 0..3, W_l (64 x 64, [out][in]) then b_l (64); then the head
# W_4 (40 x 64) and b_4 (40).
GUIDE_SHAPES = [(GUIDE_WIDTH, GUIDE_WIDTH)] * GUIDE_LAYERS + [(GUIDE_OUT, GUIDE_WIDTH)]
GUIDE_NPARAMS = sum(o * i + o for o, i in GUIDE_SHAPES)


@dataclass
class GuideConfig:
    """Position box of the guide's input normalisation and the range of the lobe sharpness."""
    pos_lo: tuple = (0.0, 0.0, 0.0)
    pos_hi: tuple = (1.0, 1.0, 1.0)
    kappa_min: float = 0.1
    kappa_max: float = 1.0e4


def guide_param_slices():
    """[(W slice, b slice)] of the flat parameter vector, per layer."""
    out, off = [], 0
    for o, i in GUIDE_SHAPES:
        w = slice(off, off + o * i)
        off += o * i
        b = slice(off, off + o)
        off += o
        out.append((w, b))
    return out


def guide_init_params(seed: int = 0, bias_scale: float = 0.0) -> np.ndarray:
    """Seeded initial weights: He-uniform W (bound sqrt(6 / fan_in)), biases U[-s, s]."""
    rng = _rng(seed)
    p = np.zeros(GUIDE_NPARAMS, np.float32)
    for (o, i), (ws, bs) in zip(GUIDE_SHAPES, guide_param_slices()):
        lim = np.sqrt(6.0 / i)
        p[ws] = rng.uniform(-lim, lim, o * i).astype(np.float32)
        if bias_scale > 0:
            p[bs] = rng.uniform(-bias_scale, bias_scale, o).astype(np.float32)
    return p


def unit_vectors(rng_or_seed, n: int) -> np.ndarray:
    rng = rng_or_seed if isinstance(rng_or_seed, np.random.Generator) else _rng(rng_or_seed)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v.astype(np.float32)


@dataclass
class GuideBatch:
    """Logged scattering vertices: position, outgoing and incident directions, loss weight."""
    x: np.ndarray
    wo: np.ndarray
    wi: np.ndarray
    weight: np.ndarray

    @property
    def n(self):
        return self.x.shape[0]


def guide_batch(n: int, seed: int = 0, cfg: GuideConfig | None = None, zero_frac: float = 0.1) -> GuideBatch:
    """Random vertices in (and slightly outside) the box, weights log-uniform over 4 decades with a
    fraction of zero weights (vertices whose paths found no light)."""
    cfg = cfg or GuideConfig()
    rng = _rng(seed)
    lo, hi = np.asarray(cfg.pos_lo), np.asarray(cfg.pos_hi)
    x = lo + (hi - lo) * rng.uniform(-0.05, 1.05, size=(n, 3))
    w = 10.0 ** rng.uniform(-2, 2, n)
    w[rng.uniform(size=n) < zero_frac] = 0.0
    return GuideBatch(_f32(x), unit_vectors(rng, n), unit_vectors(rng, n), _f32(w))


# ------------------------------------------------------------------ batched serving inputs
@dataclass
class RequestSpec:
    """One render request of a serving batch: which scene, image size, samples, depth, seed."""
    scene: int
    width: int
    height: int
    spp: int
    max_depth: int
    seed: int
    nee: bool = True


def serving_batch(n_requests: int = 64, n_scenes: int = 8, seed: int = 0, n_range=(1e4, 1e6),
                  sizes=(256, 512, 1024), spp_range=(1, 64), depth_range=(4, 8)):
    """Requests of a serving batch: scenes from the room generator with primitive counts
    log-uniform over n_range (cluster count scaled with n), requests with a size drawn from
    `sizes` (square images), spp log-uniform over spp_range (integers) and depth uniform over
    depth_range; every request names one of the scenes. Returns (scene sizes, requests)."""
    rng = _rng(seed)
    lo, hi = np.log(n_range[0]), np.log(n_range[1])
    ns = [int(round(np.exp(rng.uniform(lo, hi)))) for _ in range(n_scenes)]
    reqs = []
    for i in range(n_requests):
        size = int(rng.choice(sizes))
        spp = int(np.floor(np.exp(rng.uniform(np.log(spp_range[0]), np.log(spp_range[1] + 1)))))
        spp = min(max(spp, spp_range[0]), spp_range[1])
        depth = int(rng.integers(depth_range[0], depth_range[1] + 1))
        reqs.append(RequestSpec(int(rng.integers(0, n_scenes)), size, size, spp, depth, 1000 + i))
    return ns, reqs


def serving_scene(n: int, seed: int, width: int = 256, height: int = 256) -> Scene:
    """A room scene of n primitives for serving (aggregate clusters scaled with n)."""
    return room_scene(n, seed=seed, width=width, height=height, n_clusters=max(1, int(round(300 * n / 1e6))))
