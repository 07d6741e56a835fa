"""The GPU's phase functions and renders on the materials of the benchmark scenes, against the
FP64 oracle.

* Element by element: the phase function (Eq. 12 with the SGGX visible normals of Eq. 11), its
  sampler and the approximate pdf of App. B, through ugp_phase_query, on the same directions
  and uniforms as the oracle: Lambertian, GGX (roughness 0.02, 0.05, 0.3) and Disney bases over
  isotropic flakes, random anisotropic S, and the surface-like flakes of the room scene
  (S = n n^T + 1e-4 (I - n n^T)).
* Renders at 3 standard errors per pixel and channel (at most 1 % failing): room-style surface
  splats with near-specular GGX under the area light with light sampling and MIS; a scene with
  Disney primitives.
"""
import numpy as np
import pytest

from paper_2406_09733_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_09733_gb300 import build, ugp
    build.build()
    ugp.lib()
    return torch


def _unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _s6(S):
    return np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]])


def _flake_S(nrm, r=0.01):
    """Surface-like flakes of the room scene: eigenvalues (r^2, r^2, 1) along the normal."""
    P = np.outer(nrm, nrm)
    return _s6(P + r * r * (np.eye(3) - P))


def _random_S(rng):
    R = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    return _s6(R @ np.diag(rng.uniform(0.1, 1.0, 3)) @ R.T)


def _materials(rng):
    """(name, type, albedo, alpha, S6, dis9) for every combination the tests cover."""
    out = []
    flake_n = _unit(rng, 1)[0]
    for sname, S in (("iso", _s6(np.eye(3))), ("aniso", _random_S(rng)), ("flakes", _flake_S(flake_n))):
        out.append((f"lambert-{sname}", 0, rng.uniform(0.2, 0.8, 3), 0.3, S, np.zeros(9)))
        for a in (0.02, 0.05, 0.3):
            out.append((f"ggx{a}-{sname}", 1, rng.uniform(0.2, 0.8, 3), a, S, np.zeros(9)))
        for j in range(2):
            dis = scenes.random_disney_params(np.random.Generator(np.random.Philox(40 + j)), 1)[0]
            out.append((f"disney{j}-{sname}", 3, rng.uniform(0.2, 0.8, 3), 0.3, S, dis))
    return out


def _query(torch, ugp, mt, alb, a, S, dis, wo, wi, ue, us):
    n = wi.shape[0]
    c = lambda x, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(x)).to(dtype=dt, device="cuda")
    rep = lambda v: np.tile(np.asarray(v, np.float64), (n, 1))
    out = ugp.phase_query(c(np.full(n, mt), torch.uint8), c(rep(alb)), c(np.full(n, a)), c(rep(S)), c(wo), c(wi),
                          c(ue), c(us), disney9=c(rep(dis)))
    return [x.double().cpu().numpy() for x in out]


def test_phase_query_matches_oracle(gpu, orc):
    from paper_2406_09733_gb300 import ugp
    torch = gpu
    rng = np.random.default_rng(77)
    n = 4000
    for name, mt, alb, a, S, dis in _materials(rng):
        wo1 = _unit(rng, 1)[0]
        if name.endswith("flakes"):
            wo1 = wo1 if wo1 @ _flake_axis(S) > 0 else -wo1
        wo = np.tile(wo1, (n, 1))
        wi = _unit(rng, n)
        ue = scenes.uniforms24(rng, (n, 6)).astype(np.float64)
        us = scenes.uniforms24(rng, (n, 4)).astype(np.float64)
        ev, pdf, swi, sw, ok = _query(torch, ugp, mt, alb, a, S, dis, wo, wi, ue, us)
        if mt == 3:
            ev_o = orc.phase_eval_disney(alb, dis, S, wo1, wi, ue)
            pdf_o = orc.phase_pdf_approx_disney(alb, dis, S, wo1, wi)
            swi_o, sw_o, ok_o = orc.phase_sample_disney(alb, dis, S, wo1, us)
        else:
            ev_o = orc.phase_eval(mt, alb, a, S, wo1, wi, ue)
            pdf_o = orc.phase_pdf_approx(mt, alb, a, S, wo1, wi)
            swi_o, sw_o, ok_o = orc.phase_sample(mt, alb, a, S, wo1, us)
        rel = lambda g, o: np.abs(g - o) / np.maximum(np.abs(o), 1e-3 * np.abs(o).max() + 1e-30)
        e_ev = rel(ev, ev_o).max(1)
        e_pdf = rel(pdf, pdf_o)
        same_ok = ok.astype(bool) == ok_o
        both = ok.astype(bool) & ok_o
        ang = np.abs(swi[both] - swi_o[both]).max(1)   # |difference| of the unit vectors
        e_w = rel(sw[both], sw_o[both]).max(1)
        q = lambda e: (np.quantile(e, 0.5), np.quantile(e, 0.99), e.max()) if e.size else (0, 0, 0)
        print(f"{name:18s} eval {q(e_ev)} pdf {q(e_pdf)} ok {same_ok.mean():.4f} angle {q(ang)} weight {q(e_w)}")
        # float32 against FP64 on the same uniforms: 99 % of the records within 5e-4 (relative;
        # measured at most 2e-4, on near-specular and Disney bases over surface-like flakes, where
        # the SGGX density's float32 adjugate loses digits), every record within 1e-2; sampled
        # directions within 1e-4
        for e in (e_ev, e_pdf, e_w):
            assert np.quantile(e, 0.99) <= 5e-4 and e.max() <= 1e-2, name
        assert same_ok.mean() >= 0.999, name
        assert np.quantile(ang, 0.99) <= 1e-4 and ang.max() <= 1e-3, name


def _flake_axis(S6):
    S = np.array([[S6[0], S6[3], S6[4]], [S6[3], S6[1], S6[5]], [S6[4], S6[5], S6[2]]])
    return np.linalg.eigh(S)[1][:, -1]


def _gpu_render(torch, s, spp, max_depth, seed, chunks=4):
    from paper_2406_09733_gb300 import ugp
    bvh, mats, cam, li = ugp.scene_to_device(s)
    r = ugp.Renderer(cam.width, cam.height)
    acc = acc2 = None
    cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
    per = spp // chunks
    for c in range(chunks):
        acc, acc2 = r.render(bvh, mats, cam, li, per, max_depth, seed=seed, spp_begin=c * per, accum=acc,
                             accum_sq=acc2, ray_counts=cnt)
    torch.cuda.synchronize()
    return acc.double().cpu().numpy(), acc2.double().cpu().numpy(), cnt.cpu().numpy()


def _compare(a_g, q_g, n_g, a_o, q_o, n_o, z_max=3.0, frac=0.01):
    """Per pixel and channel |mean_gpu - mean_ref| <= z_max sqrt(se_gpu^2 + se_ref^2) + acc, with
    acc = n_g 2^-24 |mean_ref|, the worst-case rounding of the GPU's float32 running sums of n_g
    samples (a pixel that sees only the background has no variance on either side, so the float32
    sum's own rounding decides it)."""
    mg, mo = a_g / n_g, a_o / n_o
    sg = np.sqrt(np.maximum(q_g / n_g - mg ** 2, 0) / n_g)
    so = np.sqrt(np.maximum(q_o / n_o - mo ** 2, 0) / n_o)
    acc = n_g * 2.0 ** -24 * np.abs(mo)
    z = np.maximum(np.abs(mg - mo) - acc, 0) / np.maximum(np.sqrt(sg ** 2 + so ** 2), 1e-9)
    bad = (z > z_max) & (np.abs(mg - mo) > 1e-6)
    print(f"pixel-channels beyond {z_max} SE: {bad.mean():.4f} (largest z {np.sort(z.ravel())[-4:]})")
    assert bad.mean() <= frac, (bad.mean(), np.sort(z.ravel())[-6:])


def surface_splat_scene(w=20, h=20):
    """A room of 3,000 primitives (70 % surface splats with the generator's surface-like flakes,
    30 % aggregates), under lighting A (area light + background). The surface splats' bases are
    set by index: a third Lambertian, a third GGX of roughness 0.02, a third GGX of 0.05."""
    s = scenes.room_scene(3000, seed=4, width=w, height=h, n_clusters=3)
    surf = np.flatnonzero((s.mtype != scenes.MAT_EMISSIVE)[:2100])
    k = surf % 3
    s.mtype[surf] = np.where(k == 0, scenes.MAT_DIFFUSE, scenes.MAT_GGX).astype(np.uint8)
    s.roughness[surf] = np.where(k == 1, 0.02, 0.05).astype(np.float32)
    assert s.lights.has_quad
    return s


def test_render_matches_oracle_surface_splats_near_specular(gpu, orc):
    s = surface_splat_scene()
    S = s.sggx[:2100].astype(np.float64)
    det = (S[:, 0] * (S[:, 1] * S[:, 2] - S[:, 5] ** 2) - S[:, 3] * (S[:, 3] * S[:, 2] - S[:, 5] * S[:, 4])
           + S[:, 4] * (S[:, 3] * S[:, 5] - S[:, 1] * S[:, 4]))
    assert np.all(np.abs(det - 1e-8) < 1e-10)   # surface-like flakes: eigenvalues (1e-4, 1e-4, 1)
    spp_g, spp_o = 8192, 2048
    a_g, q_g, cnt = _gpu_render(gpu, s, spp_g, max_depth=4, seed=21)
    a_o, q_o, _ = orc.render(s, spp=spp_o, max_depth=4, seed=22)
    assert cnt[1] > 0 and cnt[2] == 0
    _compare(a_g, q_g, spp_g, a_o, q_o, spp_o)


def test_render_matches_oracle_disney(gpu, orc):
    """Half of the non-emissive primitives of a lit scene (isotropic and anisotropic flakes) and of
    a surface-splat room are Disney primitives with random parameters."""
    from test_gpu_render import lit_scene
    for s, spp_g, spp_o in ((scenes.with_disney(lit_scene(), 0.5, seed=3), 4096, 1024),
                            (scenes.with_disney(surface_splat_scene(16, 16), 0.5, seed=4), 8192, 2048)):
        assert (s.mtype == scenes.MAT_DISNEY).sum() > 100
        a_g, q_g, cnt = _gpu_render(gpu, s, spp_g, max_depth=4, seed=23)
        a_o, q_o, _ = orc.render(s, spp=spp_o, max_depth=4, seed=24)
        assert cnt[2] == 0
        _compare(a_g, q_g, spp_g, a_o, q_o, spp_o)
