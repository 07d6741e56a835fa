"""GPU parity at the benchmark's full size.

The benchmark's scene (the 1M-primitive room, seed 0) and all 1024 x 1024 pixel-centre camera
rays go through one free-flight query (t in [0, 4]; the room lies within t < 3) and one
transmittance query (over [0, t1], t1 uniform in [0.2, 1.6], so that segments end before, inside
and behind surfaces and clusters), each a single launch over every ray like the renderer's
extend and shadow passes. A random sample of the rays is checked
against the FP64 oracle (brute force over every primitive) with the parity contract's
tolerances:
  * T: |T - T_ref| <= 1e-5 max(T_ref, 1 - T_ref), plus how much T_ref moves when the segment's
    end moves by 4 float32 ulps (an end inside a thin surface splat);
  * t_u, t_spawn: |t - t_ref| <= 1e-5 (t1 - t0) where the primitive agrees;
  * primitive: identical, except where the oracle itself flips to the GPU's answer when u moves
    by 1e-5, or its exponential race had a near-tie (relative gap < 1e-4).
It builds the largest scene of the suite, so it runs last.
"""
import numpy as np
from conftest import parity_note
import pytest

from paper_2406_09733_gb300 import scenes

pytestmark = pytest.mark.gpu

REL = 1e-5


def _camera_dirs(cam, W, H):
    f = np.array(cam.look, float) - np.array(cam.eye, float)
    f /= np.linalg.norm(f)
    r = np.cross(f, cam.up)
    r /= np.linalg.norm(r)
    up = np.cross(r, f)
    th = np.tan(np.radians(cam.vfov_deg) / 2)
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    d = f + ((W / H) * (2 * px / W - 1) * th)[..., None] * r + ((1 - 2 * py / H) * th)[..., None] * up
    return (d / np.linalg.norm(d, axis=-1, keepdims=True)).reshape(-1, 3).astype(np.float32)


def test_full_size_queries_sampled_parity(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_09733_gb300 import build, ugp
    build.build()
    W = H = 1024
    s = scenes.room_scene(1_000_000, width=W, height=H)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bvh = ugp.build_bvh(t(s.mean), t(s.quat), t(s.scale), t(s.magnitude))
    d = _camera_dirs(s.camera, W, H)
    n = d.shape[0]
    o = np.tile(np.array(s.camera.eye, np.float32), (n, 1))
    t0, t1 = np.zeros(n, np.float32), np.full(n, 4.0, np.float32)   # the room lies within t < 3
    u, u2 = scenes.uniforms24(201, n), scenes.uniforms24(202, n)
    prim, tu, tsp, st = ugp.sample_free_flight(bvh, t(o), t(d), t(t0), t(t1), t(u), t(u2))
    # transmittance over segments of random length, so that some end inside a surface or cluster
    tT = np.random.default_rng(204).uniform(0.2, 1.6, n).astype(np.float32)
    T, st2 = ugp.trace_transmittance(bvh, t(o), t(d), t(t0), t(tT))
    torch.cuda.synchronize()
    assert int(st.max()) == 0 and int(st2.max()) == 0
    prim, tu, tsp, T = (x.cpu().numpy() for x in (prim, tu, tsp, T))
    assert (prim >= 0).mean() > 0.5   # most camera rays scatter in the room

    idx = np.sort(np.random.default_rng(203).choice(n, 256, replace=False))
    r = scenes.Rays(o[idx], d[idx], t0[idx], t1[idx])
    T_at = lambda e: orc.transmittance(s, scenes.Rays(o[idx], d[idx], t0[idx], e))[0]
    T_ref = T_at(tT[idx])
    # a segment that ends inside a surface splat 1e-5 thick: float32 resolves its end to an ulp,
    # a visible step of T there, so the bound includes T at the end moved by 4 ulps
    lo, hi = tT[idx].copy(), tT[idx].copy()
    for _ in range(4):
        lo = np.nextafter(lo, np.float32(-np.inf))
        hi = np.nextafter(hi, np.float32(np.inf))
    shift = np.maximum(np.abs(T_at(lo) - T_ref), np.abs(T_at(hi) - T_ref))
    err = np.abs(T[idx].astype(np.float64) - T_ref)
    tol = REL * np.maximum(T_ref, 1 - T_ref) + shift
    assert np.all(err <= tol), (err - tol).max()

    ref = orc.sample_free_flight(s, r, u[idx], u2[idx])
    p, pr = prim[idx], ref["prim"]
    mism = np.nonzero(p != pr)[0]
    for j in mism:
        ok = p[j] >= 0 and pr[j] >= 0 and ref["race_margin"][j] < 1e-4
        for du in (-REL, REL):
            rj = scenes.Rays(r.o[j:j + 1], r.d[j:j + 1], r.t0[j:j + 1], r.t1[j:j + 1])
            f = orc.sample_free_flight(s, rj, np.clip(u[idx][j:j + 1] + du, 0, 1 - 2 ** -24), u2[idx][j:j + 1])
            ok |= f["prim"][0] == p[j]
        assert ok, (int(idx[j]), int(p[j]), int(pr[j]))
    parity_note(f"full size: {len(mism)} of 256 sampled rays pick another primitive than the oracle, all explained")
    assert len(mism) <= 4, len(mism)
    same = (p == pr) & (p >= 0)
    span = (r.t1 - r.t0).astype(np.float64)
    assert np.all(np.abs(tu[idx][same] - ref["t_u"][same]) <= REL * span[same])
    assert np.all(np.abs(tsp[idx][same] - ref["t_spawn"][same]) <= REL * span[same])
    esc = p < 0
    assert np.all(tu[idx][esc] == r.t1[esc])


def test_full_size_white_furnace():
    """The renderer at the benchmark's size (1M-primitive room, 1024 x 1024, one launch sequence
    as the benchmark runs it) on a property that holds at any size: with every primitive a
    Lambertian of albedo 1, no emitters, no area light and a unit background, a path's weight
    stays exactly 1, so every sample is 1 (it escaped) or 0 (it reached the depth limit)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_09733_gb300 import build, ugp
    build.build()
    W = H = 1024
    s = scenes.room_scene(1_000_000, width=W, height=H)
    s.mtype[:] = scenes.MAT_DIFFUSE
    s.albedo[:] = 1.0
    s.emission[:] = 0.0
    s.lights = scenes.Lights(bg=(1.0, 1.0, 1.0))
    bvh, mats, cam, li = ugp.scene_to_device(s)
    r = ugp.Renderer(W, H)
    cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
    acc, _ = r.render(bvh, mats, cam, li, 1, 14, seed=7, ray_counts=cnt)
    torch.cuda.synchronize()
    a = acc.double().cpu().numpy()
    c = cnt.cpu().numpy()
    assert c[2] == 0 and c[0] > W * H
    assert np.all(np.abs(a - np.round(a)) < 1e-5) and a.min() >= 0.0 and a.max() <= 1.0 + 1e-5
    escaped = np.round(a[..., 0]).mean()
    assert 0.05 < escaped < 1.0   # the room is open on the camera's side
