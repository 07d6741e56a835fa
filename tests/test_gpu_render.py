"""GPU wavefront renderer against the FP64 oracle's path tracer.

Renders are compared per pixel and channel: |mean_gpu - mean_ref| <= 3 sqrt(se_gpu^2 + se_ref^2),
passing when at most 1 % of pixel-channels fail (0.27 % expected for Gaussian errors), plus
exact identities (white furnace) and resumability of the sample index.
"""
import math

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


def gpu_render(torch, s, spp, max_depth, seed=0, nee=True, spp_begin=0, chunks=1, emitters=False):
    from paper_2406_09733_gb300 import ugp
    bvh, mats, cam, li = ugp.scene_to_device(s)
    r = ugp.Renderer(cam.width, cam.height)
    table = ugp.build_emitter_table(bvh, mats) if emitters else None
    acc = acc2 = None
    cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
    per = spp // chunks
    for c in range(chunks):
        acc, acc2 = r.render(bvh, mats, cam, li, per, max_depth, seed=seed, spp_begin=spp_begin + c * per,
                             nee=nee, accum=acc, accum_sq=acc2, ray_counts=cnt, emitters=table)
    torch.cuda.synchronize()
    return acc.double().cpu().numpy(), acc2.double().cpu().numpy(), cnt.cpu().numpy()


def compare(a_g, q_g, n_g, a_o, q_o, n_o, z_max=3.0, frac=0.01):
    mg, mo = a_g / n_g, a_o / n_o
    sg = np.sqrt(np.maximum(q_g / n_g - mg ** 2, 0) / n_g)
    so = np.sqrt(np.maximum(q_o / n_o - mo ** 2, 0) / n_o)
    z = np.abs(mg - mo) / np.maximum(np.sqrt(sg ** 2 + so ** 2), 1e-9)
    bad = (z > z_max) & (np.abs(mg - mo) > 1e-6)
    assert bad.mean() <= frac, (bad.mean(), np.sort(z.ravel())[-6:])
    return z


def test_white_furnace_gpu(gpu, orc):
    """Albedo-1 flakes under a unit background: every sample that escapes before the depth limit
    contributes exactly 1.  Truncation at max_depth and the scattering rate match the oracle's."""
    s = scenes.tiny_scene(n=1000, seed=1, width=16, height=16)
    s.mtype[:] = scenes.MAT_DIFFUSE
    s.albedo[:] = 1.0
    s.emission[:] = 0.0
    s.magnitude[:] *= 5.0
    s.lights = scenes.Lights(bg=(1.0, 1.0, 1.0))
    spp, D = 64, 14
    a, q, cnt = gpu_render(gpu, s, spp=spp, max_depth=D)
    a_o, _, (ne_o, _) = orc.render(s, spp=spp, max_depth=D)
    mean, mean_o = a / spp, a_o / spp
    assert np.all(mean <= 1 + 1e-6) and cnt[2] == 0
    # samples are either exactly 1 or truncated (0); the truncated share matches the oracle
    k = np.round(a).astype(np.int64)
    assert np.all(np.abs(a - k) < 1e-3)
    assert abs((1 - mean).sum() - (1 - mean_o).sum()) <= 3 * math.sqrt((1 - mean_o).sum() * spp + 1) / spp
    assert abs(cnt[0] / ne_o - 1) < 0.02


def lit_scene(n=400, seed=3, w=24, h=24):
    s = scenes.tiny_scene(n=n, seed=seed, width=w, height=h)
    s.mtype[::3] = scenes.MAT_GGX
    s.roughness[:] = np.linspace(0.1, 0.6, n).astype(np.float32)
    rng = np.random.default_rng(seed)
    # a few anisotropic flake distributions
    for i in range(0, n, 5):
        R = np.linalg.qr(rng.normal(size=(3, 3)))[0]
        S = R @ np.diag(rng.uniform(0.1, 1.0, 3)) @ R.T
        s.sggx[i] = [S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]]
    s.camera = scenes.Camera((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), (0, 1, 0), 38.0, w, h)
    s.lights = scenes.Lights(True, (0.2, 1.2, 0.2), (0.6, 0.0, 0.0), (0.0, 0.0, 0.6), (6.0, 6.0, 6.0),
                             (0.2, 0.25, 0.3))
    return s


def test_render_matches_oracle_lit_scene(gpu, orc):
    s = lit_scene()
    spp_g, spp_o = 4096, 1024
    a_g, q_g, cnt = gpu_render(gpu, s, spp_g, max_depth=4, seed=5, chunks=4)
    a_o, q_o, _ = orc.render(s, spp=spp_o, max_depth=4, seed=6)
    assert cnt[1] > 0 and cnt[2] == 0
    compare(a_g, q_g, spp_g, a_o, q_o, spp_o)


def test_render_matches_oracle_tiny_scene_config(gpu, orc):
    """The 1,000-primitive random scene (one emissive primitive, no background, max depth 4) at
    64 x 64 with 4096 samples per pixel on both sides."""
    s = scenes.tiny_scene(width=64, height=64)
    spp_g, spp_o = 4096, 4096
    a_g, q_g, cnt = gpu_render(gpu, s, spp_g, max_depth=4, seed=7, chunks=4)
    a_o, q_o, _ = orc.render(s, spp=spp_o, max_depth=4, seed=8)
    assert (a_o > 0).mean() > 0.01   # one emitter, no background: sparse signal
    compare(a_g, q_g, spp_g, a_o, q_o, spp_o)


def test_render_is_resumable(gpu):
    s = lit_scene(n=200, w=12, h=12)
    a1, q1, _ = gpu_render(gpu, s, 64, max_depth=3, seed=9, chunks=1)
    a2, q2, _ = gpu_render(gpu, s, 64, max_depth=3, seed=9, chunks=4)
    np.testing.assert_allclose(a1, a2, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(q1, q2, rtol=1e-4, atol=1e-4)


def emitter_scene(n=300, seed=9, w=12, h=12):
    """Lit only by emissive primitives (a tenth of them), no area light, no background."""
    s = scenes.tiny_scene(n=n, seed=seed, width=w, height=h)
    rng = np.random.default_rng(122)
    s.mtype[:] = scenes.MAT_DIFFUSE
    s.mtype[rng.random(s.n) < 0.3] = scenes.MAT_GGX
    s.roughness[:] = 0.3
    em = rng.random(s.n) < 0.1
    s.mtype[em] = scenes.MAT_EMISSIVE
    s.scale[em] *= 3.0
    s.magnitude[em] *= 9.0
    s.emission[:] = 0.0
    s.emission[em] = (rng.uniform(0.5, 2.0, (em.sum(), 1)) * rng.uniform(0.3, 1.0, (em.sum(), 3))).astype(np.float32)
    s.lights = scenes.Lights(False, (0, 0, 0), (0, 0, 0), (0, 0, 0), (0, 0, 0), (0.0, 0.0, 0.0))
    return s


def test_emitter_light_sampling_matches_oracle(gpu, orc):
    """Light sampling of emissive primitives with MIS against phase sampling (same Philox streams,
    emitters in caller order on both sides) against the oracle's render, and against the GPU's
    own render without it (unbiased: the balance weights sum to one)."""
    s = emitter_scene()
    spp, D = 8192, 3
    a, q, cnt = gpu_render(gpu, s, spp=spp, max_depth=D, seed=13, emitters=True)
    a_o, q_o, (ne_o, ns_o) = orc.render(s, spp=spp, max_depth=D, seed=13, nee_emitters=1)
    assert cnt[1] > 0 and ns_o > 0 and cnt[2] == 0
    assert abs(cnt[1] / ns_o - 1) < 0.02
    compare(a, q, spp, a_o, q_o, spp)
    # the image mean against phase sampling alone, at more samples: the phase-only estimator is
    # heavy-tailed, so its sample variance settles slowly
    n2 = 16384
    a1, q1, _ = gpu_render(gpu, s, spp=n2, max_depth=D, seed=20, emitters=True)
    a0, q0, cnt0 = gpu_render(gpu, s, spp=n2, max_depth=D, seed=21)
    assert cnt0[1] == 0
    m, m0 = a1 / n2, a0 / n2
    se = np.sqrt(np.maximum(q1 / n2 - m ** 2, 0) / n2)
    se0 = np.sqrt(np.maximum(q0 / n2 - m0 ** 2, 0) / n2)
    zi = abs(m.mean() - m0.mean()) / math.sqrt((se ** 2).sum() + (se0 ** 2).sum()) * m.size
    assert zi < 4, zi


def test_emitter_table_errors(gpu):
    from paper_2406_09733_gb300 import ugp
    torch = gpu
    s = emitter_scene(n=50, w=4, h=4)
    s.lights = scenes.Lights(True, (0.2, 1.2, 0.2), (0.6, 0.0, 0.0), (0.0, 0.0, 0.6), (6.0, 6.0, 6.0),
                             (0.0, 0.0, 0.0))
    bvh, mats, cam, li = ugp.scene_to_device(s)
    table = ugp.build_emitter_table(bvh, mats)
    r = ugp.Renderer(cam.width, cam.height)
    with pytest.raises(ugp.UgpError):  # a table off its 256-byte alignment
        r.render(bvh, mats, cam, li, 1, 2, nee=True, emitters=table[1:])
    acc, _ = r.render(bvh, mats, cam, li, 1, 2, nee=False, emitters=table)
    torch.cuda.synchronize()
    assert torch.isfinite(acc).all()


def test_area_light_and_emitters_match_oracle(gpu, orc):
    """Both light samples at every vertex, one of the area light and one of an emissive primitive,
    each balanced against phase sampling, against the oracle's render with both."""
    s = emitter_scene(seed=11)
    s.lights = scenes.Lights(True, (0.35, 1.05, 0.35), (0.3, 0.0, 0.0), (0.0, 0.0, 0.3), (8.0, 8.0, 8.0),
                             (0.1, 0.15, 0.2))
    spp, D = 8192, 3
    a, q, cnt = gpu_render(gpu, s, spp=spp, max_depth=D, seed=17, emitters=True)
    a_o, q_o, (ne_o, ns_o) = orc.render(s, spp=spp, max_depth=D, seed=17, nee_emitters=1)
    assert cnt[1] > 0 and ns_o > 0 and cnt[2] == 0
    assert abs(cnt[1] / ns_o - 1) < 0.02
    compare(a, q, spp, a_o, q_o, spp)
    # the two light samples together against the area light's alone: the same image
    a1, q1, cnt1 = gpu_render(gpu, s, spp=spp, max_depth=D, seed=19)
    assert cnt1[1] < cnt[1]
    compare(a, q, spp, a1, q1, spp, z_max=4.0)

