"""Pins of the oracle's path tracer (Table 1, right column).

* White furnace: albedo-1 Lambertian flakes under a unit background conserve
  energy, so every sample that escapes contributes exactly 1.
* One Gaussian under a unit background: a camera sample escapes with
  probability T = 1 - 1/2 I and otherwise scatters once and escapes with
  weight rho, so its expectation is 1 - 1/2 I (1 - rho); 1/2 I comes from
  scipy quadrature along the same jittered camera rays.
* Light sampling with MIS and phase sampling alone estimate the same image.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation

from paper_2406_09733_gb300 import scenes

K = math.sqrt(-2 * math.log(0.01))


def test_white_furnace(orc):
    s = scenes.tiny_scene(n=1000, seed=1, width=12, height=12)
    s.mtype[:] = scenes.MAT_DIFFUSE
    s.albedo[:] = 1.0
    s.emission[:] = 0.0
    s.magnitude[:] *= 5.0
    s.lights = scenes.Lights(bg=(1.0, 1.0, 1.0))
    spp = 16
    acc, acc2, (ne, _) = orc.render(s, spp=spp, max_depth=64)
    mean = acc / spp
    # each sample is exactly 1 unless its path is cut at max_depth (vanishingly rare here)
    assert np.all(mean <= 1 + 1e-12)
    assert mean.min() >= 1 - 2.0 / spp
    assert (mean == 1.0).mean() > 0.99
    assert ne > 1.5 * 144 * spp   # paths really scatter


def _camera_rays(orc, cam, px, py, spp, seed):
    """The oracle's jittered camera rays, rebuilt from its Philox stream (bounce 15, slot 0)."""
    f = np.array(cam.look, float) - np.array(cam.eye, float)
    f /= np.linalg.norm(f)
    r = np.cross(f, cam.up); r /= np.linalg.norm(r)
    up = np.cross(r, f)
    th = math.tan(math.radians(cam.vfov_deg) / 2)
    p = py * cam.width + px
    out = []
    for smp in range(spp):
        x = orc.philox4x32_10([p, smp, 15 * 16 + 0, 0], [seed & 0xffffffff, seed >> 32])
        jx, jy = (x[0] >> 8) / 2 ** 24, (x[1] >> 8) / 2 ** 24
        xs = (2 * (px + jx) / cam.width - 1) * th * cam.width / cam.height
        ys = (1 - 2 * (py + jy) / cam.height) * th
        d = f + xs * r + ys * up
        out.append(d / np.linalg.norm(d))
    return np.array(out)


def test_single_gaussian_analytic_image(orc):
    s = scenes.tiny_scene(n=1, seed=2, width=6, height=6)
    s.mean[0] = [0.5, 0.5, 0.5]
    s.scale[0] = [0.25, 0.15, 0.2]
    s.quat[0] = Rotation.from_euler("xyz", [0.3, -0.4, 0.2]).as_quat()[[3, 0, 1, 2]]
    rho = 0.35
    s.mtype[0] = scenes.MAT_DIFFUSE
    s.albedo[0] = rho
    s.magnitude[0] = np.float32(0.9 * 2 * np.pi * 0.25 * 0.15)   # non-saturating
    s.camera = scenes.Camera((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), (0, 1, 0), 30.0, 6, 6)
    s.lights = scenes.Lights(bg=(1.0, 1.0, 1.0))
    spp, seed = 2048, 7
    acc, acc2, _ = orc.render(s, spp=spp, max_depth=3, seed=seed)
    mean = acc[..., 0] / spp
    var = acc2[..., 0] / spp - mean ** 2
    w, x, y, z = s.quat[0].astype(np.float64)
    R = Rotation.from_quat([x, y, z, w]).as_matrix()
    Sig = R @ np.diag(s.scale[0].astype(np.float64) ** 2) @ R.T
    Si = np.linalg.inv(Sig)
    g0 = float(s.magnitude[0]) / ((2 * np.pi) ** 1.5 * math.sqrt(np.linalg.det(Sig)))
    mu = s.mean[0].astype(np.float64)
    eye = np.array(s.camera.eye, float)
    fails = 0
    for py in range(6):
        for px in range(6):
            dirs = _camera_rays(orc, s.camera, px, py, spp, seed)
            halfI = []
            for d in dirs[:256]:   # expectation over the pixel's jitter, estimated on a subset
                # the k-ellipsoid chord from the quadratic (x - mu)^T Si (x - mu) = k^2 (numpy)
                p0 = eye - mu
                qa, qb, qc = d @ Si @ d, 2 * d @ Si @ p0, p0 @ Si @ p0 - K * K
                disc = qb * qb - 4 * qa * qc
                if disc <= 0:
                    halfI.append(0.0)
                    continue
                t_lo, t_hi = (-qb - math.sqrt(disc)) / (2 * qa), (-qb + math.sqrt(disc)) / (2 * qa)
                dens = lambda t: g0 * math.exp(-0.5 * (p0 + t * d) @ Si @ (p0 + t * d))
                v, _ = integrate.quad(dens, max(t_lo, 0.0), t_hi, epsabs=1e-13, epsrel=1e-11)
                halfI.append(0.5 * v)
            halfI = np.array(halfI)
            assert halfI.max() < 1.0
            expect = np.mean(1 - halfI * (1 - rho))
            se = math.sqrt(max(var[py, px], 1e-12) / spp) + np.std(halfI) * (1 - rho) / math.sqrt(256)
            fails += abs(mean[py, px] - expect) > 3.5 * se
    assert fails <= 1


def test_light_sampling_mis_matches_phase_sampling(orc):
    """nee=1 (light sampling + MIS) and nee=0 (lights only through phase sampling) agree."""
    s = scenes.tiny_scene(n=200, seed=3, width=6, height=6)
    s.mtype[:] = scenes.MAT_DIFFUSE
    s.emission[:] = 0.0
    s.mtype[::3] = scenes.MAT_GGX
    s.roughness[:] = 0.4
    s.camera = scenes.Camera((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), (0, 1, 0), 35.0, 6, 6)
    s.lights = scenes.Lights(True, (0.2, 1.2, 0.2), (0.6, 0.0, 0.0), (0.0, 0.0, 0.6), (6.0, 6.0, 6.0),
                             (0.05, 0.05, 0.05))
    spp = 16384
    a1, q1, (e1, sh1) = orc.render(s, spp=spp, max_depth=3, nee=1, seed=11)
    a0, q0, (e0, sh0) = orc.render(s, spp=spp, max_depth=3, nee=0, seed=12)
    assert sh1 > 0 and sh0 == 0
    m1, m0 = a1 / spp, a0 / spp
    se1 = np.sqrt(np.maximum(q1 / spp - m1 ** 2, 0) / spp)
    se0 = np.sqrt(np.maximum(q0 / spp - m0 ** 2, 0) / spp)
    z = np.abs(m1 - m0) / np.maximum(np.sqrt(se1 ** 2 + se0 ** 2), 1e-12)
    # phase-only light hits are heavy-tailed, so per-pixel errors get a little slack
    assert (z > 3.5).mean() <= 0.03, np.sort(z.ravel())[-5:]
    zi = abs(m1.mean() - m0.mean()) / math.sqrt((se1 ** 2).sum() + (se0 ** 2).sum()) * m1.size
    assert zi < 4, zi
    assert m1.mean() > 0.01   # the light contributes
    # MIS reduces variance relative to phase sampling alone
    assert np.median(se1) < np.median(se0)


# ---------------------------------------------------------------------------- f1: light sampling of emitters
def _emitter_scene():
    """Three isotropic emitters in well separated directions from the vertex at (0.5, 0.5, 0.5),
    of different power, the first one dense enough to saturate along its centre line."""
    s = scenes.tiny_scene(n=3, seed=7)
    s.quat[:] = [1.0, 0.0, 0.0, 0.0]
    s.mean[:] = [[0.5, 0.5, 0.95], [0.85, 0.55, 0.5], [0.45, 0.15, 0.55]]
    sig = np.array([0.04, 0.03, 0.05])
    s.scale[:] = sig[:, None]
    half_I_centre = np.array([3.0, 0.4, 0.25])  # 1/2 I through the centre, unclipped: c / (4 pi sigma^2)
    s.magnitude[:] = (half_I_centre * 4 * math.pi * sig ** 2).astype(np.float32)
    s.mtype[:] = scenes.MAT_EMISSIVE
    s.emission[:] = [[4.0, 2.0, 1.0], [0.5, 3.0, 0.5], [6.0, 6.0, 6.0]]
    return s, sig


def test_ellipsoid_points_follow_the_truncated_gaussian(orc):
    """Light-sampling points: whitened radius follows the chi-3 law truncated at k (KS against
    scipy), whitened directions are isotropic, every point lies inside the ellipsoid."""
    from scipy import stats
    k = math.sqrt(-2 * math.log(0.01))
    assert abs(orc.chi3_cdf(k) - stats.chi(3).cdf(k)) < 1e-14
    s = scenes.tiny_scene(n=5, seed=8)
    i = 3
    U = np.random.default_rng(120).random((100000, 3))
    y = orc.sample_in_ellipsoid(s, i, U)
    w, x_, y_, z = s.quat[i].astype(np.float64)
    R = Rotation.from_quat([x_, y_, z, w]).as_matrix()
    zc = (y - s.mean[i].astype(np.float64)) @ R / s.scale[i].astype(np.float64)
    r = np.linalg.norm(zc, axis=1)
    assert r.max() <= k * (1 + 1e-12)
    cdf = lambda x: stats.chi(3).cdf(x) / stats.chi(3).cdf(k)
    assert stats.kstest(r, cdf).pvalue > 1e-3
    u = zc / r[:, None]
    assert np.abs(u.mean(0)).max() < 4 / math.sqrt(len(u))
    np.testing.assert_allclose(u.T @ u / len(u), np.eye(3) / 3, atol=0.01)


def test_emitter_light_sampling_matches_quadrature(orc):
    """One-sample light estimates toward emissive primitives (no MIS) average to the direct
    emission int f_p(w) sum_j P_j(w) L_e,j dw, where P_j(w) = min(1, 1/2 I_j) is the free-flight
    probability of choosing emitter j along w (Eq. 8 with the saturation clamp), and f_p the
    closed-form phase function of a Lambertian base with S = I (Sec. 6). For an isotropic
    emitter of scale sigma and magnitude c at distance D, a direction at angle theta from its
    centre passes at whitened distance d = D sin(theta) / sigma, and App. A over the clipped
    chord gives 1/2 I = c / (4 pi sigma^2) e^{-d^2/2} erf(sqrt((k^2 - d^2) / 2)). The emitters
    lie in separate directions, so their cones do not overlap."""
    from scipy.optimize import brentq
    s, sig = _emitter_scene()
    k = math.sqrt(-2 * math.log(0.01))
    x = np.array([0.5, 0.5, 0.5])
    wo = np.array([0.3, -0.2, 0.93]); wo /= np.linalg.norm(wo)
    albedo = np.array([0.8, 0.6, 0.4])
    S6 = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    ref = np.zeros(3)
    for j in range(3):
        c = s.mean[j].astype(np.float64) - x
        D = np.linalg.norm(c)
        ax = c / D
        e1 = np.cross(ax, [1.0, 0, 0] if abs(ax[0]) < 0.9 else [0, 1.0, 0]); e1 /= np.linalg.norm(e1)
        e2 = np.cross(ax, e1)
        th_max = math.asin(k * float(sig[j]) / D)
        amp = float(s.magnitude[j]) / (4 * math.pi * float(sig[j]) ** 2)

        def P(th, j=j, D=D, amp=amp):
            d = D * math.sin(th) / float(sig[j])
            return 0.0 if d >= k else min(1.0, amp * math.exp(-0.5 * d * d) * math.erf(math.sqrt(0.5 * (k * k - d * d))))

        def integrand(ph, th, ax=ax, e1=e1, e2=e2, P=P):
            w = math.cos(th) * ax + math.sin(th) * (math.cos(ph) * e1 + math.sin(ph) * e2)
            f = orc.phase_eval(scenes.MAT_DIFFUSE, albedo, 0.5, S6, wo, w)[0, 0] / albedo[0]
            return f * P(th) * math.sin(th)

        kinks = [brentq(lambda th: P(th) - 1.0 + 1e-300, 0.0, th_max, xtol=1e-15)] if P(0.0) >= 1.0 else []
        v, _ = integrate.nquad(integrand, [[0.0, 2 * math.pi], [0.0, th_max]],
                               opts=[{"epsabs": 1e-12, "epsrel": 1e-10, "limit": 200},
                                     {"epsabs": 1e-11, "epsrel": 1e-9, "limit": 200, "points": kinks}])
        ref += v * albedo * s.emission[j].astype(np.float64)
    mean, se = orc.emitter_nee(s, x, wo, scenes.MAT_DIFFUSE, albedo, 0.5, S6, n=2_000_000, seed=121)
    assert np.all(se < 0.01 * ref), (se, ref)
    assert np.all(np.abs(mean - ref) <= 4 * se), (mean, ref, se)


def test_emitter_light_sampling_render_is_unbiased(orc):
    """A scene lit only by emissive primitives renders the same with light sampling toward them
    plus MIS (nee_emitters=1) as with emitters found by phase sampling alone: the balance weights
    of the two techniques sum to one. Pixels where phase sampling never met an emitter (zero
    sample variance) have no usable error estimate and are left out of the per-pixel test."""
    s = scenes.tiny_scene(n=300, seed=9, width=12, height=12)
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
    spp = 16384
    a1, q1, (e1, sh1) = orc.render(s, spp=spp, max_depth=3, nee_emitters=1, seed=13)
    a0, q0, (e0, sh0) = orc.render(s, spp=spp, max_depth=3, nee_emitters=0, seed=14)
    assert sh1 > 0 and sh0 == 0
    m1, m0 = a1 / spp, a0 / spp
    se1 = np.sqrt(np.maximum(q1 / spp - m1 ** 2, 0) / spp)
    se0 = np.sqrt(np.maximum(q0 / spp - m0 ** 2, 0) / spp)
    seen = se0 > 0
    assert seen.mean() > 0.9
    z = np.abs(m1 - m0)[seen] / np.sqrt(se1 ** 2 + se0 ** 2)[seen]
    assert (z > 3.5).mean() <= 0.03, np.sort(z)[-5:]
    zi = abs(m1.mean() - m0.mean()) / math.sqrt((se1 ** 2).sum() + (se0 ** 2).sum()) * m1.size
    assert zi < 4, zi
    assert m1.mean() > 0.01


def test_render_with_bvh_equals_brute_force(orc):
    """The oracle's BVH finds the same intervals as its brute-force loop (in the same order), so a
    render with it is identical to the brute-force render, value for value."""
    s = scenes.room_scene(20_000, seed=8, width=12, height=10, n_clusters=6, near_specular_frac=0.2)
    a, q, n = orc.render(s, spp=4, max_depth=5, seed=3)
    b, r, m = orc.render(s, spp=4, max_depth=5, seed=3, accel=True)
    assert n == m and n[0] > 1000
    assert np.array_equal(a, b) and np.array_equal(q, r)


def test_render_rectangle_equals_the_full_render(orc):
    """A rectangle of pixels (the CPU baseline's crops) gets the same sums as the same pixels
    of a full render, and every other pixel stays zero."""
    s = scenes.tiny_scene(n=200, seed=3, width=16, height=12)
    a, q, (ne, ns) = orc.render(s, spp=2, max_depth=2, seed=1)
    b, qb, (ne2, ns2) = orc.render(s, spp=2, max_depth=2, seed=1, rect=(3, 2, 5, 4))
    m = np.zeros((12, 16), bool)
    m[2:6, 3:8] = True
    assert np.array_equal(b[m], a[m]) and np.array_equal(qb[m], q[m])
    assert np.all(b[~m] == 0) and np.all(qb[~m] == 0)
    assert 0 < ne2 < ne
    with pytest.raises(ValueError):
        orc.render(s, spp=1, max_depth=1, rect=(10, 0, 8, 2))
