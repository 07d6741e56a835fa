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
