"""Pins of the oracle's appearance model (Sec. 6, Eq. 11-12, App. B).

Quadrature over the sphere (Gauss-Legendre in cos(theta) x uniform phi) and
numpy's eigen-decomposition are the independent references; statistical checks
use fixed seeds and chi^2 / standard-error bounds.
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.stats import chi2 as chi2d

DIFFUSE, GGX = 0, 1


def sphere_grid(nt=160, nphi=320, axis=(0, 0, 1)):
    """Quadrature nodes/weights on S^2 (exact for smooth integrands), optionally rotated."""
    x, w = np.polynomial.legendre.leggauss(nt)
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    pts = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wts = (w[:, None] * np.full(nphi, 2 * np.pi / nphi)[None]).reshape(-1)
    a = np.asarray(axis, float)
    a /= np.linalg.norm(a)
    R = Rotation.align_vectors([a], [[0, 0, 1]])[0].as_matrix()
    return pts @ R.T, wts


def random_S(rng, lo=0.2, hi=1.0):
    R = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
    ev = rng.uniform(lo, hi, 3)
    S = R @ np.diag(ev) @ R.T
    return np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]]), S


def unit(rng, n=None):
    v = rng.normal(size=3 if n is None else (n, 3))
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def test_sggx_projected_area_identity(orc):
    """int D(n) <n.w> dn = sigma(w) = sqrt(w^T S w) (the SGGX normalisation)."""
    rng = np.random.default_rng(1)
    pts, wts = sphere_grid()
    for _ in range(6):
        S6, S = random_S(rng)
        _, D = orc.sggx_eval(S6, pts)
        for _ in range(3):
            w = unit(rng)
            lhs = np.sum(wts * D * np.maximum(0, pts @ w))
            sig, _ = orc.sggx_eval(S6, w)
            assert abs(lhs - sig[0]) < 1e-4 * sig[0]
            assert abs(sig[0] - math.sqrt(w @ S @ w)) < 1e-12
    # isotropic flakes: D = 1 / pi
    _, D = orc.sggx_eval([1, 1, 1, 0, 0, 0], pts[:10])
    np.testing.assert_allclose(D, 1 / np.pi, rtol=1e-12)


def test_vndf_sampling_chi2(orc):
    rng = np.random.default_rng(2)
    for trial in range(3):
        S6, _ = random_S(rng, 0.05, 1.0)
        wo = unit(rng)
        n = 200000
        U = rng.random((n, 2))
        ns = orc.sggx_sample_vndf(S6, wo, U)
        assert np.all(ns @ wo > -1e-12)
        np.testing.assert_allclose(np.linalg.norm(ns, axis=1), 1, atol=1e-12)
        # bins in the frame of wo: 10 bands of cos, 12 sectors of phi
        b1 = np.cross(wo, [1.0, 0, 0]); b1 /= np.linalg.norm(b1); b2 = np.cross(wo, b1)
        def bins(v):
            c = np.clip(v @ wo, 0, 1 - 1e-12)
            ph = np.arctan2(v @ b2, v @ b1) % (2 * np.pi)
            return np.minimum((c * 10).astype(int), 9) * 12 + np.minimum((ph / (2 * np.pi) * 12).astype(int), 11)
        counts = np.bincount(bins(ns), minlength=120)
        pts, wts = sphere_grid(400, 480, axis=wo)
        dv = orc.sggx_dvis(S6, wo, pts)
        vis = pts @ wo > 0
        prob = np.bincount(bins(pts[vis]), weights=(wts * dv)[vis], minlength=120)
        assert abs(prob.sum() - 1) < 2e-3
        exp = prob / prob.sum() * n
        m = exp > 10
        chi2 = np.sum((counts[m] - exp[m]) ** 2 / exp[m])
        assert chi2 < chi2d.ppf(0.999, m.sum() - 1) * 1.5, (chi2, m.sum())


def test_lambert_sphere_closed_form(orc):
    """S = I with a Lambertian base: Eq. 12 by quadrature equals the closed form, and integrates to rho."""
    rng = np.random.default_rng(3)
    rho = np.array([0.3, 0.6, 0.9])
    pts, wts = sphere_grid(200, 400)
    for _ in range(5):
        wo, wi = unit(rng), unit(rng)
        # Eq. 12 with D = 1/pi and D_wo(n) = D(n) <n.wo> / sigma, sigma = 1
        integrand = ((1 / np.pi) * np.maximum(0, pts @ wo) / np.pi * np.maximum(0, pts @ wi))[:, None] * rho[None]
        ref = (wts[:, None] * integrand).sum(0)
        got = orc.phase_eval(DIFFUSE, rho, 0.3, [1, 1, 1, 0, 0, 0], wo, wi, mode=2)[0]
        # the integrand has kinks on two great circles, so the product rule converges slowly
        np.testing.assert_allclose(got, ref, rtol=2e-4)
    # backscatter: int <n.a>^2 dn = 2 pi / 3, so f_p = rho * 2 / (3 pi); forward: no overlap
    a = unit(rng)
    np.testing.assert_allclose(orc.phase_eval(DIFFUSE, rho, 0.3, [1, 1, 1, 0, 0, 0], a, a, mode=2)[0],
                               rho * 2 / (3 * np.pi), rtol=1e-12)
    np.testing.assert_allclose(orc.phase_eval(DIFFUSE, rho, 0.3, [1, 1, 1, 0, 0, 0], a, -a, mode=2)[0],
                               0.0, atol=1e-15)
    wo = unit(rng)
    f = orc.phase_eval(DIFFUSE, rho, 0.3, [1, 1, 1, 0, 0, 0], wo, pts, mode=2)
    np.testing.assert_allclose((wts[:, None] * f).sum(0), rho, rtol=1e-6)


def test_ggx_microfacet_normalisation_reciprocity_furnace(orc):
    rng = np.random.default_rng(4)
    nrm = np.array([0, 0, 1.0])
    pts, wts = sphere_grid(300, 300)
    up = pts[:, 2] > 0
    F0 = np.array([1.0, 1.0, 1.0])
    for alpha in (0.05, 0.2, 0.5):
        # projected-area normalisation of D: int D(h) <h.n> dh = 1, via the oracle's f at wo = n:
        # with wo = n, f <n.wi> = F D G2 / 4 and the half-vector map -- use instead the
        # furnace bound below; D itself is checked through the sampler's weights.
        for _ in range(3):
            wo = unit(rng)
            wo[2] = abs(wo[2]) + 0.05
            wo /= np.linalg.norm(wo)
            f = orc.base_bsdf(GGX, F0, alpha, pts[up], wo, nrm)[:, 0]
            alb = np.sum(wts[up] * f)
            assert alb <= 1.0 + 2e-3
            if alpha <= 0.05 and wo[2] > 0.5:
                assert alb > 0.97
            # sampling weight mean equals the albedo (visible-normal sampling, Heitz 2018)
            U = rng.random((100000, 2))
            h = orc.ggx_sample_vn(alpha, wo, nrm, U)
            wi = 2 * (h @ wo)[:, None] * h - wo
            fw = orc.base_bsdf(GGX, F0, alpha, wi, wo, nrm)[:, 0]
            G1 = 1 / (1 + 0.5 * (-1 + math.sqrt(1 + alpha ** 2 * (1 - wo[2] ** 2) / wo[2] ** 2)))
            Dm = alpha ** 2 / (np.pi * ((h[:, 2] ** 2) * (alpha ** 2 - 1) + 1) ** 2)
            pdf_wi = G1 * Dm * np.maximum(0, h @ wo) / wo[2] / (4 * np.maximum(1e-300, h @ wo))
            ok = wi[:, 2] > 0
            est = np.where(ok, fw / np.maximum(pdf_wi, 1e-300), 0).mean()
            se = np.where(ok, fw / np.maximum(pdf_wi, 1e-300), 0).std() / math.sqrt(len(U))
            assert abs(est - alb) < 4 * se + 3e-3
    # reciprocity of the BRDF: f(wi, wo) / <n.wi> = f(wo, wi) / <n.wo>
    for _ in range(20):
        wi, wo = unit(rng), unit(rng)
        wi[2], wo[2] = abs(wi[2]), abs(wo[2])
        a = orc.base_bsdf(GGX, [0.4, 0.5, 0.6], 0.3, wi, wo, nrm)[0] / wi[2]
        b = orc.base_bsdf(GGX, [0.4, 0.5, 0.6], 0.3, wo, wi, nrm)[0] / wo[2]
        np.testing.assert_allclose(a, b, rtol=1e-12)


def _phase_quadrature(orc, mtype, rho, alpha, S6, wo, wi, pts, wts):
    """Eq. 12 by quadrature over flake normals: int D_wo(n) f(wi, wo; n) dn."""
    dv = orc.sggx_dvis(S6, wo, pts)
    m = dv > 0
    f = np.stack([orc.base_bsdf(mtype, rho, alpha, wi, wo, n)[0] for n in pts[m]])
    return (wts[m, None] * dv[m, None] * f).sum(0)


@pytest.mark.parametrize("mtype,alpha", [(DIFFUSE, 0.3), (GGX, 0.35)])
def test_stochastic_estimator_is_unbiased(orc, mtype, alpha):
    rng = np.random.default_rng(5 + mtype)
    rho = np.array([0.7, 0.5, 0.3])
    S6, _ = random_S(rng, 0.3, 1.0)
    wo = unit(rng)
    pts, wts = sphere_grid(90, 180)
    for _ in range(2):
        wi = unit(rng)
        if mtype == GGX:  # keep the specular lobe within reach of both techniques
            wi = wo + 0.6 * unit(rng)
            wi /= np.linalg.norm(wi)
        ref = _phase_quadrature(orc, mtype, rho, alpha, S6, wo, wi, pts, wts)
        n = 200000
        est = orc.phase_eval(mtype, rho, alpha, S6, wo, np.tile(wi, (n, 1)), rng.random((n, 6)), mode=1)
        m, se = est.mean(0), est.std(0) / math.sqrt(n)
        assert np.all(np.abs(m - ref) < 4 * se + 2e-3 * ref.max()), (m, ref, se)


def test_microflake_reciprocity(orc):
    """sigma(wo) f_p(wi, wo) = sigma(wi) f_p(wo, wi) for a symmetric base BRDF."""
    rng = np.random.default_rng(7)
    S6, _ = random_S(rng, 0.3, 1.0)
    rho = np.array([0.5, 0.5, 0.5])
    pts, wts = sphere_grid(90, 180)
    for _ in range(3):
        wi, wo = unit(rng), unit(rng)
        a = orc.sggx_eval(S6, wo)[0][0] * _phase_quadrature(orc, DIFFUSE, rho, 0.3, S6, wo, wi, pts, wts)
        b = orc.sggx_eval(S6, wi)[0][0] * _phase_quadrature(orc, DIFFUSE, rho, 0.3, S6, wi, wo, pts, wts)
        np.testing.assert_allclose(a, b, rtol=2e-3, atol=1e-6)


@pytest.mark.parametrize("mtype,alpha,iso", [(DIFFUSE, 0.3, True), (DIFFUSE, 0.3, False), (GGX, 0.3, False)])
def test_phase_sampling_matches_phase_function(orc, mtype, alpha, iso):
    """E[weight g(wi)] under phase sampling equals int f_p(wi, wo) g(wi) dwi (Sec. 6)."""
    rng = np.random.default_rng(9 + mtype + 2 * iso)
    rho = np.array([0.8, 0.6, 0.4])
    S6 = np.array([1, 1, 1, 0, 0, 0.0]) if iso else random_S(rng, 0.2, 1.0)[0]
    wo = unit(rng)
    g = lambda v: 1.0 + v @ np.array([0.3, -0.5, 0.7])   # a smooth test function
    n = 200000
    wi, w, ok = orc.phase_sample(mtype, rho, alpha, S6, wo, rng.random((n, 4)))
    lhs = (w[:, 0] * g(wi)).mean()
    lse = (w[:, 0] * g(wi)).std() / math.sqrt(n)
    if iso:
        pts, wts = sphere_grid(120, 240)
        f = orc.phase_eval(mtype, rho, alpha, S6, wo, pts, mode=2)[:, 0]
        rhs, rse = np.sum(wts * f * g(pts)), 0.0
    else:   # independent estimate: uniform directions times the stochastic phase estimate
        d = unit(rng, n)
        f = orc.phase_eval(mtype, rho, alpha, S6, wo, d, rng.random((n, 6)), mode=1)[:, 0]
        vals = 4 * np.pi * f * g(d)
        rhs, rse = vals.mean(), vals.std() / math.sqrt(n)
    assert abs(lhs - rhs) < 4 * math.hypot(lse, rse) + 1e-3, (lhs, rhs, lse, rse)


def test_roughened_sggx_eigen_structure(orc):
    """App. B: same eigenvectors, eigenvalues (s1 + a^2 s3, s2 + a^2 s3, s3)."""
    rng = np.random.default_rng(11)
    for _ in range(10):
        S6, S = random_S(rng, 0.01, 1.0)
        a = rng.uniform(0.02, 0.8)
        r6 = orc.sggx_roughen(S6, a)
        Sr = np.array([[r6[0], r6[3], r6[4]], [r6[3], r6[1], r6[5]], [r6[4], r6[5], r6[2]]])
        ev, V = np.linalg.eigh(S)
        ref = V @ np.diag([ev[0] + a * a * ev[2], ev[1] + a * a * ev[2], ev[2]]) @ V.T
        np.testing.assert_allclose(Sr, ref, atol=1e-10)


def test_approximate_pdf_covers_the_phase_function(orc):
    """The MIS pdf of App. B is positive wherever the phase function is."""
    rng = np.random.default_rng(12)
    for mtype in (DIFFUSE, GGX):
        S6, _ = random_S(rng, 0.1, 1.0)
        wo = unit(rng)
        d = unit(rng, 4000)
        f = orc.phase_eval(mtype, [0.5, 0.5, 0.5], 0.3, S6, wo, d, rng.random((4000, 6)), mode=1)[:, 0]
        p = orc.phase_pdf_approx(mtype, [0.5, 0.5, 0.5], 0.3, S6, wo, d)
        assert np.all(np.isfinite(p)) and np.all(p >= 0)
        assert np.all(p[f > 1e-6] > 0)


# ---------------------------------------------------------------------------- f4: Disney base
DIS = np.array([0.2, 0.3, 0.5, 0.2, 0.4, 0.3, 0.5, 0.6, 0.7])  # metallic .. clearcoat gloss
C_BASE = np.array([0.8, 0.5, 0.3])


def _dis(**kw):
    names = ["metallic", "subsurface", "specular", "specular_tint", "roughness", "sheen", "sheen_tint",
             "clearcoat", "clearcoat_gloss"]
    d = DIS.copy()
    for k, v in kw.items():
        d[names.index(k)] = v
    return d


def test_disney_special_cases(orc):
    """Metallic 1 without clearcoat is the GGX base with F0 = C and alpha = roughness^2 (the
    pinned GGX of the oracle); at normal incidence (wi = wo = n) the diffuse term is C / pi for
    any roughness, the subsurface term 0.625 C / pi, and sheen vanishes."""
    rng = np.random.default_rng(30)
    n = np.array([0.0, 0.0, 1.0])
    for r in (0.1, 0.45, 0.9):
        d = _dis(metallic=1.0, clearcoat=0.0, roughness=r)
        wo = np.array([0.3, -0.4, 0.85]); wo /= np.linalg.norm(wo)
        wi = unit(rng, 200)
        wi[:, 2] = np.abs(wi[:, 2])
        got = orc.disney_f(C_BASE, d, wi, wo, n)
        ref = np.stack([orc.base_bsdf(GGX, C_BASE, max(1e-3, r * r), w, wo, n)[0] for w in wi])
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-15)
    for r in (0.0, 0.5, 1.0):
        base = dict(metallic=0.0, specular=0.0, clearcoat=0.0, roughness=r)
        f0 = orc.disney_f(C_BASE, _dis(subsurface=0.0, sheen=0.0, **base), n, n, n)[0]
        np.testing.assert_allclose(f0, C_BASE / np.pi, rtol=1e-14)
        f1 = orc.disney_f(C_BASE, _dis(subsurface=1.0, sheen=0.0, **base), n, n, n)[0]
        np.testing.assert_allclose(f1, 0.625 * C_BASE / np.pi, rtol=1e-14)
        f2 = orc.disney_f(C_BASE, _dis(subsurface=0.0, sheen=1.0, **base), n, n, n)[0]
        np.testing.assert_allclose(f2, C_BASE / np.pi, rtol=1e-14)


def test_disney_reciprocity(orc):
    """f(wi, wo) = f(wo, wi) for the BRDF (the cosine-weighted value divided by <n.wi>)."""
    rng = np.random.default_rng(31)
    n = np.array([0.0, 0.0, 1.0])
    for _ in range(20):
        d = rng.random(9)
        C = rng.random(3)
        a, b = unit(rng), unit(rng)
        a[2], b[2] = abs(a[2]) + 0.05, abs(b[2]) + 0.05
        a /= np.linalg.norm(a); b /= np.linalg.norm(b)
        fab = orc.disney_f(C, d, a, b, n)[0] / a[2]
        fba = orc.disney_f(C, d, b, a, n)[0] / b[2]
        np.testing.assert_allclose(fab, fba, rtol=1e-12)


def test_gtr1_is_normalised(orc):
    """int D(n.h) (n.h) dh = 1 over the hemisphere, by quadrature."""
    from scipy import integrate
    for a in (0.001, 0.01, 0.1, 0.5, 0.99):
        v, _ = integrate.quad(lambda t: orc.gtr1_D(a, math.cos(t)) * math.cos(t) * math.sin(t), 0, math.pi / 2,
                              epsabs=0, epsrel=1e-11, limit=400, points=[min(0.1, 10 * a)])
        assert abs(2 * math.pi * v - 1) < 1e-8, (a, 2 * math.pi * v)


@pytest.mark.parametrize("seed", [32, 33, 34])
def test_disney_sampler_matches_its_pdf_and_the_albedo(orc, seed):
    """The base sampler's accepted samples have the mixture density: the pdf integrates (by
    quadrature) to the acceptance rate, and the mean weight f <n.wi> / pdf equals the directional
    albedo int f <n.wi> dwi by quadrature."""
    rng = np.random.default_rng(seed)
    d, C = rng.random(9), rng.random(3)
    n = np.array([0.0, 0.0, 1.0])
    wo = unit(rng); wo[2] = abs(wo[2]) + 0.1; wo /= np.linalg.norm(wo)
    pts, wts = sphere_grid(200, 400)
    up = pts[:, 2] > 0
    p = orc.disney_pdf(C, d, wo, n, pts[up])
    f = orc.disney_f(C, d, pts[up], wo, n)
    N = 400000
    wi, w, ok = orc.disney_sample(C, d, wo, n, rng.random((N, 2)))
    acc = ok.mean()
    assert abs((wts[up] * p).sum() - acc) < 4 * math.sqrt(acc * (1 - acc) / N) + 2e-4, ((wts[up] * p).sum(), acc)
    albedo = (wts[up, None] * f).sum(0)
    m, se = w.mean(0), w.std(0) / math.sqrt(N)
    assert np.all(np.abs(m - albedo) < 4 * se + 1e-3 * albedo.max()), (m, albedo, se)


def test_disney_phase_function(orc):
    """With a Disney base: the stochastic evaluation of Eq. 12 averages to its quadrature over
    flake normals, phase sampling averages to the phase function's integral (an independent
    uniform-direction estimate), and the App. B pdf is positive wherever the phase function is."""
    rng = np.random.default_rng(35)
    d = _dis(metallic=0.3, roughness=0.5, clearcoat=0.4)
    S6, _ = random_S(rng, 0.3, 1.0)
    wo = unit(rng)
    pts, wts = sphere_grid(90, 180)
    for _ in range(2):
        wi = wo + 0.8 * unit(rng)
        wi /= np.linalg.norm(wi)
        dv = orc.sggx_dvis(S6, wo, pts)
        m = dv > 0
        fb = np.stack([orc.disney_f(C_BASE, d, wi, wo, nn)[0] for nn in pts[m]])
        ref = (wts[m, None] * dv[m, None] * fb).sum(0)
        N = 200000
        est = orc.phase_eval_disney(C_BASE, d, S6, wo, np.tile(wi, (N, 1)), rng.random((N, 6)))
        mean, se = est.mean(0), est.std(0) / math.sqrt(N)
        assert np.all(np.abs(mean - ref) < 4 * se + 2e-3 * ref.max()), (mean, ref, se)
    g = lambda v: 1.0 + v @ np.array([0.3, -0.5, 0.7])
    N = 200000
    wi, w, ok = orc.phase_sample_disney(C_BASE, d, S6, wo, rng.random((N, 4)))
    lhs, lse = (w[:, 0] * g(wi)).mean(), (w[:, 0] * g(wi)).std() / math.sqrt(N)
    dirs = unit(rng, N)
    f = orc.phase_eval_disney(C_BASE, d, S6, wo, dirs, rng.random((N, 6)))[:, 0]
    vals = 4 * np.pi * f * g(dirs)
    rhs, rse = vals.mean(), vals.std() / math.sqrt(N)
    assert abs(lhs - rhs) < 4 * math.hypot(lse, rse) + 1e-3, (lhs, rhs, lse, rse)
    p = orc.phase_pdf_approx_disney(C_BASE, d, S6, wo, dirs[:4000])
    assert np.all(np.isfinite(p)) and np.all(p[f[:4000] > 1e-6] > 0)


def _golden_disney():
    from fractions import Fraction
    path = os.path.join(os.path.dirname(__file__), "golden", "disney_diffuse_grazing.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, dis, wi, wo, a, b, c, rtol = [x.strip() for x in line.split("|")]
        rows.append((name, np.array([float(x) for x in dis.split()]), [float(x) for x in wi.split()],
                     [float(x) for x in wo.split()], *[float(Fraction(x)) for x in (a, b, c)], float(rtol)))
    return rows


def _dir(cos_t, phi_deg):
    s = math.sqrt(max(0.0, 1.0 - cos_t * cos_t))
    p = math.radians(phi_deg)
    return np.array([s * math.cos(p), s * math.sin(p), cos_t])


def test_disney_diffuse_grazing_golden(orc):
    """The diffuse, subsurface and sheen terms at grazing and intermediate angles equal the values
    that Burley's published formulas reduce to there (hand-derived in the fixture): retro-
    reflection up to (1/2 + 2 roughness)^2 at grazing, Lambertian when F_D90 = 1, the Schlick
    weight (1 - cos)^5 at 60 degrees, the subsurface term's F_ss90 = roughness cos^2(theta_d), and
    the sheen weight reaching the sheen colour at theta_d = 90 degrees."""
    C = np.array([0.6, 0.3, 0.9])
    n = np.array([0.0, 0.0, 1.0])
    rows = _golden_disney()
    assert len(rows) == 12
    for name, dis, wi, wo, a, b, c, rtol in rows:
        w_i, w_o = _dir(*wi), _dir(*wo)
        got = orc.disney_f_diffuse(C, dis, w_i, w_o, n)[0] / w_i[2]
        want = a * C / np.pi + b + c * C / 0.45
        np.testing.assert_allclose(got, want, rtol=rtol, err_msg=name)
