"""Pins of the oracle's learned guide (vMF-mixture proposal, its training loss and Adam).

What fixes each part independently of the oracle's own code:
* BF16 rounding: torch's float32 -> bfloat16 conversion (round to nearest even).
* Encoding: trigonometric identities between the features (sin^2 + cos^2 = 1, the double
  angle formulas tie each frequency to the previous one) and the raw angle features against
  the direction they encode.
* Forward pass: invariances of a ReLU network (permuting hidden units, positive rescaling
  between consecutive layers), a hand-built network with a known output, and the effect of
  BF16 rounding on a crafted activation.
* Mixture: the density integrates to 1 over the sphere (Gauss-Legendre x uniform quadrature);
  samples follow the density (chi-square over equal-area bins against quadrature); the mean
  cosine of a vMF lobe is the Langevin function coth(kappa) - 1/kappa.
* Loss gradient: central finite differences in FP64, on the head outputs and on the full
  parameter vector (BF16 rounding off), and torch autograd on the whole gradient.
* Adam: closed form of the first step and of a constant gradient.
* One-sample MIS: a guided render has the plain render's mean (unbiasedness, Sec. 6).
"""
import math

import numpy as np
import pytest
import torch

from paper_2406_09733_gb300 import scenes

CFG = scenes.GuideConfig()


class _Cfg:
    def __init__(self, rb, base=CFG):
        self.pos_lo, self.pos_hi = base.pos_lo, base.pos_hi
        self.kappa_min, self.kappa_max = base.kappa_min, base.kappa_max
        self.round_bf16 = rb


EXACT = _Cfg(0)


# ----------------------------------------------------------------------------- BF16 rounding
def test_bf16_round_matches_torch(orc):
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.uniform(-8, 8, 4000),
                        [0.0, -0.0, 1.0, -1.0, 65504.0, 1e-30]]).astype(np.float32)
    # exact ties: 1 + 2^-8 (rounds to even, down) and 1 + 3 * 2^-8 (rounds to even, up)
    x = np.concatenate([x, np.float32([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8)])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = orc.bf16_round(x.astype(np.float64))
    assert np.array_equal(got, ref)
    assert got[-3] == 1.0 and got[-2] == 1 + 4 * 2 ** -8


# ----------------------------------------------------------------------------- encoding
def test_encoding_identities(orc):
    b = scenes.guide_batch(500, seed=3)
    f = orc.guide_encode(EXACT, b.x, b.wo, round_bf16=0)
    assert f.shape == (500, 64)
    # sin^2 + cos^2 = 1 for every pair
    pairs = f[:, :52].reshape(500, 26, 2)
    assert np.allclose((pairs ** 2).sum(-1), 1.0, atol=1e-14)
    # frequencies double from one pair to the next: sin 2a = 2 sin a cos a, cos 2a = cos^2 - sin^2
    for base, nl in ((0, 6), (12, 6), (24, 6), (36, 4), (44, 4)):
        for l in range(nl - 1):
            s0, c0 = f[:, base + 2 * l], f[:, base + 2 * l + 1]
            s1, c1 = f[:, base + 2 * l + 2], f[:, base + 2 * l + 3]
            assert np.allclose(s1, 2 * s0 * c0, atol=1e-12)
            assert np.allclose(c1, c0 ** 2 - s0 ** 2, atol=1e-12)
    # lowest position frequency is pi * x_normalised (x clamped to the box)
    xn = np.clip(b.x.astype(np.float64), 0, 1)
    assert np.allclose(f[:, 0], np.sin(np.pi * xn[:, 0]), atol=1e-12)
    assert np.allclose(f[:, 52:55], xn, atol=0)
    # the raw angles encode the direction
    wo = b.wo.astype(np.float64)
    assert np.allclose(np.cos(np.pi * f[:, 55]), wo[:, 2], atol=1e-12)
    ph = 2 * np.pi * (f[:, 56] - 0.5)
    st = np.sqrt(1 - wo[:, 2] ** 2)
    assert np.allclose(np.cos(ph) * st, wo[:, 0], atol=1e-6)   # float32 unit vectors
    assert np.allclose(np.sin(ph) * st, wo[:, 1], atol=1e-6)
    # the lowest direction frequency is the angle itself
    assert np.allclose(f[:, 37], wo[:, 2], atol=1e-12)            # cos(theta)
    assert np.allclose(f[:, 45], np.cos(ph), atol=1e-12)          # cos(phi)
    assert np.all(f[:, 57:] == 0)


# ----------------------------------------------------------------------------- forward
def _layers(p):
    return [(p[w].reshape(o, i).copy(), p[bb].copy())
            for (o, i), (w, bb) in zip(scenes.GUIDE_SHAPES, scenes.guide_param_slices())]


def _flat(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers]).astype(np.float32)


def test_forward_relu_invariances(orc):
    p = scenes.guide_init_params(seed=5, bias_scale=0.1)
    b = scenes.guide_batch(64, seed=6)
    Y0, _ = orc.guide_forward(EXACT, p, b.x, b.wo, round_bf16=0)
    L = _layers(p)
    rng = np.random.default_rng(1)
    # permuting the hidden units of layer 1 (rows of W1, b1, columns of W2)
    perm = rng.permutation(64)
    Lp = [list(t) for t in L]
    Lp[1][0], Lp[1][1] = L[1][0][perm], L[1][1][perm]
    Lp[2][0] = L[2][0][:, perm]
    Y1, _ = orc.guide_forward(EXACT, _flat(Lp), b.x, b.wo, round_bf16=0)
    assert np.allclose(Y1, Y0, rtol=0, atol=1e-12)
    # positive rescaling between layers 2 and 3 (powers of two keep float32 exact)
    Ls = [list(t) for t in L]
    Ls[2][0], Ls[2][1] = L[2][0] * 4.0, L[2][1] * 4.0
    Ls[3][0] = L[3][0] * 0.25
    Y2, _ = orc.guide_forward(EXACT, _flat(Ls), b.x, b.wo, round_bf16=0)
    assert np.allclose(Y2, Y0, rtol=0, atol=1e-12)
    # a permutation that is not matched by the next layer changes the output (the check bites)
    Lb = [list(t) for t in L]
    Lb[1][0], Lb[1][1] = L[1][0][perm], L[1][1][perm]
    Y3, _ = orc.guide_forward(EXACT, _flat(Lb), b.x, b.wo, round_bf16=0)
    assert np.abs(Y3 - Y0).max() > 1e-3


def test_forward_hand_built_network(orc):
    """W0 = 0, b0 = v >= 0, W1..W3 = I, b = 0: the head sees v, so Y = W4 v + b4."""
    rng = np.random.default_rng(2)
    v = rng.uniform(0, 2, 64).astype(np.float32)
    W4 = rng.normal(size=(40, 64)).astype(np.float32)
    b4 = rng.normal(size=40).astype(np.float32)
    I = np.eye(64, dtype=np.float32)
    layers = [(np.zeros((64, 64), np.float32), v), (I, np.zeros(64, np.float32)),
              (I, np.zeros(64, np.float32)), (I, np.zeros(64, np.float32)), (W4, b4)]
    b = scenes.guide_batch(8, seed=1)
    Y, _ = orc.guide_forward(EXACT, _flat(layers), b.x, b.wo, round_bf16=0)
    expect = W4.astype(np.float64) @ v.astype(np.float64) + b4
    assert np.allclose(Y, expect[None, :], rtol=0, atol=1e-12)
    # with BF16 rounding the head sees bf16(v) and bf16(W4)
    Yr, _ = orc.guide_forward(EXACT, _flat(layers), b.x, b.wo, round_bf16=1)
    tb = lambda a: torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).double().numpy()
    expect_r = tb(W4) @ tb(v) + b4
    assert np.allclose(Yr, expect_r[None, :], rtol=0, atol=1e-12)
    assert np.abs(Yr - Y).max() > 1e-4   # rounding is visible


def test_forward_matches_torch_float64(orc):
    p = scenes.guide_init_params(seed=8, bias_scale=0.2)
    b = scenes.guide_batch(200, seed=9)
    F = torch.from_numpy(orc.guide_encode(EXACT, b.x, b.wo, round_bf16=0))
    h = F
    for l, (W, bb) in enumerate(_layers(p)):
        h = torch.nn.functional.linear(h, torch.from_numpy(W).double(), torch.from_numpy(bb).double())
        if l < 4:
            h = torch.relu(h)
    Y, _ = orc.guide_forward(EXACT, p, b.x, b.wo, round_bf16=0)
    assert np.allclose(Y, h.numpy(), rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------- mixture
def _sphere_quadrature(n_ct=400, n_ph=800, seed=0):
    """Nodes and weights of Gauss-Legendre in cos(theta) x uniform in phi, in a random frame."""
    x, w = np.polynomial.legendre.leggauss(n_ct)
    ph = (np.arange(n_ph) + 0.5) * 2 * np.pi / n_ph
    ct = np.repeat(x, n_ph)
    st = np.sqrt(1 - ct ** 2)
    p = np.tile(ph, n_ct)
    dirs = np.stack([st * np.cos(p), st * np.sin(p), ct], 1)
    Q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return dirs @ Q.T, np.repeat(w, n_ph) * (2 * np.pi / n_ph)


def _random_mixture(rng, kappas):
    mu = rng.normal(size=(8, 3))
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    pi = rng.uniform(0.2, 1, 8)
    pi /= pi.sum()
    mix = np.zeros((8, 5))
    mix[:, :3], mix[:, 3], mix[:, 4] = mu, kappas, pi
    return mix


def test_mixture_normalised(orc):
    rng = np.random.default_rng(4)
    dirs, w = _sphere_quadrature()
    for kap in ([0.1] * 8, [1.0] * 8, [10.0] * 8, [0.1, 1, 3, 10, 30, 50, 80, 100]):
        mix = _random_mixture(rng, np.array(kap, float))
        q = orc.mixture_pdf(np.repeat(mix.reshape(1, 40), len(dirs), 0), dirs)
        assert abs((q * w).sum() - 1.0) < 1e-9, kap


def test_mixture_from_head_outputs(orc):
    b = scenes.guide_batch(100, seed=11)
    p = scenes.guide_init_params(seed=12, bias_scale=0.5)
    Y, mix = orc.guide_forward(CFG, p, b.x, b.wo)
    assert np.allclose(np.linalg.norm(mix[:, :, :3], axis=2), 1.0, atol=1e-14)
    assert np.allclose(mix[:, :, 4].sum(1), 1.0, atol=1e-14)
    assert np.all(mix[:, :, 3] >= CFG.kappa_min) and np.all(mix[:, :, 3] <= CFG.kappa_max)
    # kappa = kappa_min + log(1 + e^s), pi = softmax(a), as stated
    s, a = Y[:, 3::5], Y[:, 4::5]
    assert np.allclose(mix[:, :, 3], CFG.kappa_min + np.logaddexp(0, s), rtol=1e-13)
    e = np.exp(a - a.max(1, keepdims=True))
    assert np.allclose(mix[:, :, 4], e / e.sum(1, keepdims=True), rtol=1e-13)


def test_vmf_mean_cosine_is_langevin(orc):
    """E[mu . w] of a vMF lobe is coth(kappa) - 1/kappa (sampled with the mixture sampler)."""
    rng = np.random.default_rng(5)
    n = 100_000
    for kap in (0.1, 1.0, 10.0, 1e4):
        mix = _random_mixture(rng, np.full(8, kap))
        mix[:, 4] = 0.0
        mix[3, 4] = 1.0                       # one lobe only
        U = rng.random((n, 3))
        wi, pdf = orc.mixture_sample(np.repeat(mix.reshape(1, 40), n, 0), U)
        assert np.allclose(np.linalg.norm(wi, axis=1), 1.0, atol=1e-12)
        c = wi @ mix[3, :3]
        mean_c = 1 / math.tanh(kap) - 1 / kap
        var_c = 1 - 2 * mean_c / kap - mean_c ** 2   # Var of the cosine: 1 - 2 L(k)/k - L(k)^2
        assert abs(c.mean() - mean_c) < 5 * math.sqrt(var_c / n) + 1e-12, kap
        q = orc.mixture_pdf(np.repeat(mix.reshape(1, 40), n, 0), wi)
        assert np.allclose(pdf, q, rtol=1e-12)


def test_mixture_sampling_chi2(orc):
    from scipy import stats
    rng = np.random.default_rng(6)
    mix = _random_mixture(rng, np.array([0.5, 2, 5, 10, 20, 1, 3, 8], float))
    n = 400_000
    wi, _ = orc.mixture_sample(np.repeat(mix.reshape(1, 40), n, 0), rng.random((n, 3)))
    # equal-area bins: 20 bands uniform in z, 40 sectors in phi
    nb_z, nb_p = 20, 40
    iz = np.minimum(((wi[:, 2] + 1) / 2 * nb_z).astype(int), nb_z - 1)
    ip = np.minimum(((np.arctan2(wi[:, 1], wi[:, 0]) + np.pi) / (2 * np.pi) * nb_p).astype(int), nb_p - 1)
    counts = np.bincount(iz * nb_p + ip, minlength=nb_z * nb_p)
    # expected mass per bin by Gauss-Legendre in z x midpoint in phi inside each bin
    gz, gw = np.polynomial.legendre.leggauss(24)
    expect = np.zeros(nb_z * nb_p)
    sub = 24
    for a in range(nb_z):
        z0, z1 = -1 + 2 * a / nb_z, -1 + 2 * (a + 1) / nb_z
        z = 0.5 * (z1 - z0) * gz + 0.5 * (z1 + z0)
        wz = 0.5 * (z1 - z0) * gw
        for c in range(nb_p):
            p0 = -np.pi + 2 * np.pi * c / nb_p
            ph = p0 + (np.arange(sub) + 0.5) * (2 * np.pi / nb_p) / sub
            Z, P = np.meshgrid(z, ph, indexing="ij")
            W = np.outer(wz, np.full(sub, 2 * np.pi / nb_p / sub))
            st = np.sqrt(1 - Z ** 2)
            d = np.stack([st * np.cos(P), st * np.sin(P), Z], -1).reshape(-1, 3)
            q = orc.mixture_pdf(np.repeat(mix.reshape(1, 40), len(d), 0), d)
            expect[a * nb_p + c] = (q * W.ravel()).sum()
    assert abs(expect.sum() - 1) < 1e-6
    e = expect * n
    keep = e > 20
    chi2 = ((counts[keep] - e[keep]) ** 2 / e[keep]).sum() + (counts[~keep].sum() - e[~keep].sum()) ** 2 / max(e[~keep].sum(), 1)
    p = stats.chi2.sf(chi2, keep.sum())
    assert p > 1e-4, (chi2, keep.sum())


# ----------------------------------------------------------------------------- loss and gradients
def test_head_gradient_finite_differences(orc):
    rng = np.random.default_rng(7)
    for trial in range(6):
        Y = rng.normal(size=40) * 1.5
        Y[3::5] = rng.uniform(-3, 4, 8)
        wi = rng.normal(size=3)
        wi /= np.linalg.norm(wi)
        w = float(10 ** rng.uniform(-1, 1))
        loss, dY = orc.mixture_loss_grad(CFG, Y, wi, w)
        h = 1e-6
        fd = np.zeros(40)
        for j in range(40):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[j] += h
            Ym[j] -= h
            fd[j] = (orc.mixture_loss_grad(CFG, Yp, wi, w)[0] - orc.mixture_loss_grad(CFG, Ym, wi, w)[0]) / (2 * h)
        assert np.allclose(dY, fd, rtol=1e-5, atol=1e-7 * max(1, abs(loss))), (trial, np.abs(dY - fd).max())


def test_head_loss_is_negative_log_density(orc):
    rng = np.random.default_rng(8)
    p = scenes.guide_init_params(seed=3, bias_scale=0.5)
    b = scenes.guide_batch(20, seed=4)
    Y, mix = orc.guide_forward(CFG, p, b.x, b.wo)
    q = orc.mixture_pdf(mix.reshape(-1, 40), b.wi.astype(np.float64))
    for i in range(20):
        loss, _ = orc.mixture_loss_grad(CFG, Y[i], b.wi[i].astype(np.float64), 2.5)
        assert abs(loss - (-2.5 * math.log(q[i]))) < 1e-10 * max(1, abs(loss))


def test_clamped_kappa_has_no_sharpness_gradient(orc):
    cfg = _Cfg(1, scenes.GuideConfig(kappa_max=5.0))
    Y = np.zeros(40)
    Y[3::5] = 20.0             # softplus(20) + 0.1 > 5: clamped
    Y[0::5] = 1.0
    _, dY = orc.mixture_loss_grad(cfg, Y, np.array([0.0, 0.0, 1.0]), 1.0)
    assert np.all(dY[3::5] == 0)
    assert np.any(dY[4::5] != 0)


def test_full_gradient_finite_differences(orc):
    p = scenes.guide_init_params(seed=13, bias_scale=0.2)
    b = scenes.guide_batch(24, seed=14)
    loss, g = orc.guide_loss_grad(EXACT, p, b.x, b.wo, b.wi, b.weight, round_bf16=0)
    rng = np.random.default_rng(3)
    h = 1e-3   # float32 parameters: a step large against their rounding, small against curvature
    idx = []
    for (w, bb) in scenes.guide_param_slices():
        idx += list(rng.integers(w.start, w.stop, 6)) + list(rng.integers(bb.start, bb.stop, 2))
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += np.float32(h)
        pm[i] -= np.float32(h)
        hp, hm = float(pp[i]) - float(p[i]), float(p[i]) - float(pm[i])
        lp = orc.guide_loss_grad(EXACT, pp, b.x, b.wo, b.wi, b.weight, round_bf16=0)[0]
        lm = orc.guide_loss_grad(EXACT, pm, b.x, b.wo, b.wi, b.weight, round_bf16=0)[0]
        fd = (lp - lm) / (hp + hm)
        assert abs(fd - g[i]) <= 2e-4 * max(abs(g).max(), 1e-12) + 1e-3 * abs(g[i]), (i, fd, g[i])


def test_full_gradient_matches_torch_autograd(orc):
    p = scenes.guide_init_params(seed=15, bias_scale=0.2)
    b = scenes.guide_batch(300, seed=16)
    loss, g = orc.guide_loss_grad(EXACT, p, b.x, b.wo, b.wi, b.weight, round_bf16=0)
    F = torch.from_numpy(orc.guide_encode(EXACT, b.x, b.wo, round_bf16=0))
    params = [(torch.from_numpy(W).double().requires_grad_(), torch.from_numpy(bb).double().requires_grad_())
              for W, bb in _layers(p)]
    h = F
    for l, (W, bb) in enumerate(params):
        h = h @ W.T + bb
        if l < 4:
            h = torch.relu(h)
    Y = h.view(-1, 8, 5)
    mu = Y[..., :3] / Y[..., :3].norm(dim=-1, keepdim=True)
    kap = torch.clamp(CFG.kappa_min + torch.nn.functional.softplus(Y[..., 3]), max=CFG.kappa_max)
    logpi = torch.log_softmax(Y[..., 4], -1)
    wi = torch.from_numpy(b.wi.astype(np.float64))
    cos = (mu * wi[:, None, :]).sum(-1)
    logv = torch.log(kap) - math.log(2 * math.pi) - torch.log(-torch.expm1(-2 * kap)) + kap * (cos - 1)
    logq = torch.logsumexp(logpi + logv, -1)
    L = -(torch.from_numpy(b.weight.astype(np.float64)) * logq).mean()
    L.backward()
    tg = np.concatenate([np.concatenate([W.grad.numpy().ravel(), bb.grad.numpy()]) for W, bb in params])
    assert abs(L.item() - loss) < 1e-12 * max(1, abs(loss))
    assert np.allclose(g, tg, rtol=1e-9, atol=1e-12 * np.abs(tg).max())


def test_bf16_gradient_close_to_exact(orc):
    p = scenes.guide_init_params(seed=17, bias_scale=0.2)
    b = scenes.guide_batch(256, seed=18)
    _, g0 = orc.guide_loss_grad(EXACT, p, b.x, b.wo, b.wi, b.weight, round_bf16=0)
    _, g1 = orc.guide_loss_grad(EXACT, p, b.x, b.wo, b.wi, b.weight, round_bf16=1)
    cos = g0 @ g1 / np.linalg.norm(g0) / np.linalg.norm(g1)
    assert cos > 0.99
    assert np.abs(g1 - g0).max() > 0   # the rounding changes the gradient


# ----------------------------------------------------------------------------- Adam
def test_adam_closed_forms(orc):
    rng = np.random.default_rng(9)
    n = 100
    th0 = rng.normal(size=n)
    g = rng.normal(size=n) * 10 ** rng.uniform(-3, 2, n)
    lr, eps = 1e-3, 1e-8
    th, m, v = th0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, 51):
        th, m, v = orc.adam_step(th, m, v, g, t, lr=lr, b1=0.9, b2=0.99, eps=eps)
        # with a constant gradient the bias-corrected moments are g and g^2 at every step
        expect = th0 - t * lr * g / (np.abs(g) + eps)
        assert np.allclose(th, expect, rtol=0, atol=1e-12 * t), t


# ----------------------------------------------------------------------------- guided render
def test_guided_render_is_unbiased(orc):
    """One-sample MIS with a guide (random weights, a poor proposal) keeps the plain mean."""
    s = scenes.tiny_scene(n=200, seed=3, width=5, height=5)
    s.mtype[:] = scenes.MAT_DIFFUSE
    s.emission[:] = 0.0
    s.mtype[::3] = scenes.MAT_GGX
    s.roughness[:] = 0.4
    s.camera = scenes.Camera((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), (0, 1, 0), 35.0, 5, 5)
    s.lights = scenes.Lights(True, (0.2, 1.2, 0.2), (0.6, 0.0, 0.0), (0.0, 0.0, 0.6), (6.0, 6.0, 6.0),
                             (0.05, 0.05, 0.05))
    p = scenes.guide_init_params(seed=21, bias_scale=1.0)
    spp = 4096
    a1, q1, _ = orc.render(s, spp=spp, max_depth=3, seed=31, guide=(p, CFG), guide_alpha=0.5)
    a0, q0, _ = orc.render(s, spp=spp, max_depth=3, seed=32)
    m1, m0 = a1 / spp, a0 / spp
    se1 = np.sqrt(np.maximum(q1 / spp - m1 ** 2, 0) / spp)
    se0 = np.sqrt(np.maximum(q0 / spp - m0 ** 2, 0) / spp)
    z = np.abs(m1 - m0) / np.maximum(np.sqrt(se1 ** 2 + se0 ** 2), 1e-12)
    assert (z > 3.5).mean() <= 0.04, np.sort(z.ravel())[-5:]
    zi = abs(m1.sum() - m0.sum()) / math.sqrt((se1 ** 2).sum() + (se0 ** 2).sum())
    assert zi < 4, zi
    # the guide really changes the samples (a different estimator, same mean)
    assert np.abs(m1 - m0).max() > 0
