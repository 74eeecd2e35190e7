"""Pins of the FNO oracle (no GPU): closed forms of GELU and of the spectral convolution on
single Fourier modes, linearity, central finite differences of every parameter block's
gradient, and Adam's first step."""
import numpy as np
import pytest

from oracle import fno_oracle as F


def small_cfg():
    return F.FNOConfig(n=8, width=3, modes=2, layers=2, cin=2)


def random_theta(cfg, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(F.num_params(cfg))


def test_gelu_closed_forms():
    z = np.linspace(-6, 6, 101)
    g = F.gelu(z)
    assert F.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(F.gelu(-z), g - z, atol=1e-15)         # Phi(-z) = 1 - Phi(z)
    np.testing.assert_allclose(F.gelu(np.array([1.0])), [0.8413447460685429], rtol=1e-14)  # Phi(1)
    h = 1e-6
    np.testing.assert_allclose(F.gelu_grad(z), (F.gelu(z + h) - F.gelu(z - h)) / (2 * h), atol=1e-8)


@pytest.mark.parametrize("kx,ky,kept", [(3, 2, True), (0, 2, True), (1, -3, True), (4, 1, False),
                                        (2, 4, False), (0, 0, True)])
def test_identity_spectral_conv_keeps_exactly_the_retained_modes(kx, ky, kept):
    n, m, C = 16, 4, 2
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    f = np.cos(2 * np.pi * (kx * x + ky * y) / n + 0.4)
    h = np.stack([f, 0.5 * f], axis=-1)[None]
    Wr = np.zeros((2 * m, m, C, C))
    Wr[:, :, np.arange(C), np.arange(C)] = 1.0
    s, _ = F.spectral_conv(h, Wr, np.zeros_like(Wr), m)
    np.testing.assert_allclose(s, h if kept else 0 * h, atol=1e-13)


def test_spectral_conv_mode_multiplier():
    """A single mode times a complex weight w = r e^{i phi} gives r cos(theta + phi)."""
    n, m = 16, 4
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    th = 2 * np.pi * (2 * x + 1 * y) / n
    h = np.cos(th)[None, ..., None]
    Wr = np.zeros((2 * m, m, 1, 1))
    Wi = np.zeros_like(Wr)
    r, phi = 0.7, 0.9
    Wr[1, 2, 0, 0], Wi[1, 2, 0, 0] = r * np.cos(phi), r * np.sin(phi)        # (ky=1, kx=2)
    s, _ = F.spectral_conv(h, Wr, Wi, m)
    np.testing.assert_allclose(s[0, ..., 0], r * np.cos(th + phi), atol=1e-13)


def test_forward_is_affine_in_the_projection():
    cfg = small_cfg()
    th = random_theta(cfg, 1)
    x = np.random.default_rng(2).standard_normal((2, cfg.n, cfg.n, cfg.cin))
    P = F.unflatten(cfg, th.copy())
    out = F.forward(cfg, th, x)
    th2 = th.copy()
    F.unflatten(cfg, th2)["bq"][0] += 1.5
    np.testing.assert_allclose(F.forward(cfg, th2, x), out + 1.5, atol=1e-13)
    assert out.shape == (2, cfg.n, cfg.n) and P["Wq"].shape == (cfg.width, 1)


def test_gradients_match_central_differences():
    cfg = small_cfg()
    rng = np.random.default_rng(3)
    th = random_theta(cfg, 4)
    x = rng.standard_normal((2, cfg.n, cfg.n, cfg.cin))
    t = rng.standard_normal((2, cfg.n, cfg.n))
    L0, g = F.loss_and_grad(cfg, th, x, t)
    assert L0 == pytest.approx(F.loss(cfg, th, x, t), rel=1e-14)
    # every parameter block, several entries each
    o = 0
    for name, shp in F.param_shapes(cfg):
        k = int(np.prod(shp))
        for idx in rng.choice(k, size=min(k, 5), replace=False):
            i = o + idx
            e = 1e-6
            tp, tm = th.copy(), th.copy()
            tp[i] += e
            tm[i] -= e
            fd = (F.loss(cfg, tp, x, t) - F.loss(cfg, tm, x, t)) / (2 * e)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, idx, fd, g[i])
        o += k


def test_adam_first_step_is_sign_step():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = F.adam_update(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
