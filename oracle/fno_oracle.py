"""FP64 CPU oracle of the learned corrector: a Fourier neural operator (FNO) forward pass,
its gradients, the mean-squared loss and one Adam update.

TEST INFRASTRUCTURE ONLY (same rule as ttsh_oracle): only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline leg may use it.  It shares no code with the CUDA path.

The corrector is not part of the paper; its definition is the Fourier neural operator of
Li et al., "Fourier Neural Operator for Parametric Partial Differential Equations" (ICLR
2021), with these choices:

  x  : (B, n, n, Cin) input channels, indexed [b][y][x][c]
  h0 = x Wp + bp                                  lift, Cin -> C
  for l = 0..L-1:
      s  = SpectralConv_l(h_l)
      z  = h_l Wl + bl + s
      h_{l+1} = GELU(z)  (no activation after the last layer)
  out = h_L Wq + bq                               projection, C -> 1

  SpectralConv(h) = irfft2( P( W * P^T( rfft2(h) ) ) ): rfft2 over (y, x), unnormalised;
  the kept modes are kx in [0, m) and ky in {0..m-1} U {n-m..n-1}; per kept mode the
  channels are mixed by a complex C x C matrix W[ky, kx] (input index first); all other
  modes are zero; irfft2 carries the 1/n^2 factor and drops the imaginary part of the kx = 0
  column after the inverse over y (numpy's convention).
  GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2.

Gradients are derived by hand with the chain rule (adjoint of each linear map written out);
tests pin them against central finite differences.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.special import erf


@dataclass(frozen=True)
class FNOConfig:
    n: int = 256
    width: int = 32
    modes: int = 16
    layers: int = 4
    cin: int = 4


def param_shapes(cfg: FNOConfig):
    """Ordered (name, shape) list; the flat parameter vector concatenates them in this order."""
    C, m, L = cfg.width, cfg.modes, cfg.layers
    shapes = [("Wp", (cfg.cin, C)), ("bp", (C,))]
    for l in range(L):
        shapes += [(f"Wr{l}", (2 * m, m, C, C)), (f"Wi{l}", (2 * m, m, C, C)),
                   (f"W{l}", (C, C)), (f"b{l}", (C,))]
    shapes += [("Wq", (C, 1)), ("bq", (1,))]
    return shapes


def unflatten(cfg, theta):
    out, o = {}, 0
    for name, shp in param_shapes(cfg):
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    assert o == theta.size
    return out


def num_params(cfg):
    return sum(int(np.prod(s)) for _, s in param_shapes(cfg))


def kept_ky(n, m):
    return np.concatenate([np.arange(m), np.arange(n - m, n)])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def spectral_conv(h, Wr, Wi, m):
    """h (B, n, n, C) -> (B, n, n, C_out); also returns the kept input modes (for dW)."""
    B, n, _, C = h.shape
    H = np.fft.rfft2(h, axes=(1, 2))                  # (B, n, n/2+1, C), [b][ky][kx][c]
    ky = kept_ky(n, m)
    Hs = H[:, ky][:, :, :m]                           # (B, 2m, m, C)
    W = Wr + 1j * Wi                                  # (2m, m, Cin, Cout)
    Ys = np.einsum("bykc,ykco->byko", Hs, W)
    Y = np.zeros((B, n, n // 2 + 1, W.shape[-1]), dtype=complex)
    Y[:, ky, :m] = Ys
    return np.fft.irfft2(Y, s=(n, n), axes=(1, 2)), Hs


def spectral_conv_backward(ds, Hs, Wr, Wi, m):
    """Adjoint of spectral_conv: returns (dh, dWr, dWi) for upstream gradient ds."""
    B, n, _, Cout = ds.shape
    ky = kept_ky(n, m)
    # y = irfft2(Y): dy/dRe Y = (c_kx/n^2) cos, dy/dIm Y = -(c_kx/n^2) sin  ->  dY = c fft2(ds)/n^2
    D = np.fft.fft2(ds, axes=(1, 2))[:, ky][:, :, :m]
    ckx = np.where(np.arange(m) == 0, 1.0, 2.0)[None, None, :, None]
    dY = D * ckx / (n * n)                            # (B, 2m, m, Cout), as dRe + i dIm
    W = Wr + 1j * Wi
    # Y_o = sum_i W_io H_i:  dH_i = sum_o conj(W_io) dY_o,  dW_io = dY_o conj(H_i)
    dHs = np.einsum("byko,ykco->bykc", dY, np.conj(W))
    dW = np.einsum("bykc,byko->ykco", np.conj(Hs), dY)
    # H = rfft2(h) on kept modes: dh = Re(sum_kept dH e^{+i theta}) = Re(n^2 ifft2(dH placed))
    full = np.zeros((B, n, n, dHs.shape[-1]), dtype=complex)
    full[:, ky, :m] = dHs
    dh = np.real(np.fft.ifft2(full, axes=(1, 2))) * (n * n)
    return dh, np.real(dW), np.imag(dW)


def forward(cfg, theta, x, keep=False):
    P = unflatten(cfg, theta)
    h = x @ P["Wp"] + P["bp"]
    cache = []
    for l in range(cfg.layers):
        s, Hs = spectral_conv(h, P[f"Wr{l}"], P[f"Wi{l}"], cfg.modes)
        z = h @ P[f"W{l}"] + P[f"b{l}"] + s
        cache.append((h, z, Hs))
        h = gelu(z) if l < cfg.layers - 1 else z
    out = (h @ P["Wq"] + P["bq"])[..., 0]
    return (out, cache, h) if keep else out


def loss(cfg, theta, x, target):
    """Mean over all points of (out - target)^2."""
    out = forward(cfg, theta, x)
    return float(np.mean((out - target) ** 2))


def loss_and_grad(cfg, theta, x, target):
    P = unflatten(cfg, theta)
    out, cache, hL = forward(cfg, theta, x, keep=True)
    npts = out.size
    dout = 2.0 * (out - target) / npts                # (B, n, n)
    G = {k: np.zeros_like(v) for k, v in P.items()}
    G["Wq"] = np.einsum("byxc,byx->c", hL, dout)[:, None]
    G["bq"] = np.array([dout.sum()])
    dh = dout[..., None] * P["Wq"][:, 0]
    for l in reversed(range(cfg.layers)):
        h, z, Hs = cache[l]
        dz = dh * gelu_grad(z) if l < cfg.layers - 1 else dh
        G[f"W{l}"] = np.einsum("byxi,byxo->io", h, dz)
        G[f"b{l}"] = dz.sum(axis=(0, 1, 2))
        dh_s, G[f"Wr{l}"], G[f"Wi{l}"] = spectral_conv_backward(dz, Hs, P[f"Wr{l}"], P[f"Wi{l}"], cfg.modes)
        dh = dz @ P[f"W{l}"].T + dh_s
    G["Wp"] = np.einsum("byxi,byxo->io", x, dh)
    G["bp"] = dh.sum(axis=(0, 1, 2))
    grad = np.concatenate([G[name].reshape(-1) for name, _ in param_shapes(cfg)])
    return float(np.mean((out - target) ** 2)), grad


def adam_update(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; t is the 1-based step."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
