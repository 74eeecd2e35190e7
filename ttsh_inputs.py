"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the CPU oracle.

This module holds no arithmetic of the method itself (no transform, no time step, no
mask filtering).  It only builds the inputs the paper's workloads are made of:

* the binary masks K_naive of Appendix E (circle: masked where |x| >= R; dumbbell: the
  logical AND of two circle masks, i.e. masked outside both circles);
* the uniform-noise initial velocity ("random initial state", Sec. III.A and Sec. IV.A),
  drawn with the counter-based SplitMix64 generator of Steele, Lea & Flood,
  "Fast splittable pseudorandom number generators" (OOPSLA 2014);
* the model constants of Table I.

Conventions (readings of the paper, each listed in the design notes):
* grid coordinate x_i = (i - N/2) * dx on both axes, arrays indexed [y][x] (row-major), so
  the circle centre sits exactly on grid point (N/2, N/2);
* draw number 2*p is v_x and 2*p + 1 is v_y at flattened point p = y*N + x; a draw z maps to
  u = (z >> 11) * 2**-53 in [0, 1) and to amplitude * (2u - 1); masked points get 0.
"""
from __future__ import annotations

import numpy as np

# Table I (Appendix B) model constants; dt from Table I, dx is per-workload.
TABLE1 = dict(a=0.5, b=1.6, lam=9.0, gamma_v=40.0, gamma_w=4.0, dt=0.01)

_GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index) -> np.ndarray:
    """Output number `index` (0-based) of the SplitMix64 stream started at `seed`.

    SplitMix64 advances its state by the golden gamma and then applies the 64-bit finaliser;
    output i therefore depends only on seed + (i + 1) * gamma (counter-based form).
    """
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx + np.uint64(1)) * _GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, index) -> np.ndarray:
    """53-bit uniform double in [0, 1) from SplitMix64 draw `index`."""
    z = splitmix64(seed, index)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def grid_coords(n: int, dx: float):
    """Coordinates (X, Y), each shape (n, n) indexed [y][x], with x_i = (i - n/2) dx."""
    c = (np.arange(n, dtype=np.float64) - n // 2) * dx
    X, Y = np.meshgrid(c, c, indexing="xy")
    return X, Y


def circle_mask(n: int, dx: float, radius: float, center=(0.0, 0.0)) -> np.ndarray:
    """Binary K_naive for a circular domain: 1 (masked) where |x - c| >= R, else 0."""
    X, Y = grid_coords(n, dx)
    r2 = (X - center[0]) ** 2 + (Y - center[1]) ** 2
    return (r2 >= radius * radius).astype(np.uint8)


def dumbbell_mask(n: int, dx: float, radius: float, distance: float) -> np.ndarray:
    """Binary K_naive for a dumbbell: logical AND of two circle masks centred at (+-D/2, 0)."""
    left = circle_mask(n, dx, radius, (-0.5 * distance, 0.0))
    right = circle_mask(n, dx, radius, (0.5 * distance, 0.0))
    return (left & right).astype(np.uint8)


def blob_mask(n: int, dx: float, seed: int, lobes: int = 5, obstacle: float = 1.0) -> np.ndarray:
    """An irregular binary domain: the union of `lobes` discs (centres and radii from
    SplitMix64 draws) is unmasked, except a masked disc obstacle of radius `obstacle` at the
    first lobe's centre.  Stands in for the paper's arbitrary-image boundaries."""
    X, Y = grid_coords(n, dx)
    L = n * dx
    u = uniform01(seed, np.arange(3 * lobes))
    inside = np.zeros((n, n), dtype=bool)
    for i in range(lobes):
        cx, cy = (u[3 * i] - 0.5) * 0.3 * L, (u[3 * i + 1] - 0.5) * 0.3 * L
        r = (0.12 + 0.08 * u[3 * i + 2]) * L
        inside |= (X - cx) ** 2 + (Y - cy) ** 2 < r * r
        if i == 0:
            ox, oy = cx, cy
    inside &= (X - ox) ** 2 + (Y - oy) ** 2 >= obstacle * obstacle
    return (~inside).astype(np.uint8)


def noise_velocity(mask: np.ndarray, seed: int, amplitude: float = 0.01):
    """Uniform noise U[-A, A) for (v_x, v_y) at unmasked points (mask == 0), zero elsewhere."""
    n = mask.shape[0]
    p = np.arange(n * n, dtype=np.uint64)
    vx = amplitude * (2.0 * uniform01(seed, 2 * p) - 1.0)
    vy = amplitude * (2.0 * uniform01(seed, 2 * p + 1) - 1.0)
    inside = (mask.reshape(-1) == 0)
    vx = np.where(inside, vx, 0.0).reshape(n, n)
    vy = np.where(inside, vy, 0.0).reshape(n, n)
    return vx, vy


# Synthetic workloads with the paper's shapes.  Box lengths and radii follow the paper's
# regimes (single vortex near R = 5.2, oscillating pair near R = 5.4, turbulence for R >= 8).
def perturbation_directions(n: int, k: int, seed: int) -> np.ndarray:
    """k seeded random perturbation directions of a state, as (k, D) doubles in the stored
    half-spectrum layout (columns mx = 0..n/4, entries my = 0..n/4 then -n/4..-1, interleaved
    re/im) followed by the two mean-flow components: uniform in [-1, 1) on the modes
    0 < mx^2 + my^2 <= (n/4)^2, zero elsewhere, the mx = 0 column Hermitian (the my < 0
    entries are the conjugates of the my > 0 ones, my = 0 is real) like a state's."""
    M = n // 4
    NK = 2 * M + 1
    D = 2 * (M + 1) * NK + 2
    u = 2.0 * uniform01(seed, np.arange(k * D, dtype=np.uint64)).reshape(k, D) - 1.0
    spec = u[:, :-2].reshape(k, M + 1, NK, 2)
    my = np.array([j if j <= M else j - NK for j in range(NK)])
    mx = np.arange(M + 1)
    m2 = mx[:, None] ** 2 + my[None, :] ** 2
    spec[:, (m2 == 0) | (m2 > M * M), :] = 0.0
    spec[:, 0, 0, 1] = 0.0
    for j in range(1, M + 1):
        spec[:, 0, NK - j, 0] = spec[:, 0, j, 0]
        spec[:, 0, NK - j, 1] = -spec[:, 0, j, 1]
    return np.concatenate([spec.reshape(k, -1), u[:, -2:]], axis=1)


WORKLOADS = {
    "circle64_fp64": dict(n=64, dx=0.25, radius=5.2, seed=1, steps=2000),
    "circle512": dict(n=512, dx=0.04, radius=5.4, seed=2, steps=20000),
    "circle2048_turbulent": dict(n=2048, dx=0.02, radius=12.0, seed=4, steps=10000),
    "circle4096_turbulent": dict(n=4096, dx=0.01, radius=12.0, seed=4, steps=1000),
    "circle8192_paper_grid": dict(n=8192, dx=0.005, radius=12.0, seed=4, steps=100),
}


def sweep_domains():
    """The 48-domain sweep of the batched workload: 24 circles (12 radii across the
    stationary, oscillatory and chaotic regimes, each as a forward and a backward member of a
    hysteresis sweep) and 24 dumbbells (R in {2.8, pi, 3.5} x D/R in 8 steps from 1.0 to 1.9),
    on 128^2 to 512^2 grids.  Returns a list of dicts (name, n, dx, mask, seed)."""
    out = []
    circles = [(r, 128, 0.16) for r in (5.0, 5.1, 5.2, 5.25, 5.3, 5.35)] + \
              [(r, 256, 0.08) for r in (5.4, 5.6, 5.8, 6.4)] + [(r, 512, 0.08) for r in (7.2, 8.0)]
    i = 0
    for direction in ("forward", "backward"):
        for r, n, dx in circles:
            out.append(dict(name=f"circle R={r} ({direction})", n=n, dx=dx,
                            mask=circle_mask(n, dx, r), seed=100 + i))
            i += 1
    for r in (2.8, float(np.pi), 3.5):
        for ratio in np.linspace(1.0, 1.9, 8):
            out.append(dict(name=f"dumbbell R={r:.4f} D/R={ratio:.3f}", n=256, dx=0.08,
                            mask=dumbbell_mask(256, 0.08, r, ratio * r), seed=100 + i))
            i += 1
    return out
