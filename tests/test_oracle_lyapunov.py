"""Pins of the oracle's Lyapunov analysis (Sec. III.C) against closed forms.

With b = lambda = 0 the scheme of Algorithm 1 is linear and diagonal in Fourier space: a
vorticity mode m != 0 inside the 1/2-rule disc is multiplied each step by
exp[(a - (1 - k^2)^2) dt] (1 - (gamma_v + gamma_w) K dt) for a uniform mask K, and the mean
flow by exp[(a - 1) dt] (1 - gamma_v K dt).  Its Lyapunov exponents are the logs of these
factors over dt, each with the real dimension of its eigenspace (a Hermitian pair of modes
counts 2, the mean flow 2).  Once the directions have converged, the per-interval rates equal
them exactly; the running averages approach them as 1/T.
"""
import numpy as np
import pytest

import ttsh_inputs as ti
from oracle import ttsh_oracle as O


def zero_state(p):
    n = p.n
    return O.project_velocity(np.zeros((n, n)), np.zeros((n, n)), p)


def test_linear_exponents_without_mask():
    # L = 2 pi: dk = 1, so |m| = 1 has k = 1 (sigma = a = 0.5, 4 real dimensions); |m|^2 = 2
    # has sigma = a - 1 = -0.5 (4 dimensions), the same rate as the mean flow (2 dimensions)
    n = 16
    p = O.Params(n=n, dx=2 * np.pi / n, b=0.0, lam=0.0, dt=0.1)
    K = np.zeros((n, n))
    q0 = ti.perturbation_directions(n, 6, 3)
    ex, last, s, Q = O.lyapunov(zero_state(p), K, p, q0, 1e-3, 300, 10)
    expect = np.array([0.5] * 4 + [-0.5] * 2)
    np.testing.assert_allclose(last, expect, atol=1e-9)
    np.testing.assert_allclose(ex, expect, atol=0.15)   # running average: transient / T
    assert np.all(s.w_hat == 0)


def test_linear_exponents_with_uniform_mask():
    n = 16
    p = O.Params(n=n, dx=2 * np.pi / n, b=0.0, lam=0.0, dt=0.01)
    K = O.process_mask(np.ones((n, n), np.uint8))
    assert np.allclose(K, 1.0, atol=1e-12)
    q0 = ti.perturbation_directions(n, 4, 4)
    ex, last, _, _ = O.lyapunov(zero_state(p), K, p, q0, 1e-3, 1500, 10)
    mean = (p.a - 1.0) + np.log(1.0 - p.gamma_v * p.dt) / p.dt
    top = p.a + np.log(1.0 - (p.gamma_v + p.gamma_w) * p.dt) / p.dt
    np.testing.assert_allclose(last, [mean, mean, top, top], rtol=1e-9)


def test_directions_are_orthonormal_in_real_space():
    # the weighted inner product is Parseval's: sum_x omega omega' + v^(0).v'^(0)
    n = 16
    p = O.Params(n=n, dx=0.5)
    mask = ti.circle_mask(n, p.dx, 3.0)
    K = O.process_mask(mask)
    vx, vy = ti.noise_velocity(mask, 2, 0.3)
    s = O.project_velocity(vx, vy, p)
    _, _, _, Q = O.lyapunov(s, K, p, ti.perturbation_directions(n, 3, 1), 1e-6, 20, 10)
    fields = []
    for q in Q:
        st = O.vector_state(q, p)
        v0 = np.array([np.real(O.dft2(st.vx)[0, 0]), np.real(O.dft2(st.vy)[0, 0])])
        fields.append((O.vorticity(st), v0))
    G = np.array([[np.sum(a[0] * b[0]) + a[1] @ b[1] for b in fields] for a in fields])
    np.testing.assert_allclose(G, np.eye(3), atol=1e-12)


def test_state_vector_round_trip():
    n = 16
    p = O.Params(n=n, dx=0.5)
    mask = ti.circle_mask(n, p.dx, 3.0)
    vx, vy = ti.noise_velocity(mask, 5, 0.3)
    s = O.project_velocity(vx, vy, p)
    t = O.vector_state(O.state_vector(s, p), p)
    assert np.max(np.abs(t.w_hat - s.w_hat)) <= 1e-15
    assert np.max(np.abs(t.vx - s.vx)) <= 1e-15 and np.max(np.abs(t.vy - s.vy)) <= 1e-15


def test_nonlinear_exponents_do_not_depend_on_eps():
    n = 16
    p = O.Params(n=n, dx=0.5)
    mask = ti.circle_mask(n, p.dx, 3.0)
    K = O.process_mask(mask)
    vx, vy = ti.noise_velocity(mask, 7, 0.3)
    s = O.run(O.project_velocity(vx, vy, p), K, p, 50)
    q0 = ti.perturbation_directions(n, 2, 9)
    a, _, _, _ = O.lyapunov(s, K, p, q0, 1e-5, 100, 10)
    b, _, _, _ = O.lyapunov(s, K, p, q0, 1e-6, 100, 10)
    np.testing.assert_allclose(a, b, rtol=1e-3, atol=1e-3)


def test_interval_must_divide_steps():
    n = 16
    p = O.Params(n=n, dx=0.5)
    with pytest.raises(ValueError):
        O.lyapunov(zero_state(p), np.zeros((n, n)), p, ti.perturbation_directions(n, 1, 0), 1e-3, 15, 10)
