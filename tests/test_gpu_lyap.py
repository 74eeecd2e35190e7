"""Lyapunov exponents on the GPU (ttsh_lyap_*) against the FP64 oracle.

Same inputs on both sides (state, seeded directions q0, eps, interval).  In double
precision the two sides run the same finite-difference perturbation scheme and the same QR
(positive diagonal, unique), so exponents, last-interval rates and directions agree to
rounding amplified by the differencing (1e-7 relative here).  The linear scheme's exponents
are known in closed form (see test_oracle_lyapunov.py) and are checked in both precisions.
"""
import numpy as np
import pytest

import ttsh_inputs as ti
from oracle import ttsh_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2304_03306_gb300 import build, ttsh
    build.build()
    ttsh.load_library()
    return ttsh


def half_state_vector(dom):
    w, v0 = dom.spectral_state()
    return np.concatenate([np.stack([w.real, w.imag], axis=-1).reshape(-1), v0])


@pytest.mark.parametrize("prec,tol", [(64, 1e-9), (32, 2e-4)])
def test_linear_exponents_closed_form(T, prec, tol):
    n = 16
    dx = 2 * np.pi / n
    dom = T.Domain(np.zeros((n, n), np.uint8), n, dx, precision=prec, b=0.0, lam=0.0, dt=0.1)
    q0 = ti.perturbation_directions(n, 6, 3)
    L = T.Lyapunov(dom, q0, 1e-3)
    L.step(300, 10)
    ex, last = L.result()
    np.testing.assert_allclose(last, [0.5] * 4 + [-0.5] * 2, atol=tol)
    assert dom.steps == 300
    L.close()


@pytest.mark.parametrize("n", [32, 64])
def test_nonlinear_exponents_match_oracle_fp64(T, n):
    dx = 16.0 / n
    mask = ti.circle_mask(n, dx, 5.0)
    vx, vy = ti.noise_velocity(mask, 21, 0.3)
    dom = T.Domain(mask, n, dx, precision=64)
    dom.set_velocity(vx, vy)
    dom.step(40)
    p = O.Params(n=n, dx=dx)
    K = O.process_mask(mask)
    s = O.run(O.project_velocity(vx, vy, p), K, p, 40)
    u = O.state_vector(s, p)
    np.testing.assert_allclose(half_state_vector(dom), u, rtol=0, atol=1e-12 * np.abs(u).max())
    q0 = ti.perturbation_directions(n, 4, 8)
    eps = 1e-6 * np.linalg.norm(u)
    L = T.Lyapunov(dom, q0, eps)
    L.step(100, 10)
    ex, last = L.result()
    q = L.directions()
    oex, olast, _, oq = O.lyapunov(s, K, p, q0, eps, 100, 10)
    np.testing.assert_allclose(ex, oex, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(last, olast, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(q, oq, atol=1e-7)
    L.close()


def test_rejects_bad_arguments(T):
    n = 16
    dom = T.Domain(np.zeros((n, n), np.uint8), n, 0.5, precision=32)
    D = 2 * (n // 4 + 1) * (n // 2 + 1) + 2
    with pytest.raises(T.TTSHError):
        T.Lyapunov(dom, np.zeros((17, D)), 1e-3)        # k > 16
    with pytest.raises(T.TTSHError):
        T.Lyapunov(dom, ti.perturbation_directions(n, 2, 0), 0.0)
    L = T.Lyapunov(dom, ti.perturbation_directions(n, 2, 0), 1e-3)
    with pytest.raises(T.TTSHError):
        L.result()                                      # no interval yet
    with pytest.raises(T.TTSHError):
        L.step(15, 10)                                  # not a multiple
    L.step(20, 10)
    with pytest.raises(T.TTSHError):
        L.step(20, 5)                                   # interval changed
    L.close()
