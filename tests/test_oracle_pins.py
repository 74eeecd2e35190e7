"""Pins of the FP64 oracle to what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than its own formulas: the DFT
definition summed by brute force, closed-form solutions of the linearised and
single-mode equations, exact index-permutation symmetries of the circular domain,
Parseval's identity and the limits of the order parameter.  Together they fail on a
dropped term, a wrong sign, a swapped kx/ky, a wrong cutoff or a wrong normalisation
anywhere in Algorithm 1 / Algorithm 2 as the oracle implements them.
"""
import json
import os

import numpy as np
import pytest

import ttsh_inputs as ti
from oracle import ttsh_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def coords(p):
    return ti.grid_coords(p.n, p.dx)


def stream_mode(p, m, amp, phase=0.3):
    """Real-space fields of psi = amp cos(k.x + phase): v = (d_y psi, -d_x psi),
    omega = -lap psi = k^2 psi, written analytically (no transform involved)."""
    X, Y = coords(p)
    dk = 2 * np.pi / (p.n * p.dx)
    kx, ky = dk * m[0], dk * m[1]
    th = kx * X + ky * Y + phase
    vx = -amp * ky * np.sin(th)
    vy = amp * kx * np.sin(th)
    w = amp * (kx * kx + ky * ky) * np.cos(th)
    return vx, vy, w, (kx, ky)


def state_from_real(vx, vy, w):
    return O.State(vx.copy(), vy.copy(), O.dft2(w))


def growth(p, k2):
    """Exact one-step factor of the linear operator a - (1 + lap)^2 on a Fourier mode."""
    return np.exp((p.a - (1.0 - k2) ** 2) * p.dt)


# --------------------------------------------------------------------------- DFT (P10)

def test_dft_matches_brute_force_definition():
    rng = np.random.default_rng(0)
    n = 8
    f = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    F = np.zeros((n, n), complex)
    for ky in range(n):
        for kx in range(n):
            acc = 0j
            for y in range(n):
                for x in range(n):
                    acc += f[y, x] * np.exp(-2j * np.pi * (kx * x + ky * y) / n)
            F[ky, kx] = acc / n
    np.testing.assert_allclose(O.dft2(f), F, atol=1e-13)
    np.testing.assert_allclose(O.dft2_naive(f), F, atol=1e-13)
    np.testing.assert_allclose(O.idft2(F), f, atol=1e-13)
    np.testing.assert_allclose(O.idft2_naive(F), f, atol=1e-13)


@pytest.mark.parametrize("n", [16, 32])
def test_fft_equals_naive_dft_and_parseval(n):
    rng = np.random.default_rng(n)
    f = rng.standard_normal((n, n))
    np.testing.assert_allclose(O.dft2(f), O.dft2_naive(f), atol=1e-12)
    assert abs(np.sum(np.abs(O.dft2(f)) ** 2) - np.sum(f * f)) < 1e-10 * np.sum(f * f)


def test_mirror_is_minus_k():
    n = 8
    MX, MY = O.index_grid(n)
    F = MX * 100 + MY
    Fm = O.mirror(F)
    for iy in range(n):
        for ix in range(n):
            assert Fm[iy, ix] == F[(-iy) % n, (-ix) % n]


# -------------------------------------------------------- stream function / curl (c1)

def test_projection_reproduces_analytic_vorticity_and_velocity():
    """psi = cos(k.x) with v = (d_y psi, -d_x psi), omega = k^2 psi (Appendix A relations):
    projecting the analytic v must give back the analytic omega and v (pins the +ik sign)."""
    p = O.Params(n=32, dx=0.5)
    for m in [(1, 0), (0, 2), (3, -2), (2, 5)]:
        vx, vy, w, _ = stream_mode(p, m, 0.7)
        s = O.project_velocity(vx, vy, p)
        np.testing.assert_allclose(O.vorticity(s), w, atol=1e-13)
        np.testing.assert_allclose(s.vx, vx, atol=1e-13)
        np.testing.assert_allclose(s.vy, vy, atol=1e-13)


# ------------------------------------------------------------ linear single mode (P1)

@pytest.mark.parametrize("m", [(1, 0), (0, 1), (2, 3), (-3, 3), (4, -1), (8, 0), (5, 6)])
def test_linear_single_mode_exact_growth(m):
    """b = lambda = 0, K = 0: each mode grows by exactly exp[(a - (1 - k^2)^2) dt] per step
    (the integrating factor of Appendix D integrates the linear operator exactly)."""
    p = O.Params(n=32, dx=0.25, b=0.0, lam=0.0)
    amp = 0.3
    vx, vy, w, (kx, ky) = stream_mode(p, m, amp)
    s = state_from_real(vx, vy, w)
    K = np.zeros((p.n, p.n))
    nsteps = 7
    s = O.run(s, K, p, nsteps)
    g = growth(p, kx * kx + ky * ky) ** nsteps
    assert (m[0] ** 2 + m[1] ** 2) <= (p.n // 4) ** 2
    np.testing.assert_allclose(O.vorticity(s), g * w, atol=1e-13 * max(1, np.abs(w).max()))
    np.testing.assert_allclose(s.vx, g * vx, atol=1e-13)
    np.testing.assert_allclose(s.vy, g * vy, atol=1e-13)


@pytest.mark.parametrize("m", [(8, 1), (6, 6), (9, 0), (12, 5)])
def test_modes_beyond_half_rule_are_removed(m):
    """|m|^2 > (N/4)^2 is zeroed by Algorithm 1 (the 1/2 rule); |m| = N/4 on the axis is kept
    (the previous test includes (8, 0) at N = 32)."""
    p = O.Params(n=32, dx=0.25, b=0.0, lam=0.0)
    assert m[0] ** 2 + m[1] ** 2 > (p.n // 4) ** 2
    vx, vy, w, _ = stream_mode(p, m, 0.3)
    s0 = state_from_real(vx, vy, w)
    s = O.step(s0, np.zeros((p.n, p.n)), p)
    n = p.n
    assert s.w_hat[m[1] % n, m[0] % n] == 0 and s.w_hat[-m[1] % n, -m[0] % n] == 0
    assert np.abs(s.w_hat).max() <= 1e-13 * np.abs(s0.w_hat).max()
    vmax = max(np.abs(vx).max(), np.abs(vy).max())
    assert np.abs(s.vx).max() < 1e-14 * vmax and np.abs(s.vy).max() < 1e-14 * vmax


# --------------------------------------------------------------- uniform mask (P2)

def test_uniform_mask_damping_closed_form():
    """K = c, b = lambda = 0: curl(K v) = c omega, so each mode is multiplied by
    exp(sigma dt) (1 - (gamma_v + gamma_w) c dt) per step; the mean flow by
    exp((a - 1) dt) (1 - gamma_v c dt) (Eq. avg)."""
    p = O.Params(n=32, dx=0.25, b=0.0, lam=0.0)
    c = 0.37
    m = (2, 1)
    vx, vy, w, (kx, ky) = stream_mode(p, m, 0.2)
    U, V = 0.013, -0.021
    s = state_from_real(vx + U, vy + V, w)
    K = np.full((p.n, p.n), c)
    nsteps = 5
    s = O.run(s, K, p, nsteps)
    g = (growth(p, kx * kx + ky * ky) * (1 - (p.gamma_v + p.gamma_w) * c * p.dt)) ** nsteps
    gm = (np.exp((p.a - 1) * p.dt) * (1 - p.gamma_v * c * p.dt)) ** nsteps
    np.testing.assert_allclose(O.vorticity(s), g * w, atol=1e-14)
    np.testing.assert_allclose(s.vx, g * vx + gm * U, atol=1e-14)
    np.testing.assert_allclose(s.vy, g * vy + gm * V, atol=1e-14)


def test_uniform_flow_cubic_mean_equation():
    """Uniform v = (U, V), K = 0: omega stays 0 and the mean follows Eq. (avg) with the
    Euler step: U' = exp((a-1) dt) (U - dt b (U^2 + V^2) U)."""
    p = O.Params(n=16, dx=0.5)
    U, V = 0.8, -0.35
    s = O.State(np.full((16, 16), U), np.full((16, 16), V), np.zeros((16, 16), complex))
    s = O.step(s, np.zeros((16, 16)), p)
    q = U * U + V * V
    g = np.exp((p.a - 1) * p.dt)
    np.testing.assert_allclose(s.vx, g * (U - p.dt * p.b * q * U), atol=1e-15)
    np.testing.assert_allclose(s.vy, g * (V - p.dt * p.b * q * V), atol=1e-15)
    assert np.abs(s.w_hat).max() == 0.0


# ---------------------------------------------------- cubic term, single mode (P3)

def _omega_mode_fields(p, m, n_harm, amp_w, phase):
    """omega = amp_w cos(n theta), theta = k.x + phase, and its stream-function velocity
    v = amp_w/(n k^2) sin(n theta) (-ky, kx), written analytically."""
    X, Y = coords(p)
    dk = 2 * np.pi / (p.n * p.dx)
    kx, ky = dk * m[0], dk * m[1]
    th = n_harm * (kx * X + ky * Y + phase)
    k2 = kx * kx + ky * ky
    w = amp_w * np.cos(th)
    vx = amp_w / (n_harm * k2) * np.sin(th) * (-ky)
    vy = amp_w / (n_harm * k2) * np.sin(th) * kx
    return vx, vy, w


@pytest.mark.parametrize("m,third_kept", [((1, 2), True), ((2, 1), True), ((2, 2), False)])
def test_cubic_term_single_mode_one_step(m, third_kept):
    """v = A e sin(theta), e = (-ky, kx)/|k|: v.grad(omega) = 0 and
    |v|^2 v = A^3 e (3/4 sin theta - 1/4 sin 3 theta), so curl(-b |v|^2 v) =
    -b A^3 |k| (3/4 cos theta - 3/4 cos 3 theta); one Euler step with the integrating factor
    has a closed form on the theta and 3 theta harmonics (3 theta removed if 3|m| > N/4)."""
    p = O.Params(n=32, dx=0.25, b=1.6, lam=9.0)
    phase = 0.4
    dk = 2 * np.pi / (p.n * p.dx)
    kabs = dk * np.hypot(*m)
    A = 0.9
    vx, vy, w = _omega_mode_fields(p, m, 1, A * kabs, phase)
    s = O.step(state_from_real(vx, vy, w), np.zeros((p.n, p.n)), p)
    c1 = growth(p, kabs ** 2) * (A * kabs - p.dt * p.b * A ** 3 * kabs * 0.75)
    c3 = growth(p, 9 * kabs ** 2) * (p.dt * p.b * A ** 3 * kabs * 0.75)
    assert (9 * (m[0] ** 2 + m[1] ** 2) <= (p.n // 4) ** 2) == third_kept
    if not third_kept:
        c3 = 0.0
    ex1 = _omega_mode_fields(p, m, 1, c1, phase)
    ex3 = _omega_mode_fields(p, m, 3, c3, phase)
    np.testing.assert_allclose(O.vorticity(s), ex1[2] + ex3[2], atol=1e-14)
    np.testing.assert_allclose(s.vx, ex1[0] + ex3[0], atol=1e-14)
    np.testing.assert_allclose(s.vy, ex1[1] + ex3[1], atol=1e-14)


# --------------------------------------------------------- advection, two modes (P3b)

def test_advection_two_perpendicular_modes_one_step():
    """omega = A cos(p x) + B cos(q y): v = (-B sin(q y)/q, A sin(p x)/p) and
    v.grad(omega) = A B (p/q - q/p) sin(p x) sin(q y); with b = 0 and K = 0 one step is
    E(p) A cos px + E(q) B cos qy - dt lambda A B (p/q - q/p)/2 E(k') [cos(px - qy) - cos(px + qy)],
    |k'|^2 = p^2 + q^2, E(k) = exp[(a - (1 - k^2)^2) dt]."""
    pr = O.Params(n=32, dx=0.25, b=0.0, lam=9.0)
    X, Y = coords(pr)
    dk = 2 * np.pi / (pr.n * pr.dx)
    p, q = 2 * dk, 3 * dk
    A, B = 0.5, -0.8
    w = A * np.cos(p * X) + B * np.cos(q * Y)
    vx = -B * np.sin(q * Y) / q
    vy = A * np.sin(p * X) / p
    s = O.step(O.State(vx, vy, O.dft2(w)), np.zeros((pr.n, pr.n)), pr)
    coef = -pr.dt * pr.lam * A * B * (p / q - q / p) / 2
    Ek = growth(pr, p * p + q * q)
    w_ex = (growth(pr, p * p) * A * np.cos(p * X) + growth(pr, q * q) * B * np.cos(q * Y)
            + coef * Ek * (np.cos(p * X - q * Y) - np.cos(p * X + q * Y)))
    np.testing.assert_allclose(O.vorticity(s), w_ex, atol=1e-14)


# -------------------------------------------------------------------- mask (P9)

def test_mask_lowpass_cutoff_and_square():
    """Algorithm 2: a raised cosine with |m| <= N/8 passes and is squared; a mode with
    |m| > N/8 is removed; the cutoff is inclusive at |m| = N/8 (reading c3)."""
    n = 64
    p = O.Params(n=n, dx=0.25)
    X, Y = coords(p)
    dk = 2 * np.pi / (n * p.dx)
    kept = 0.5 + 0.5 * np.cos(dk * (8 * X))                   # |m| = 8 = N/8: kept
    np.testing.assert_allclose(O.process_mask(kept), kept ** 2, atol=1e-14)
    diag = 0.5 + 0.5 * np.cos(dk * (5 * X + 6 * Y))           # |m|^2 = 61 <= 64: kept
    np.testing.assert_allclose(O.process_mask(diag), diag ** 2, atol=1e-14)
    cut = 0.5 + 0.5 * np.cos(dk * (8 * X + 1 * Y))            # |m|^2 = 65 > 64: removed
    np.testing.assert_allclose(O.process_mask(cut), 0.25 * np.ones((n, n)), atol=1e-14)
    np.testing.assert_allclose(O.process_mask(np.ones((n, n))), 1.0, atol=1e-14)


def test_circle_mask_properties():
    n = 128
    p = O.Params(n=n, dx=0.125)
    kn = ti.circle_mask(n, p.dx, 5.0)
    K = O.process_mask(kn)
    assert K.min() >= 0.0
    Kh = O.dft2(K)
    _, _, M2 = O.wavenumbers(p)
    assert np.abs(Kh[M2 > (n // 4) ** 2]).max() < 1e-13      # K^2 is band-limited to N/4
    X, Y = coords(p)
    r = np.hypot(X, Y)
    assert np.abs(K[r < 3.0] ).max() < 0.05                  # ~0 deep inside
    assert np.abs(K[r > 7.5] - 1).max() < 0.1                # ~1 deep in the wall
    assert K[n // 2, n // 2] == pytest.approx(K[n // 2, n // 2].real)


# ------------------------------------------------------- invariants (P4, P5, P6)

def _noise_state(n, dx, R, seed):
    p = O.Params(n=n, dx=dx)
    mask = ti.circle_mask(n, dx, R)
    vx, vy = ti.noise_velocity(mask, seed, 0.5)
    return p, O.process_mask(mask), O.project_velocity(vx, vy, p)


def test_invariants_after_steps():
    p, K, s = _noise_state(32, 0.5, 5.0, 7)
    s = O.run(s, K, p, 10)
    _, _, M2 = O.wavenumbers(p)
    KX, KY, _ = O.wavenumbers(p)
    assert s.w_hat[0, 0] == 0                                  # P5, exactly
    assert np.abs(s.w_hat[M2 > (p.n // 4) ** 2]).max() == 0    # dealiased exactly
    herm = np.abs(O.mirror(s.w_hat) - np.conj(s.w_hat)).max()
    assert herm <= 1e-15 * np.abs(s.w_hat).max()               # P6
    Vx, Vy = O.dft2(s.vx), O.dft2(s.vy)
    div = np.abs(KX * Vx + KY * Vy).max()
    scale = np.abs(np.hypot(KX, KY) * np.hypot(np.abs(Vx), np.abs(Vy))).max()
    assert div <= 1e-14 * scale                                 # P4
    curl = 1j * (KX * Vy - KY * Vx)
    assert np.abs(curl - s.w_hat).max() <= 1e-14 * np.abs(s.w_hat).max()


def test_projection_is_idempotent():
    p, K, s = _noise_state(32, 0.5, 5.0, 3)
    s2 = O.project_velocity(s.vx, s.vy, p)
    np.testing.assert_allclose(s2.w_hat, s.w_hat, atol=1e-15)
    np.testing.assert_allclose(s2.vx, s.vx, atol=1e-16)


# ---------------------------------------------------------- D4 symmetry (P7)

def _rot90(vx, vy, w):
    """Rotation by +90 degrees about the grid point (N/2, N/2): v'(x) = R v(R^-1 x)."""
    n = vx.shape[0]
    iy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    src_y = (n - ix) % n        # y-coordinate of R^-1 x is -x
    src_x = iy                  # x-coordinate of R^-1 x is  y
    return -vy[src_y, src_x], vx[src_y, src_x], w[src_y, src_x]


def _reflect_x(vx, vy, w):
    n = vx.shape[0]
    src_x = (n - np.arange(n)) % n
    return -vx[:, src_x], vy[:, src_x], -w[:, src_x]


@pytest.mark.parametrize("transform", [_rot90, _reflect_x])
def test_d4_symmetry_of_circle_trajectory(transform):
    p, K, s = _noise_state(32, 0.5, 5.0, 11)
    w0 = O.vorticity(s)
    tvx, tvy, _ = transform(s.vx, s.vy, w0)
    st = O.project_velocity(tvx, tvy, p)
    a = O.run(s, K, p, 30)
    b = O.run(st, K, p, 30)
    ex = transform(a.vx, a.vy, O.vorticity(a))
    scale = np.abs(a.vx).max()
    assert np.abs(b.vx - ex[0]).max() <= 1e-12 * scale
    assert np.abs(b.vy - ex[1]).max() <= 1e-12 * scale
    assert np.abs(O.vorticity(b) - ex[2]).max() <= 1e-12 * np.abs(ex[2]).max()


def test_fft_and_naive_dft_give_the_same_step():
    p, K, s = _noise_state(16, 1.0, 5.0, 5)
    a = O.run(s, K, p, 3)
    b = O.run(s, K, p, 3, dft=O.dft2_naive, idft=O.idft2_naive)
    np.testing.assert_allclose(a.w_hat, b.w_hat, atol=1e-14)
    np.testing.assert_allclose(a.vx, b.vx, atol=1e-15)


# -------------------------------------------------------------- diagnostics

def test_energy_enstrophy_single_mode():
    p = O.Params(n=32, dx=0.25)
    m, A = (2, 3), 0.6
    dk = 2 * np.pi / (p.n * p.dx)
    kabs = dk * np.hypot(*m)
    vx, vy, w = _omega_mode_fields(p, m, 1, A * kabs, 0.1)
    d = O.diagnostics(O.State(vx, vy, O.dft2(w)), p, nbins=p.n // 4 + 1)
    assert d["energy"] == pytest.approx(A * A / 4, rel=1e-13)
    assert d["enstrophy"] == pytest.approx(A * A * kabs ** 2 / 4, rel=1e-13)
    spec = d["spectrum"]
    assert spec.sum() == pytest.approx(d["energy"], rel=1e-13)         # P11 Parseval
    assert spec[int(round(np.hypot(*m)))] == pytest.approx(d["energy"], rel=1e-13)


def test_spectrum_parseval_random_state():
    p, K, s = _noise_state(64, 0.25, 5.0, 9)
    s = O.run(s, K, p, 5)
    d = O.diagnostics(s, p, nbins=p.n // 4 + 1)
    assert d["spectrum"].sum() == pytest.approx(d["energy"], rel=1e-13)


def test_vortex_order_parameter_limits():
    p = O.Params(n=64, dx=0.25)
    X, Y = coords(p)
    r = np.hypot(X, Y)
    f = np.exp(-r * r)
    psi_az = O.vortex_order_parameter(-Y * f, X * f, p)
    assert psi_az == pytest.approx(1.0, abs=1e-14)
    psi_rad = O.vortex_order_parameter(X * f, Y * f, p)
    assert psi_rad == pytest.approx(-(2 / np.pi) / (1 - 2 / np.pi), abs=1e-14)


def test_vortex_order_parameter_about_an_off_grid_centre():
    """Solid-body rotation about a centre that is no grid point: v = (-(y - y0), x - x0) is
    purely azimuthal about (x0, y0), so |e_theta . v| = |v| at every point and Psi = 1
    exactly.  Measured about the box origin instead, or with the centre offset taken with the
    wrong sign on either axis, the same field has a radial part and Psi drops well below 1."""
    p = O.Params(n=64, dx=0.25)
    X, Y = coords(p)
    x0, y0 = 0.37, -0.61                    # between grid points on both axes
    vx, vy = -(Y - y0), X - x0
    assert O.vortex_order_parameter(vx, vy, p, center=(x0, y0)) == pytest.approx(1.0, abs=1e-13)
    for wrong in [(0.0, 0.0), (-x0, y0), (x0, -y0), (y0, x0)]:
        assert O.vortex_order_parameter(vx, vy, p, center=wrong) < 0.99


def test_vortex_order_parameter_at_the_centre_point():
    """Reading c12: at the centre itself e_theta := 0, so a velocity there adds |v| to the
    denominator only.  Field zero everywhere except v = (0.3, -0.4) at the grid point that is
    the centre: sum|e_theta . v| = 0, sum|v| = 0.5, Psi = (0 - 2/pi) / (1 - 2/pi).  Adding a
    unit azimuthal velocity at one other point gives ratio 1/1.5.  The centre is a grid point
    away from the box origin, so its index must come from the offset with the right sign."""
    p = O.Params(n=32, dx=0.5)
    i0, j0 = 11, 23                         # row (y) and column (x) of the centre point
    c = (np.arange(p.n) - p.n // 2) * p.dx
    centre = (c[j0], c[i0])
    vx = np.zeros((p.n, p.n))
    vy = np.zeros((p.n, p.n))
    vx[i0, j0], vy[i0, j0] = 0.3, -0.4
    two_pi = 2 / np.pi
    assert O.vortex_order_parameter(vx, vy, p, center=centre) == pytest.approx(
        (0.0 - two_pi) / (1 - two_pi), abs=1e-14)
    # one more point, 3 cells to the right of the centre (+x): e_theta there is (0, 1)
    vy[i0, j0 + 3] = 1.0
    assert O.vortex_order_parameter(vx, vy, p, center=centre) == pytest.approx(
        (1.0 / 1.5 - two_pi) / (1 - two_pi), abs=1e-14)
    # the same field about a centre one cell off: the centre point's velocity now counts
    # in the numerator (its e_theta is a unit vector), so Psi differs
    off = (c[j0 + 1], c[i0])
    assert abs(O.vortex_order_parameter(vx, vy, p, center=off) -
               (1.0 / 1.5 - two_pi) / (1 - two_pi)) > 1e-3


# ------------------------------------------------------------ inputs / constants

def test_table1_constants_match_golden():
    g = json.load(open(os.path.join(GOLDEN, "table1_params.json")))
    p = O.Params(n=g["n"], dx=g["dx"])
    assert (p.a, p.b, p.lam, p.gamma_v, p.gamma_w, p.dt) == (
        g["a"], g["b"], g["lambda"], g["gamma_v"], g["gamma_w"], g["dt"])
    t = ti.TABLE1
    assert (t["a"], t["b"], t["lam"], t["gamma_v"], t["gamma_w"], t["dt"]) == (
        g["a"], g["b"], g["lambda"], g["gamma_v"], g["gamma_w"], g["dt"])


def test_splitmix64_published_vectors():
    # First outputs of SplitMix64 seeded with 1234567 (reference implementation by Vigna).
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    assert [int(v) for v in ti.splitmix64(1234567, np.arange(5))] == ref


def test_noise_only_inside_mask():
    mask = ti.circle_mask(64, 0.25, 5.0)
    vx, vy = ti.noise_velocity(mask, 1, 0.01)
    assert np.all(vx[mask == 1] == 0) and np.all(vy[mask == 1] == 0)
    assert np.abs(vx).max() <= 0.01 and np.abs(vx[mask == 0]).min() >= 0
    assert abs(vx[mask == 0].mean()) < 0.002


# ---------------------------------------------------------- PSD and Psi_2 (Sec. III.B, IV.B)

def test_temporal_psd_of_a_single_frequency():
    """omega = f(x) cos(W0 t + phi) sampled at t_j = j dt, j < T, with W0 T dt a multiple of pi:
    sum_t omega e^{-i W0 t} = (T/2) e^{i phi} f, so S(W0) = (T/2)^2 N^-2 sum f^2, while a
    frequency on the same grid away from +-W0 gives 0."""
    n, T, dt = 16, 40, 0.25
    rng = np.random.default_rng(4)
    f = rng.standard_normal((n, n))
    W0 = 2 * np.pi * 3 / (T * dt)
    times = np.arange(T) * dt
    fields = [f * np.cos(W0 * t + 0.7) for t in times]
    S = O.temporal_psd(fields, times, [W0, 2 * np.pi * 5 / (T * dt)])
    assert S[0] == pytest.approx((T / 2) ** 2 * np.sum(f * f) / (n * n), rel=1e-12)
    assert abs(S[1]) <= 1e-20 * S[0] + 1e-22


def _two_peaks(p, centres, amps, width=0.6):
    X, Y = coords(p)
    w = np.zeros((p.n, p.n))
    for (cx, cy), a in zip(centres, amps):
        w += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / width ** 2)
    return w


@pytest.mark.parametrize("amps,expect", [((1.0, 1.0), 1.0), ((1.0, -1.0), 0.0), ((2.0, -0.5), 0.6),
                                         ((-0.3, -0.9), 1.0)])
def test_dumbbell_order_parameter_closed_forms(amps, expect):
    p = O.Params(n=64, dx=0.25)
    centres = [(-2.0, 0.0), (2.0, 0.0)]          # grid points: x = (i - 32) * 0.25
    w = _two_peaks(p, centres, amps)
    psi2, a, b = O.dumbbell_order_parameter(w, p, centres, 1.5)
    assert psi2 == pytest.approx(expect, abs=1e-12)
    assert a == pytest.approx(amps[0], rel=1e-12) and b == pytest.approx(amps[1], rel=1e-12)


def test_dumbbell_region_is_closed_and_excludes_outside_peaks():
    p = O.Params(n=64, dx=0.25)
    w = np.zeros((64, 64))
    w[32, 32 - 8] = 0.5          # (-2, 0): left centre
    w[32, 32 + 8] = -0.5         # (+2, 0): right centre
    w[32, 32 - 14] = 5.0         # (-3.5, 0): exactly 1.5 from the left centre -> inside
    w[32, 32 + 15] = 9.0         # (+3.75, 0): 1.75 from the right centre -> outside
    psi2, a, b = O.dumbbell_order_parameter(w, p, [(-2.0, 0.0), (2.0, 0.0)], 1.5)
    assert (a, b) == (5.0, -0.5)
    assert psi2 == pytest.approx(4.5 / 5.5, abs=1e-15)


def test_threaded_transforms_equal_the_default_ones():
    """The all-core transform pair used for large-grid tests is the same unitary DFT."""
    rng = np.random.default_rng(4)
    f = rng.standard_normal((64, 64))
    dft, idft = O.threaded_dft(2)
    np.testing.assert_allclose(dft(f), O.dft2(f), atol=1e-13)
    np.testing.assert_allclose(idft(O.dft2(f)), f, atol=1e-13)
    p = O.Params(n=32, dx=0.5)
    mask = ti.circle_mask(32, 0.5, 5.2)
    s = O.project_velocity(*ti.noise_velocity(mask, 3, 0.3), p)
    K = O.process_mask(mask)
    a = O.step(s, K, p)
    b = O.step(s, K, p, dft=dft, idft=idft)
    np.testing.assert_allclose(O.vorticity(b), O.vorticity(a), atol=1e-14)
