"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative L2 over the whole field unless stated):
  FP64 domains: 1e-12 after up to 100 steps (rounding-order differences only);
  FP32 domains: 1e-5 after 100 steps (FP32 unit round-off 6e-8 times the transform depth
  and the number of steps, well inside the bound).
Exact checks: omega^(0) = 0, modes outside the 1/2-rule disc are 0, the stored mx = 0
column is Hermitian, checkpoint/resume and graph replay are bit-identical.
"""
import numpy as np
import pytest

import ttsh_inputs as ti
from oracle import ttsh_oracle as O

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}


@pytest.fixture(scope="module")
def T():
    from paper_2304_03306_gb300 import build, ttsh
    build.build()
    ttsh.load_library()
    return ttsh


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def half_layout(w_hat):
    """Oracle full FFT-ordered spectrum [ky][kx] -> the library's [mx][j] half layout."""
    n = w_hat.shape[0]
    M = n // 4
    NK = 2 * M + 1
    ky = np.array([j if j <= M else j - NK for j in range(NK)])
    return w_hat[np.ix_(ky % n, np.arange(M + 1))].T


def setup(T, n, dx, radius, prec, seed, amp=0.01, mask=None):
    if mask is None:
        mask = ti.circle_mask(n, dx, radius)
    p = O.Params(n=n, dx=dx)
    dom = T.Domain(mask, n, dx, precision=prec)
    vx, vy = ti.noise_velocity(mask, seed, amp)
    dom.set_velocity(vx, vy)
    K = O.process_mask(mask)
    s = O.project_velocity(vx, vy, p)
    return dom, p, K, s


def check_fields(dom, s, tol):
    vx, vy, w = dom.fields()
    assert rel(w, O.vorticity(s)) <= tol
    assert rel(np.stack([vx, vy]), np.stack([s.vx, s.vy])) <= tol


# ------------------------------------------------------------------- Algorithm 2

@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("n,dx,shape", [(16, 1.0, "circle"), (64, 0.25, "circle"),
                                        (256, 0.08, "dumbbell"), (512, 0.04, "circle")])
def test_mask_matches_oracle(T, prec, n, dx, shape):
    R = 5.2 if shape == "circle" else 3.0
    mask = ti.circle_mask(n, dx, R) if shape == "circle" else ti.dumbbell_mask(n, dx, R, 1.5 * R)
    dom = T.Domain(mask, n, dx, precision=prec)
    K = dom.mask()
    Ko = O.process_mask(mask)
    assert np.abs(K - Ko).max() <= (1e-13 if prec == 64 else 2e-6)
    assert K.min() >= 0.0


# --------------------------------------------------------- initial-state projection

@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("n,dx", [(16, 1.0), (32, 0.5), (128, 0.125)])
def test_projection_matches_oracle(T, prec, n, dx):
    dom, p, K, s = setup(T, n, dx, 5.0, prec, 3, amp=0.5)
    check_fields(dom, s, TOL[prec] / 10)
    w_hat, v0 = dom.spectral_state()
    ref = half_layout(s.w_hat)
    assert rel(w_hat, ref) <= TOL[prec] / 10
    np.testing.assert_allclose(v0, [np.sum(s.vx) / n, np.sum(s.vy) / n], rtol=TOL[prec],
                               atol=1e-15 * n)


# ---------------------------------------------------------------- Algorithm 1 parity

@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("n,dx,R,steps", [(16, 1.0, 5.0, 100), (32, 0.5, 5.2, 100),
                                          (64, 0.25, 5.2, 100), (128, 0.16, 5.3, 100),
                                          (256, 0.08, 5.6, 100)])
def test_steps_match_oracle(T, prec, n, dx, R, steps):
    dom, p, K, s = setup(T, n, dx, R, prec, 1, amp=0.3)
    dom.step(steps)
    s = O.run(s, K, p, steps)
    check_fields(dom, s, TOL[prec])
    w_hat, v0 = dom.spectral_state()
    assert rel(w_hat, half_layout(s.w_hat)) <= TOL[prec]


@pytest.mark.parametrize("prec", [32, 64])
def test_bench_workload_512(T, prec):
    """The timed workload's configuration (512^2 circle, dx = 0.04, R = 5.4, noise 0.01,
    seed 2) over 100 steps, with the step loop replayed as a CUDA graph."""
    w = ti.WORKLOADS["circle512"]
    dom, p, K, s = setup(T, w["n"], w["dx"], w["radius"], prec, w["seed"], amp=0.01)
    dom.step(100)
    s = O.run(s, K, p, 100)
    check_fields(dom, s, TOL[prec])


def test_fp64_workload_64_over_2000_steps(T):
    """The 64^2 FP64 configuration (circle R = 5.2, dx = 0.25, noise 0.01, seed 1) over its
    full 2000 steps against the oracle."""
    w = ti.WORKLOADS["circle64_fp64"]
    dom, p, K, s = setup(T, w["n"], w["dx"], w["radius"], 64, w["seed"], amp=0.01)
    dom.step(2000)
    s = O.run(s, K, p, 2000)
    check_fields(dom, s, 1e-12)
    w_hat, _ = dom.spectral_state()
    assert rel(w_hat, half_layout(s.w_hat)) <= 1e-12


def test_fp64_workload_64_reaches_the_stationary_vortex(T):
    """Long run of the same configuration: a single stationary vortex (P8) - the state stops
    changing, the velocity is nearly azimuthal (Psi > 0.8) and |omega| peaks at the centre."""
    w = ti.WORKLOADS["circle64_fp64"]
    n, dx = w["n"], w["dx"]
    dom, p, K, s = setup(T, n, dx, w["radius"], 64, w["seed"], amp=0.01)
    dom.step(30000)
    w0, _ = dom.spectral_state()
    dom.step(1)
    w1, _ = dom.spectral_state()
    assert np.linalg.norm(w1 - w0) / np.linalg.norm(w1) < 1e-9
    d = dom.diagnostics()
    assert d["psi"] > 0.8
    _, _, om = dom.fields()
    X, Y = ti.grid_coords(n, dx)
    iy, ix = np.unravel_index(np.argmax(np.abs(om)), om.shape)
    assert np.hypot(X[iy, ix], Y[iy, ix]) <= 2 * dx


def test_fp32_and_fp64_series_agree_on_the_512_workload(T):
    """The 512^2 configuration's energy and order-parameter series in both precisions (before
    any chaotic amplification the FP32 run tracks the FP64 one)."""
    w = ti.WORKLOADS["circle512"]
    series = {}
    for prec in (32, 64):
        dom, _, _, _ = setup(T, w["n"], w["dx"], w["radius"], prec, w["seed"], amp=0.01)
        series[prec] = dom.record(2000, 10)
    a, b = series[32], series[64]
    assert np.array_equal(a[:, 0], b[:, 0])
    assert rel(a[:, 1], b[:, 1]) <= 1e-4 and rel(a[:, 3], b[:, 3]) <= 1e-4


@pytest.mark.parametrize("prec", [32, 64])
def test_2048_few_steps(T, prec):
    w = ti.WORKLOADS["circle2048_turbulent"]
    dom, p, K, s = setup(T, w["n"], w["dx"], w["radius"], prec, w["seed"], amp=0.3)
    dom.step(3)
    s = O.run(s, K, p, 3)
    check_fields(dom, s, TOL[prec])


def threaded_oracle_run(s, K, p, steps):
    """The oracle with its transforms on all host cores (the same unitary DFT pair)."""
    dft, idft = O.threaded_dft()
    return O.run(s, K, p, steps, dft=dft, idft=idft)


_LARGE_REF = {}


def large_reference(n, dx, R, seed, steps):
    """Oracle state after `steps` steps from the seeded noise (amplitude 0.3), cached per case."""
    key = (n, dx, R, seed, steps)
    if key not in _LARGE_REF:
        mask = ti.circle_mask(n, dx, R)
        p = O.Params(n=n, dx=dx)
        vx, vy = ti.noise_velocity(mask, seed, 0.3)
        dft, idft = O.threaded_dft()
        K = O.process_mask(mask, dft=dft, idft=idft)
        s = O.project_velocity(vx, vy, p, dft=dft, idft=idft)
        _LARGE_REF.clear()
        _LARGE_REF[key] = (mask, vx, vy, threaded_oracle_run(s, K, p, steps))
    return _LARGE_REF[key]


@pytest.mark.parametrize("prec,n,dx,steps", [(32, 4096, 0.01, 2), (64, 4096, 0.01, 2), (32, 8192, 0.005, 1)])
def test_dense_turbulent_state_at_full_size(T, prec, n, dx, steps):
    """A dense noise state (amplitude 0.3) of the turbulent circle, R = 12, on the 4096^2 grid
    and the paper's 8192^2 grid, with the default (autotuner's first) row and column plans
    of those sizes - at 8192^2 the clustered row pass and the column pass that holds two of
    its three fields at a time - against the oracle element by element."""
    mask, vx, vy, ref = large_reference(n, dx, 12.0, 4, steps)
    dom = T.Domain(mask, n, dx, precision=prec)
    dom.set_velocity(vx, vy)
    dom.step(steps)
    gvx, gvy, gw = dom.fields()
    dom.close()
    assert rel(gw, O.vorticity(ref)) <= TOL[prec]
    assert rel(np.stack([gvx, gvy]), np.stack([ref.vx, ref.vy])) <= TOL[prec]


# --------------------------------------------------------- device initial state

@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("n,dx,shape,seed", [(64, 0.25, "circle", 1), (256, 0.08, "dumbbell", 7),
                                             (512, 0.04, "circle", 2**64 - 12345)])
def test_init_noise_equals_the_host_generator_bit_for_bit(T, prec, n, dx, shape, seed):
    """ttsh_init_noise draws the random initial state on the device; projected, it gives the
    same state bits as the host generator's field passed through ttsh_set_velocity (the
    counter-based SplitMix64 definition, including a seed above 2^63)."""
    mask = ti.circle_mask(n, dx, 5.4) if shape == "circle" else ti.dumbbell_mask(n, dx, 3.0, 4.5)
    a = T.Domain(mask, n, dx, precision=prec)
    a.init_noise(seed, 0.01)
    b = T.Domain(mask, n, dx, precision=prec)
    b.set_velocity(*ti.noise_velocity(mask, seed, 0.01))
    wa, va = a.spectral_state()
    wb, vb = b.spectral_state()
    assert np.array_equal(wa, wb) and np.array_equal(va, vb)
    assert np.abs(wa).max() > 0
    assert a.steps == 0
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_init_noise_then_100_steps_match_oracle(T, prec):
    """The timed workload's initial state made on the device, then 100 steps, against the
    oracle started from the host generator's field."""
    w = ti.WORKLOADS["circle512"]
    n, dx = w["n"], w["dx"]
    mask = ti.circle_mask(n, dx, w["radius"])
    dom = T.Domain(mask, n, dx, precision=prec)
    dom.init_noise(w["seed"], 0.01)
    dom.step(100)
    p = O.Params(n=n, dx=dx)
    s = O.run(O.project_velocity(*ti.noise_velocity(mask, w["seed"], 0.01), p), O.process_mask(mask), p, 100)
    check_fields(dom, s, TOL[prec])
    dom.close()


# --------------------------------------------------------- closed forms at any size

@pytest.mark.parametrize("prec,n", [(32, 16), (32, 8192), (64, 16), (64, 4096), (32, 1024)])
def test_linear_single_mode_closed_form(T, prec, n):
    """b = lambda = 0, K = 0: a mode grows by exp[(a - (1 - k^2)^2) dt] per step exactly."""
    dx = 16.0 / n
    mask = np.zeros((n, n), np.uint8)
    dom = T.Domain(mask, n, dx, precision=prec, b=0.0, lam=0.0)
    X, Y = ti.grid_coords(n, dx)
    dk = 2 * np.pi / (n * dx)
    m = (2, 3)
    kx, ky = dk * m[0], dk * m[1]
    th = kx * X + ky * Y + 0.3
    A = 0.4
    vx, vy = -A * ky * np.sin(th), A * kx * np.sin(th)
    w0 = A * (kx * kx + ky * ky) * np.cos(th)
    dom.set_velocity(vx, vy)
    steps = 150
    dom.step(steps)
    g = np.exp((0.5 - (1 - kx * kx - ky * ky) ** 2) * 0.01) ** steps
    gvx, gvy, gw = dom.fields()
    tol = 1e-12 if prec == 64 else 2e-5
    assert rel(gw, g * w0) <= tol
    assert rel(np.stack([gvx, gvy]), g * np.stack([vx, vy])) <= tol


def _mode_fields(terms, X, Y):
    """omega = sum a cos(kx x + ky y + ph) and its stream-function velocity
    v = sum a / k^2 sin(kx x + ky y + ph) (-ky, kx), written analytically."""
    w = np.zeros_like(X)
    vx = np.zeros_like(X)
    vy = np.zeros_like(X)
    for a, kx, ky, ph in terms:
        th = kx * X + ky * Y + ph
        k2 = kx * kx + ky * ky
        w += a * np.cos(th)
        s = np.sin(th) * (a / k2)
        vx -= ky * s
        vy += kx * s
    return vx, vy, w


@pytest.mark.parametrize("n", [4096, 8192])
def test_nonlinear_closed_forms_every_row_variant_at_full_size(T, n):
    """One step of two closed forms with the nonlinear terms at work, at full grid sizes and
    for every row-pass variant (clustered ones included): (i) b = 0, K = 0, omega =
    A cos(px) + B cos(qy): the advection term makes the cos(px -+ qy) pair with amplitude
    -+ dt lambda A B (p/q - q/p)/2; (ii) a single mode v = A e sin(theta), e perpendicular to
    k: |v|^2 v = A^3 e (3/4 sin theta - 1/4 sin 3 theta), advection vanishes.  Every mode is
    then multiplied by E(k) = exp[(a - (1 - k^2)^2) dt]."""
    L = 16.0
    dx = L / n
    X, Y = ti.grid_coords(n, dx)
    dk = 2 * np.pi / L
    a_, dt, lam, b = 0.5, 0.01, 9.0, 1.6

    def E(k2):
        return np.exp((a_ - (1 - k2) ** 2) * dt)

    p, q = 2 * dk, 3 * dk
    A, B = 0.5, -0.8
    c = -dt * lam * A * B * (p / q - q / p) / 2
    adv0 = [(A, p, 0.0, 0.0), (B, 0.0, q, 0.0)]
    adv1 = [(E(p * p) * A, p, 0.0, 0.0), (E(q * q) * B, 0.0, q, 0.0),
            (c * E(p * p + q * q), p, -q, 0.0), (-c * E(p * p + q * q), p, q, 0.0)]
    kx, ky, ph, Am = dk * 1, dk * 2, 0.4, 0.9
    ka = np.hypot(kx, ky)
    cub0 = [(Am * ka, kx, ky, ph)]
    cub1 = [(E(ka * ka) * (Am * ka - dt * b * Am ** 3 * ka * 0.75), kx, ky, ph),
            (E(9 * ka * ka) * (dt * b * Am ** 3 * ka * 0.75), 3 * kx, 3 * ky, 3 * ph)]
    mask = np.zeros((n, n), np.uint8)
    for bb, t0, t1 in ((0.0, adv0, adv1), (b, cub0, cub1)):
        dom = T.Domain(mask, n, dx, precision=32, b=bb, lam=lam)
        vx, vy, _ = _mode_fields(t0, X, Y)
        dom.set_velocity(vx, vy)
        w0, v00 = dom.spectral_state()
        ex = _mode_fields(t1, X, Y)
        plan = dom.plan()
        for rv in range(plan["n_row_variants"]):
            dom.set_plan(rv, 0, launch_mode=0)
            dom.set_spectral_state(w0, v00)
            dom.step(1)
            gvx, gvy, gw = dom.fields()
            assert rel(gw, ex[2]) <= 2e-5, (rv, dom.plan())
            assert rel(np.stack([gvx, gvy]), np.stack(ex[:2])) <= 2e-5, (rv, dom.plan())
        dom.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_uniform_mask_closed_form(T, prec):
    """K_naive = 1 everywhere gives K = 1; with b = lambda = 0 each mode is multiplied by
    exp(sigma dt)(1 - (gamma_v + gamma_w) dt) and the mean flow by exp((a-1)dt)(1 - gamma_v dt)."""
    n, dx = 64, 0.25
    mask = np.ones((n, n), np.uint8)
    dom = T.Domain(mask, n, dx, precision=prec, b=0.0, lam=0.0)
    X, Y = ti.grid_coords(n, dx)
    dk = 2 * np.pi / (n * dx)
    kx, ky = dk * 1, dk * 2
    th = kx * X + ky * Y
    vx, vy = -0.2 * ky * np.sin(th) + 0.05, 0.2 * kx * np.sin(th) - 0.03
    dom.set_velocity(vx, vy)
    dom.step(5)
    g = (np.exp((0.5 - (1 - kx * kx - ky * ky) ** 2) * 0.01) * (1 - 44 * 0.01)) ** 5
    gm = (np.exp(-0.5 * 0.01) * (1 - 40 * 0.01)) ** 5
    gvx, gvy, _ = dom.fields()
    tol = 1e-12 if prec == 64 else 1e-5
    assert rel(gvx, g * (vx - 0.05) + gm * 0.05) <= tol
    assert rel(gvy, g * (vy + 0.03) - gm * 0.03) <= tol


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("prec", [64, 32])
def test_invariants_of_gpu_state(T, prec):
    n, dx = 128, 0.16
    dom, p, K, s = setup(T, n, dx, 5.3, prec, 5, amp=0.3)
    dom.step(40)
    w_hat, _ = dom.spectral_state()
    M = n // 4
    NK = 2 * M + 1
    assert w_hat[0, 0] == 0                                          # P5 exactly
    mx = np.arange(M + 1)[:, None]
    my = np.array([j if j <= M else j - NK for j in range(NK)])[None, :]
    assert np.all(w_hat[(mx * mx + my * my) > M * M] == 0)           # 1/2 rule exactly
    col0 = w_hat[0]
    assert np.all(col0[1:M + 1] == np.conj(col0[NK - 1:M:-1]))      # Hermitian exactly
    vx, vy, _ = dom.fields()
    KX, KY, _ = O.wavenumbers(p)
    Vx, Vy = np.fft.fft2(vx, norm="ortho"), np.fft.fft2(vy, norm="ortho")
    div = np.abs(KX * Vx + KY * Vy).max() / (np.abs(np.hypot(KX, KY)) * np.hypot(np.abs(Vx), np.abs(Vy))).max()
    assert div <= (1e-13 if prec == 64 else 1e-6)                   # P4


# ------------------------------------------------------------------ diagnostics

@pytest.mark.parametrize("prec", [64, 32])
def test_max_div_reports_incompressibility_and_leaves_stepping_unchanged(T, prec):
    """ttsh_diag.max_div: max |k.v^| / max |k||v^| of the real-space velocity (P4, div v = 0
    by the stream-function construction) is at round-off level; the float transforms always
    leave some.  Taking diagnostics between steps does not change the trajectory."""
    n, dx = 128, 0.16
    dom, p, K, s = setup(T, n, dx, 5.3, prec, 5, amp=0.3)
    ref, _, _, _ = setup(T, n, dx, 5.3, prec, 5, amp=0.3)
    dom.step(20)
    d = dom.diagnostics()
    assert 0.0 <= d["max_div"] <= (1e-13 if prec == 64 else 1e-6)
    if prec == 32:
        assert d["max_div"] > 0.0
    dom.step(20)
    ref.step(40)
    wa, va = dom.spectral_state()
    wb, vb = ref.spectral_state()
    assert np.array_equal(wa, wb) and np.array_equal(va, vb)


def test_fma_peak_probe(T):
    """The measured FMA throughputs the rooflines use are in the range GB300's unit counts
    allow (FP32: 152 SMs x 128 lanes x 2 flops x <= 2.07 GHz = 80.5 TFLOP/s nominal; FP64 a
    small fraction of that on this part)."""
    f32 = T.ttsh_fma_peak(32, 1 << 16)
    f64 = T.ttsh_fma_peak(64, 1 << 11)
    assert 20.0 < f32 < 90.0
    assert 0.05 < f64 < f32

@pytest.mark.parametrize("prec", [64, 32])
def test_diagnostics_match_oracle(T, prec):
    n, dx = 128, 0.16
    dom, p, K, s = setup(T, n, dx, 5.3, prec, 6, amp=0.3)
    dom.step(20)
    s = O.run(s, K, p, 20)
    nb = n // 4 + 1
    d = dom.diagnostics(nbins=nb + 3, centre=(0.1, -0.05))
    o = O.diagnostics(s, p, center=(0.1, -0.05), nbins=nb + 3)
    tol = 1e-11 if prec == 64 else 2e-5
    for k in ["energy", "enstrophy", "psi"]:
        assert abs(d[k] - o[k]) <= tol * max(abs(o[k]), 1e-3), (k, d[k], o[k])
    assert abs(d["mean_vx"] - o["mean_vx"]) <= 1e-6 and abs(d["mean_vy"] - o["mean_vy"]) <= 1e-6
    assert rel(d["spectrum"], o["spectrum"]) <= tol
    assert np.all(d["spectrum"][nb:] == 0)
    assert d["spectrum"].sum() == pytest.approx(d["energy"], rel=1e-6 if prec == 32 else 1e-12)
    assert d["nonfinite"] == 0 and d["status"] == T.TTSH_OK and d["step"] == 20
    # a second call gives identical bits (fixed-order reductions)
    d2 = dom.diagnostics(nbins=nb + 3, centre=(0.1, -0.05))
    assert d2["energy"] == d["energy"] and np.array_equal(d2["spectrum"], d["spectrum"])


def test_nonfinite_state_is_reported(T):
    n = 32
    dom, p, K, s = setup(T, n, 0.5, 5.0, 32, 1)
    w_hat, v0 = dom.spectral_state()
    w_hat[1, 1] = np.nan
    dom.set_spectral_state(w_hat, v0)
    d = dom.diagnostics()
    assert d["status"] == T.TTSH_E_NONFINITE and d["nonfinite"] > 0


def test_bounded_wait_timeout_is_reported_once_and_the_domain_stays_usable(T):
    """Failure detection without a GPU fault: a kernel's bounded wait on an mbarrier phase
    that nothing completes runs out after 1 ms and sets the status word; ttsh_synchronize
    reports TTSH_E_TIMEOUT once, and stepping afterwards still matches the oracle."""
    n, dx = 64, 0.25
    dom, p, K, s = setup(T, n, dx, 5.2, 32, 1, amp=0.3)
    dom.step(5)
    dom.synchronize()
    with pytest.raises(T.TTSHError):
        dom.test_bounded_wait(0.0)
    dom.test_bounded_wait(1e-3)
    with pytest.raises(T.TTSHError) as e:
        dom.synchronize()
    assert e.value.status == T.TTSH_E_TIMEOUT
    dom.synchronize()   # reported once
    dom.step(10)
    check_fields(dom, O.run(s, K, p, 15), TOL[32])


def test_stream_switch_keeps_order_and_results(T):
    """Work queued on the old stream runs before work issued after ttsh_set_stream."""
    import torch
    n, dx = 64, 0.25
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    mask = ti.circle_mask(n, dx, 5.2)
    vx, vy = ti.noise_velocity(mask, 3, 0.3)
    a = T.Domain(mask, n, dx, precision=32, stream=s1.cuda_stream)
    b = T.Domain(mask, n, dx, precision=32)
    a.set_velocity(vx, vy)
    b.set_velocity(vx, vy)
    a.step(300)
    a.set_stream(s2.cuda_stream)
    a.step(40)
    b.step(340)
    a.synchronize()
    wa, va = a.spectral_state()
    wb, vb = b.spectral_state()
    assert np.array_equal(wa, wb) and np.array_equal(va, vb)


# ------------------------------------------------------- checkpoint / graphs

@pytest.mark.parametrize("prec", [32, 64])
def test_checkpoint_resume_is_bit_exact(T, prec):
    n, dx = 64, 0.25
    mask = ti.circle_mask(n, dx, 5.2)
    vx, vy = ti.noise_velocity(mask, 9, 0.3)
    a = T.Domain(mask, n, dx, precision=prec)
    a.set_velocity(vx, vy)
    a.step(30)
    w_hat, v0 = a.spectral_state()
    a.step(170)
    b = T.Domain(mask, n, dx, precision=prec)
    b.set_spectral_state(w_hat, v0)
    b.step(170)
    wa, va = a.spectral_state()
    wb, vb = b.spectral_state()
    assert np.array_equal(wa, wb) and np.array_equal(va, vb)


def test_graph_replay_equals_eager_launches(T):
    n, dx = 64, 0.25
    mask = ti.circle_mask(n, dx, 5.2)
    vx, vy = ti.noise_velocity(mask, 4, 0.3)
    a = T.Domain(mask, n, dx, precision=32)
    b = T.Domain(mask, n, dx, precision=32)
    a.set_velocity(vx, vy)
    b.set_velocity(vx, vy)
    a.step(300)
    for _ in range(300):
        b.step(1)
    assert a.steps == b.steps == 300
    assert np.array_equal(a.spectral_state()[0], b.spectral_state()[0])


@pytest.mark.parametrize("prec,mode", [(32, 1), (64, 1), (32, 2), (64, 2), (32, 3)])
def test_launch_modes_are_bit_identical(T, prec, mode):
    n, dx = 64, 0.25
    mask = ti.circle_mask(n, dx, 5.2)
    vx, vy = ti.noise_velocity(mask, 12, 0.3)
    a = T.Domain(mask, n, dx, precision=prec)
    b = T.Domain(mask, n, dx, precision=prec)
    for d in (a, b):
        d.set_velocity(vx, vy)
    b.set_plan(0, 0, launch_mode=mode)
    assert b.plan()["launch_mode"] == mode and a.plan()["launch_mode"] == 0
    a.step(300)          # graph replays plus eager steps
    b.step(300)
    assert np.array_equal(a.spectral_state()[0], b.spectral_state()[0])
    sa, sb = a.record(130, 10), b.record(130, 10)
    assert np.array_equal(sa, sb)
    assert np.array_equal(a.spectral_state()[0], b.spectral_state()[0])
    with pytest.raises(T.TTSHError):
        T.ttsh_set_launch_mode(a.h, 4)


def test_fp64_8192_is_unsupported(T):
    with pytest.raises(T.TTSHError) as e:
        T.Domain(np.zeros((8192, 8192), np.uint8), 8192, 0.005, precision=64)
    assert e.value.status == T.TTSH_E_UNSUPPORTED


# ------------------------------------------------------------ D4 symmetry

def test_rotation_symmetry_on_gpu(T):
    n, dx = 64, 0.25
    mask = ti.circle_mask(n, dx, 5.2)
    vx, vy = ti.noise_velocity(mask, 13, 0.3)
    iy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    sy, sx = (n - ix) % n, iy
    rvx, rvy = -vy[sy, sx], vx[sy, sx]
    a = T.Domain(mask, n, dx, precision=64)
    b = T.Domain(mask, n, dx, precision=64)
    a.set_velocity(vx, vy)
    b.set_velocity(rvx, rvy)
    a.step(60)
    b.step(60)
    ax, ay, aw = a.fields()
    bx, by, bw = b.fields()
    assert rel(np.stack([bx, by]), np.stack([-ay[sy, sx], ax[sy, sx]])) <= 1e-12
    assert rel(bw, aw[sy, sx]) <= 1e-12


# ------------------------------------------------------- tile-shape variants / autotuner

@pytest.mark.parametrize("prec,n,dx,R", [(32, 64, 0.25, 5.2), (32, 512, 0.04, 5.4), (64, 128, 0.16, 5.3),
                                         (32, 2048, 0.02, 12.0)])
def test_every_step_variant_matches_oracle(T, prec, n, dx, R):
    steps = 20 if n <= 512 else 2
    dom, p, K, s = setup(T, n, dx, R, prec, 3, amp=0.3)
    w0, v00 = dom.spectral_state()
    ref = O.run(s, K, p, steps)
    plan = dom.plan()
    assert plan["n_row_variants"] >= 1 and plan["n_col_variants"] >= 1
    for rv in range(plan["n_row_variants"]):
        for cv in range(plan["n_col_variants"]):
            for mode in (0, 3):   # ordinary launches with cp.async staging; PDL with TMA staging
                dom.set_plan(rv, cv, launch_mode=mode)
                dom.set_spectral_state(w0, v00)
                dom.step(steps)
                vx, vy, w = dom.fields()
                assert rel(w, O.vorticity(ref)) <= TOL[prec], (rv, cv, mode)
                assert rel(np.stack([vx, vy]), np.stack([ref.vx, ref.vy])) <= TOL[prec], (rv, cv, mode)


def test_autotune_selects_a_valid_plan_and_keeps_state(T):
    n, dx = 256, 0.08
    dom, p, K, s = setup(T, n, dx, 5.6, 32, 8, amp=0.3)
    before = dom.spectral_state()
    plan = dom.autotune(iters=20)
    after = dom.spectral_state()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert 0 <= plan["row_variant"] < plan["n_row_variants"]
    assert 0 <= plan["col_variant"] < plan["n_col_variants"]
    assert plan == dom.plan()
    dom.step(30)
    vx, vy, w = dom.fields()
    ref = O.run(s, K, p, 30)
    assert rel(w, O.vorticity(ref)) <= TOL[32]
    with pytest.raises(T.TTSHError):
        dom.set_plan(plan["n_row_variants"], 0)


# ------------------------------------------------------------------ batched stepping

def _domain_copy(T, mask, n, dx, prec, vx, vy):
    d = T.Domain(mask, n, dx, precision=prec)
    d.set_velocity(vx, vy)
    return d


def test_batch_equals_individual_domains_bit_for_bit(T):
    specs = [(64, 0.25, 32, "c", 5.2), (64, 0.25, 32, "c", 5.0), (128, 0.16, 32, "c", 5.3),
             (128, 0.16, 64, "c", 5.3), (256, 0.08, 32, "d", 3.0), (32, 0.5, 64, "c", 5.0)]
    batched, alone = [], []
    for i, (n, dx, prec, shape, R) in enumerate(specs):
        mask = ti.circle_mask(n, dx, R) if shape == "c" else ti.dumbbell_mask(n, dx, R, 1.4 * R)
        vx, vy = ti.noise_velocity(mask, 40 + i, 0.3)
        batched.append(_domain_copy(T, mask, n, dx, prec, vx, vy))
        alone.append(_domain_copy(T, mask, n, dx, prec, vx, vy))
    b = T.Batch(batched)
    assert b.groups == 5        # the two 64^2 float circles share a launch group
    b.step(70)                  # two graph replays of 32 steps + 6 eager steps
    b.synchronize()
    for d in alone:
        d.step(70)
    for d1, d2 in zip(batched, alone):
        assert d1.steps == d2.steps == 70
        w1, v1 = d1.spectral_state()
        w2, v2 = d2.spectral_state()
        assert np.array_equal(w1, w2) and np.array_equal(v1, v2)
    b.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_persistent_batch_equals_individual_domains_bit_for_bit(T, prec):
    """One persistent launch per call advances domains of every size it holds (16^2 to 512^2,
    circles and dumbbells, several per size) with the single-domain results bit for bit; a
    second call starts from where the first stopped; the grouped launches give the same bits."""
    specs = [(512, 0.04, "c", 5.4), (16, 1.0, "c", 5.0), (256, 0.08, "d", 3.0), (128, 0.16, "c", 5.3),
             (32, 0.5, "c", 5.2), (64, 0.25, "c", 5.2), (256, 0.08, "c", 5.6), (128, 0.16, "d", 2.8),
             (64, 0.25, "d", 2.9)]
    batched, alone = [], []
    for i, (n, dx, shape, R) in enumerate(specs):
        mask = ti.circle_mask(n, dx, R) if shape == "c" else ti.dumbbell_mask(n, dx, R, 1.4 * R)
        vx, vy = ti.noise_velocity(mask, 60 + i, 0.3)
        batched.append(_domain_copy(T, mask, n, dx, prec, vx, vy))
        alone.append(_domain_copy(T, mask, n, dx, prec, vx, vy))
    b = T.Batch(batched)
    assert b.persistent
    total = 0
    for nsteps, persistent in ((70, True), (3, True), (40, False), (1, True)):
        b.set_persistent(persistent)
        b.step(nsteps)
        b.synchronize()
        total += nsteps
        for d in alone:
            d.step(nsteps)
        for d1, d2 in zip(batched, alone):
            assert d1.steps == d2.steps == total
            w1, v1 = d1.spectral_state()
            w2, v2 = d2.spectral_state()
            assert np.array_equal(w1, w2) and np.array_equal(v1, v2), (d1.n, nsteps, persistent)
    for d in batched:
        d.synchronize()          # no bounded wait ran out
    b.close()


def test_persistent_stepper_wait_timeout_is_reported_and_the_batch_stays_usable(T):
    """A dependency wait of the persistent stepper that cannot complete (one block, a column
    item whose row items are not in its work list) runs out after its limit; the first domain
    reports TTSH_E_TIMEOUT once, nothing was stepped, and the batch then steps on with the
    single-domain results."""
    specs = [(128, 0.16, 5.3), (64, 0.25, 5.2)]
    batched, alone = [], []
    for i, (n, dx, R) in enumerate(specs):
        mask = ti.circle_mask(n, dx, R)
        vx, vy = ti.noise_velocity(mask, 70 + i, 0.3)
        batched.append(_domain_copy(T, mask, n, dx, 32, vx, vy))
        alone.append(_domain_copy(T, mask, n, dx, 32, vx, vy))
    b = T.Batch(batched)
    assert b.persistent
    w_before, _ = batched[0].spectral_state()
    b.test_stalled_wait(0.05)
    with pytest.raises(T.TTSHError) as e:
        batched[0].synchronize()
    assert e.value.status == T.TTSH_E_TIMEOUT
    batched[0].synchronize()                       # reported once
    batched[1].synchronize()                       # the other domain was not involved
    w_after, _ = batched[0].spectral_state()
    assert np.array_equal(w_before, w_after)
    b.step(20)
    b.synchronize()
    for d1, d2 in zip(batched, alone):
        d2.step(20)
        w1, v1 = d1.spectral_state()
        w2, v2 = d2.spectral_state()
        assert np.array_equal(w1, w2) and np.array_equal(v1, v2)
    b.close()


def test_persistent_batch_needs_one_precision_and_default_tiles(T):
    m = ti.circle_mask(64, 0.25, 5.0)
    mixed = [T.Domain(m, 64, 0.25, precision=32), T.Domain(m, 64, 0.25, precision=64)]
    b = T.Batch(mixed)
    assert not b.persistent
    with pytest.raises(T.TTSHError) as e:
        b.set_persistent(True)
    assert e.value.status == T.TTSH_E_UNSUPPORTED
    b.close()
    big = [T.Domain(np.zeros((1024, 1024), np.uint8), 1024, 0.04, precision=32),
           T.Domain(m, 64, 0.25, precision=32)]
    b = T.Batch(big)
    assert not b.persistent
    b.close()


def test_batch_sweep_workload_matches_oracle_on_samples(T):
    doms = ti.sweep_domains()
    assert len(doms) == 48
    assert sum(d["n"] ** 2 for d in doms) == 3342336
    objs = []
    for d in doms:
        o = T.Domain(d["mask"], d["n"], d["dx"], precision=32)
        vx, vy = ti.noise_velocity(d["mask"], d["seed"], 0.3)
        o.set_velocity(vx, vy)
        objs.append(o)
    b = T.Batch(objs)
    assert b.persistent              # the whole sweep in one launch per call
    b.step(10)
    b.synchronize()
    for idx in (0, 13, 22, 40):      # a 128^2, 256^2 and 512^2 circle and a dumbbell
        d = doms[idx]
        p = O.Params(n=d["n"], dx=d["dx"])
        vx, vy = ti.noise_velocity(d["mask"], d["seed"], 0.3)
        ref = O.run(O.project_velocity(vx, vy, p), O.process_mask(d["mask"]), p, 10)
        gvx, gvy, gw = objs[idx].fields()
        assert rel(gw, O.vorticity(ref)) <= TOL[32], d["name"]
        assert rel(np.stack([gvx, gvy]), np.stack([ref.vx, ref.vy])) <= TOL[32], d["name"]
    b.close()


def test_batch_rejects_bad_input(T):
    m = ti.circle_mask(64, 0.25, 5.0)
    d = T.Domain(m, 64, 0.25, precision=32)
    with pytest.raises(T.TTSHError) as e:
        T.Batch([d, d])
    assert e.value.status == T.TTSH_E_INVALID
    big = T.Domain(np.zeros((2048, 2048), np.uint8), 2048, 0.02, precision=32)
    with pytest.raises(T.TTSHError) as e:
        T.Batch([d, big])
    assert e.value.status == T.TTSH_E_UNSUPPORTED


# ----------------------------------------- arbitrary boundary shapes (binary image input)

@pytest.mark.parametrize("prec", [64, 32])
def test_arbitrary_shape_with_obstacle_matches_oracle(T, prec):
    n, dx = 128, 0.16
    mask = ti.blob_mask(n, dx, seed=17)
    assert 0.2 < mask.mean() < 0.95                       # a real interior and a real wall
    dom, p, K, s = setup(T, n, dx, None, prec, 23, amp=0.3, mask=mask)
    assert np.abs(dom.mask() - K).max() <= (1e-13 if prec == 64 else 2e-6)
    dom.step(60)
    s = O.run(s, K, p, 60)
    check_fields(dom, s, TOL[prec])


# ------------------------------------------- temporal PSD and dumbbell order parameter

@pytest.mark.parametrize("prec", [64, 32])
def test_temporal_psd_matches_definition(T, prec):
    n, dx = 64, 0.25
    dom, p, K, s = setup(T, n, dx, 5.6, prec, 31, amp=0.3)
    omegas = np.linspace(0.0, 3.0, 7)
    dom.psd_begin(omegas)
    fields, times = [], []
    for k in range(6):
        dom.step(15)
        t = 15 * (k + 1) * p.dt
        dom.psd_accumulate(t)
        fields.append(dom.fields()[2])
        times.append(t)
    S = dom.psd_result()
    ref = O.temporal_psd(fields, times, omegas)          # the definition on the GPU's own fields
    np.testing.assert_allclose(S, ref, rtol=1e-11 if prec == 64 else 2e-6)
    traj = []
    for _ in range(6):
        s = O.run(s, K, p, 15)
        traj.append(O.vorticity(s))
    np.testing.assert_allclose(S, O.temporal_psd(traj, times, omegas), rtol=TOL[prec] * 10)


@pytest.mark.parametrize("prec", [64, 32])
def test_dumbbell_order_parameter_matches_definition(T, prec):
    n, dx, R, D = 128, 0.08, 3.0, 4.2
    mask = ti.dumbbell_mask(n, dx, R, D)
    dom, p, K, s = setup(T, n, dx, None, prec, 37, amp=0.3, mask=mask)
    dom.step(40)
    centres = [(-D / 2, 0.0), (D / 2, 0.0)]
    psi2, a, b = dom.dumbbell_order(np.array(centres).reshape(-1), D / 2)
    w = dom.fields()[2]
    ref = O.dumbbell_order_parameter(w, p, centres, D / 2)
    assert (a, b) == (ref[1], ref[2])                     # the same peaks, exactly
    assert psi2 == pytest.approx(ref[0], rel=1e-14, abs=1e-15)
    with pytest.raises(T.TTSHError):
        dom.dumbbell_order(np.array([0.01, 0.01, 0.02, 0.0]), 1e-4)   # a disc with no grid point
