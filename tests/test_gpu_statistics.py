"""FP32 against FP64 beyond the time over which the two trajectories stay together (GPU).

Statistics, not states, are compared once rounding differences have been amplified:
* the 512^2 oscillating-pair configuration (R = 5.4, dx = 0.04, noise 0.01, seed 2),
  2e4 steps with the order parameter recorded every 10 steps: the mean and standard
  deviation of Psi, and the mean energy, in FP32 and FP64 within 2 %;
* the 2048^2 turbulent configuration (R = 12, dx = 0.02, noise 0.01, seed 4), 1e4 steps,
  the energy spectrum E(s) averaged over the last 2e3 steps (a sample every 20 steps).  Its
  FP32-vs-FP64 difference sum|dE| / sum E is compared with the spread of the same statistic
  between runs that differ only in the noise seed: a single 2e3-step window of this chaotic
  flow does not determine E(s) to 2 % (two FP32 runs from different seeds differ by about
  10 %), so the check is that FP32 and FP64 differ no more than independent samples do.
"""
import numpy as np
import pytest

import ttsh_inputs as ti

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2304_03306_gb300 import build, ttsh
    build.build()
    ttsh.load_library()
    return ttsh


def test_512_order_parameter_statistics_fp32_vs_fp64(T):
    w = ti.WORKLOADS["circle512"]
    mask = ti.circle_mask(w["n"], w["dx"], w["radius"])
    series = {}
    for prec in (32, 64):
        d = T.Domain(mask, w["n"], w["dx"], precision=prec)
        d.init_noise(w["seed"], 0.01)
        series[prec] = d.record(20000, 10)
        d.close()
    for lo in (0, 1000):                                    # whole run, second half
        a, b = series[32][lo:], series[64][lo:]
        assert abs(a[:, 3].mean() - b[:, 3].mean()) <= 0.02 * abs(b[:, 3].mean())
        assert abs(a[:, 3].std() - b[:, 3].std()) <= 0.02 * b[:, 3].std()
        assert abs(a[:, 1].mean() - b[:, 1].mean()) <= 0.02 * b[:, 1].mean()
    assert np.all(series[32][:, 4] == 0) and np.all(series[64][:, 4] == 0)


def _window_spectrum(T, prec, seed, total=10000, last=2000, every=20):
    w = ti.WORKLOADS["circle2048_turbulent"]
    n, dx = w["n"], w["dx"]
    d = T.Domain(ti.circle_mask(n, dx, w["radius"]), n, dx, precision=prec)
    d.init_noise(seed, 0.01)
    d.step(total - last)
    first = d.diagnostics(nbins=n // 4 + 1)["spectrum"]
    acc = np.zeros(n // 4 + 1)
    for _ in range(last // every):
        d.step(every)
        acc += d.diagnostics(nbins=n // 4 + 1)["spectrum"]
    d.close()
    return acc / (last // every), first


def _diff(a, b):
    return float(np.abs(a - b).sum() / b.sum())


def test_2048_spectrum_fp32_is_within_the_spread_of_independent_samples(T):
    seed = ti.WORKLOADS["circle2048_turbulent"]["seed"]
    s64, first64 = _window_spectrum(T, 64, seed)
    s32, first32 = _window_spectrum(T, 32, seed)
    others = [_window_spectrum(T, 32, seed + k)[0] for k in (1, 2, 3)]
    # the two runs from the same initial state have separated by the start of the window
    assert _diff(first32, first64) > 1e-3
    d_prec = _diff(s32, s64)
    members = [s32] + others
    spread = [_diff(members[i], members[j]) for i in range(len(members)) for j in range(i)]
    print(f"2048^2 window E(s): FP32 vs FP64 {d_prec:.4f}; seed-to-seed FP32 spread "
          f"{min(spread):.4f}..{max(spread):.4f}")
    assert d_prec <= max(spread)
    # the FP64 run is no outlier either: its distance to the FP32 members' mean is within
    # the members' own distances to that mean
    mean32 = np.mean(members, axis=0)
    assert _diff(s64, mean32) <= max(_diff(m, mean32) for m in members) * 1.5
