"""Device-side time series (ttsh_step_record) against the oracle and against ttsh_diagnostics.

The recorder samples energy, enstrophy and the order parameter of Sec. III.C inside the row
pass of the sampled step.  Its per-thread sums are taken in the domain precision, so an
FP32 series agrees with the double-accumulated ttsh_diagnostics of the same state to a few
FP32 unit round-offs (2e-6 relative here), and with the FP64 oracle within the FP32 field
tolerance; an FP64 series agrees with the oracle to 1e-11.  Recording must not change the
trajectory: the state after a recorded run is bit-identical to plain stepping.
"""
import numpy as np
import pytest

import ttsh_inputs as ti
from oracle import ttsh_oracle as O

pytestmark = pytest.mark.gpu

CENTRE = (0.1, -0.05)


@pytest.fixture(scope="module")
def T():
    from paper_2304_03306_gb300 import build, ttsh
    build.build()
    ttsh.load_library()
    return ttsh


def pair(T, n, dx, R, prec, seed, amp=0.3):
    mask = ti.circle_mask(n, dx, R)
    vx, vy = ti.noise_velocity(mask, seed, amp)
    doms = []
    for _ in range(2):
        d = T.Domain(mask, n, dx, precision=prec)
        d.set_velocity(vx, vy)
        doms.append(d)
    return doms, mask, vx, vy


def close(a, b, tol, floor=1e-3):
    return abs(a - b) <= tol * max(abs(b), floor)


# Psi = (S2 / S3 - 2/pi) / (1 - 2/pi) is an affine map of the ratio S2 / S3 of two sums (Sec.
# III.C), so a relative rounding error e of that ratio moves Psi by e (|Psi| + (2/pi) /
# (1 - 2/pi)): near Psi = 0 the error is relative to the ratio, not to Psi.
PSI_OFFSET = (2 / np.pi) / (1 - 2 / np.pi)


def close_q(kind, a, b, tol):
    if kind == "psi":
        return abs(a - b) <= tol * (abs(b) + PSI_OFFSET)
    return close(a, b, tol)


@pytest.mark.parametrize("prec", [64, 32])
def test_recorded_series_matches_oracle(T, prec):
    n, dx = 128, 0.16
    (dom, _), mask, vx, vy = pair(T, n, dx, 5.3, prec, 6)
    p = O.Params(n=n, dx=dx)
    K = O.process_mask(mask)
    s = O.project_velocity(vx, vy, p)
    ser = dom.record(45, 10, centre=CENTRE)
    assert ser.shape == (5, 5) and dom.steps == 45
    assert np.array_equal(ser[:, 0], [0, 10, 20, 30, 40])
    assert np.all(ser[:, 4] == 0)
    tol = 1e-11 if prec == 64 else 2e-5
    for j in range(5):
        o = O.diagnostics(s, p, center=CENTRE)
        for c, k in ((1, "energy"), (2, "enstrophy"), (3, "psi")):
            assert close_q(k, ser[j, c], o[k], tol), (j, k, ser[j, c], o[k])
        s = O.run(s, K, p, 10)


@pytest.mark.parametrize("prec", [32, 64])
def test_record_graph_path_keeps_trajectory_and_matches_diagnostics(T, prec):
    n, dx = 64, 0.25
    (a, b), _, _, _ = pair(T, n, dx, 5.2, prec, 4)
    ser = a.record(300, 10, centre=CENTRE)   # 60-step graphs with 6 samples each
    assert ser.shape == (30, 5) and a.steps == 300
    tol = 2e-6 if prec == 32 else 1e-13
    for j in range(30):
        d = b.diagnostics(centre=CENTRE)
        assert ser[j, 0] == b.steps == 10 * j
        for c, k in ((1, "energy"), (2, "enstrophy"), (3, "psi")):
            assert close_q(k, ser[j, c], d[k], tol), (j, k, ser[j, c], d[k])
        b.step(10)
    wa, va = a.spectral_state()
    wb, vb = b.spectral_state()
    assert np.array_equal(wa, wb) and np.array_equal(va, vb)


def test_record_sparse_samples_and_repeatability(T):
    n, dx = 64, 0.25
    (a, b), _, _, _ = pair(T, n, dx, 5.2, 32, 8)
    w0, v0 = a.spectral_state()
    ser = a.record(250, 100)   # every > graph length: eager samples, plain graphs between
    assert np.array_equal(ser[:, 0], [0, 100, 200]) and a.steps == 250
    for j in range(3):
        d = b.diagnostics()
        for c, k in ((1, "energy"), (2, "enstrophy"), (3, "psi")):
            assert close_q(k, ser[j, c], d[k], 2e-6), (j, k, ser[j, c], d[k])
        b.step(min(100, 250 - b.steps))
    assert np.array_equal(a.spectral_state()[0], b.spectral_state()[0])
    # the same run again gives the same bits
    a.set_spectral_state(w0, v0)
    assert np.array_equal(a.record(250, 100), ser)


def test_record_counts_from_the_current_step(T):
    n, dx = 32, 0.5
    (a, _), _, _, _ = pair(T, n, dx, 5.0, 32, 2)
    a.step(7)
    ser = a.record(5, 2)
    assert np.array_equal(ser[:, 0], [7, 9, 11]) and a.steps == 12


def test_record_rejects_bad_arguments(T):
    import torch
    n, dx = 32, 0.5
    (a, _), _, _, _ = pair(T, n, dx, 5.0, 32, 3)
    buf = torch.zeros(5 * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TTSHError):
        a.step_record(50, 10, buf.data_ptr(), 4)          # 5 samples, room for 4
    with pytest.raises(T.TTSHError):
        a.step_record(50, 0, buf.data_ptr(), 4)           # every < 1
    host = np.zeros(5 * 8)
    with pytest.raises(T.TTSHError):
        a.step_record(10, 2, host.ctypes.data, 8)         # not device memory
    with pytest.raises(T.TTSHError):
        a.step_record(-1, 2, buf.data_ptr(), 4)
    assert a.steps == 0
    a.step_record(0, 3, None, 0)                          # nothing to record
    assert a.steps == 0
