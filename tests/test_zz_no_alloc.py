"""ttsh_step_noalloc against the domain API (GPU).

Some callers cannot let a library allocate device memory: their memory belongs to their own
pool or a fixed budget, or an allocation's implicit device synchronisation would stall their
other work.  ttsh_step_noalloc serves them by advancing state buffers the caller owns, with
its scratch in a fixed array inside the library.  These tests hand it device buffers made by
torch, call it twice in a row, and compare each result with a domain advanced by the same
number of steps through ttsh_step, within the parity tolerances of the other GPU tests.

The first test runs on a non-blocking stream, so that in a fresh process the entry point's
first call (which writes its twiddle tables) is ordered only by its own set-up wait, and
the comparison synchronises that stream alone.  The cases cover both precisions up to the
scratch limit, n = 512 in double precision.  The file is named to be collected last.
"""
import numpy as np
import pytest

import ttsh_inputs as ti

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}


@pytest.fixture(scope="module")
def T():
    from paper_2304_03306_gb300 import build, ttsh
    build.build()
    ttsh.load_library()
    return ttsh


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_case(T, prec, n, dx, R, stream_kind):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    mask = ti.circle_mask(n, dx, R)
    vx, vy = ti.noise_velocity(mask, 21, 0.3)
    dom = T.Domain(mask, n, dx, precision=prec)
    dom.set_velocity(vx, vy)
    w_hat, v0 = dom.spectral_state()
    K = dom.mask()
    dt = torch.float32 if prec == 32 else torch.float64
    stream = torch.cuda.Stream(device=dev) if stream_kind == "non-blocking" else torch.cuda.current_stream(dev)
    with torch.cuda.stream(stream):
        K_d = torch.tensor(K, dtype=dt, device=dev).contiguous()
        w_d = torch.tensor(np.stack([w_hat.real, w_hat.imag], axis=-1), dtype=dt, device=dev).contiguous()
        v_d = torch.tensor(v0, dtype=dt, device=dev).contiguous()
    p = T.ttsh_default_params(n=n, dx=dx, precision=prec)
    for nsteps in (7, 13):
        T.ttsh_step_noalloc(p, K_d.data_ptr(), w_d.data_ptr(), v_d.data_ptr(), nsteps, stream.cuda_stream)
        stream.synchronize()           # only the stream the call was issued on
        dom.step(nsteps)
        ref_w, ref_v0 = dom.spectral_state()
        with torch.cuda.stream(stream):
            got = w_d.cpu().double().numpy()
            got_v = v_d.cpu().double().numpy()
        got_w = got[..., 0] + 1j * got[..., 1]
        assert rel(got_w, ref_w) <= TOL[prec]
        np.testing.assert_allclose(got_v, ref_v0, rtol=TOL[prec], atol=1e-300)
    dom.close()


def test_noalloc_first_call_on_a_non_blocking_stream(T):
    run_case(T, 32, 256, 0.08, 5.4, "non-blocking")


@pytest.mark.parametrize("prec,n,dx,R", [(64, 64, 0.25, 5.2), (32, 512, 0.04, 5.4), (32, 128, 0.16, 5.3),
                                         (64, 512, 0.04, 5.4)])
@pytest.mark.parametrize("stream_kind", ["current", "non-blocking"])
def test_noalloc_matches_domain_step_twice(T, prec, n, dx, R, stream_kind):
    run_case(T, prec, n, dx, R, stream_kind)


def test_noalloc_rejects_sizes_beyond_its_scratch(T):
    p = T.ttsh_default_params(n=1024, dx=0.02, precision=32)
    with pytest.raises(T.TTSHError) as e:
        T.ttsh_step_noalloc(p, 1, 1, 1, 1)          # rejected before any pointer is used
    assert e.value.status == T.TTSH_E_INVALID
    assert "512" in str(e.value)
