"""ttsh_step_noalloc against the domain API (GPU).

Some callers cannot let a library allocate device memory: their memory belongs to their own
pool or a fixed budget, or an allocation's implicit device synchronisation would stall their
other work.  ttsh_step_noalloc serves them by advancing state buffers the caller owns, with
its scratch in a fixed array inside the library.  This test hands it device buffers made by
torch, calls it twice in a row, and compares each result with a domain advanced by the same
number of steps through ttsh_step, within the parity tolerances of the other GPU tests.
It sits in its own file named to be collected last.
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


@pytest.mark.parametrize("prec,n,dx,R", [(64, 64, 0.25, 5.2), (32, 512, 0.04, 5.4), (32, 128, 0.16, 5.3)])
def test_noalloc_matches_domain_step_twice(T, prec, n, dx, R):
    torch = pytest.importorskip("torch")
    mask = ti.circle_mask(n, dx, R)
    vx, vy = ti.noise_velocity(mask, 21, 0.3)
    dom = T.Domain(mask, n, dx, precision=prec)
    dom.set_velocity(vx, vy)
    w_hat, v0 = dom.spectral_state()
    K = dom.mask()
    dt = torch.float32 if prec == 32 else torch.float64
    dev = torch.device("cuda", 0)
    K_d = torch.tensor(K, dtype=dt, device=dev).contiguous()
    w_d = torch.tensor(np.stack([w_hat.real, w_hat.imag], axis=-1), dtype=dt, device=dev).contiguous()
    v_d = torch.tensor(v0, dtype=dt, device=dev).contiguous()
    p = T.ttsh_default_params(n=n, dx=dx, precision=prec)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for nsteps in (7, 13):
        T.ttsh_step_noalloc(p, K_d.data_ptr(), w_d.data_ptr(), v_d.data_ptr(), nsteps, stream)
        torch.cuda.synchronize(dev)
        dom.step(nsteps)
        ref_w, ref_v0 = dom.spectral_state()
        got = w_d.cpu().double().numpy()
        got_w = got[..., 0] + 1j * got[..., 1]
        assert rel(got_w, ref_w) <= TOL[prec]
        np.testing.assert_allclose(v_d.cpu().double().numpy(), ref_v0, rtol=TOL[prec], atol=1e-300)
    dom.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(T):
    p = T.ttsh_default_params(n=1024, dx=0.02, precision=32)
    with pytest.raises(T.TTSHError) as e:
        T.ttsh_step_noalloc(p, 1, 1, 1, 1)          # rejected before any pointer is used
    assert e.value.status == T.TTSH_E_INVALID
    assert "512" in str(e.value)
