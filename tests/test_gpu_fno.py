"""Learned corrector (FNO) on the GPU against the FP64 oracle.

The kernels use BF16 weights (and BF16 activations as tensor-core operands) with FP32
accumulation, so the oracle is run with the same BF16-rounded weights and the comparison
tolerance is 3e-2 relative L2, a few BF16 unit round-offs (2^-8 = 3.9e-3) amplified through
the layers.  Weight gradients are compared block by block.
"""
import numpy as np
import pytest

import ttsh_inputs as ti
from oracle import fno_oracle as F
from oracle import ttsh_oracle as O

pytestmark = pytest.mark.gpu

TOL = 3e-2


@pytest.fixture(scope="module")
def T():
    from paper_2304_03306_gb300 import build, ttsh
    build.build()
    ttsh.load_library()
    return ttsh


@pytest.fixture(scope="module")
def torch():
    return pytest.importorskip("torch")


def bf16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + (((u >> 16) & 1) + 0x7FFF)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def oracle_theta(cfg, theta):
    """The parameters as the kernels use them: learned mixing weights in BF16."""
    th = theta.astype(np.float64).copy()
    P = F.unflatten(cfg, th)
    for l in range(cfg.layers):
        for k in (f"Wr{l}", f"Wi{l}", f"W{l}"):
            P[k][...] = bf16(P[k])
    return th


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CFG = dict(n=32, width=32, modes=4, layers=2, max_batch=2)
# the corrector's configured size: 256^2 coarse grid, width 32, 16 modes, 4 layers
CFG_FULL = dict(n=256, width=32, modes=16, layers=4, max_batch=2)
SIZES = [pytest.param(CFG, id="n32-m4-l2"), pytest.param(CFG_FULL, id="n256-m16-l4")]


def make(T, seed=0, **kw):
    c = dict(CFG, **kw)
    net = T.FNO(seed=seed, **c)
    cfg = F.FNOConfig(n=c["n"], width=c["width"], modes=c["modes"], layers=c["layers"], cin=4)
    return net, cfg


def test_param_count_matches_oracle_layout(T):
    net, cfg = make(T)
    assert net.nparams == F.num_params(cfg)


@pytest.mark.parametrize("size", SIZES)
def test_forward_matches_oracle(T, torch, size):
    net, cfg = make(T, seed=3, **size)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, cfg.n, cfg.n, 4)).astype(np.float32)
    xd = torch.tensor(x, device="cuda")
    yd = torch.zeros((2, cfg.n, cfg.n), device="cuda")
    net.forward(xd.data_ptr(), yd.data_ptr(), 2)
    torch.cuda.synchronize()
    theta = net.get_params()
    ref = F.forward(cfg, oracle_theta(cfg, theta), x.astype(np.float64))
    assert rel(yd.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("size", SIZES)
def test_gradients_match_oracle_block_by_block(T, torch, size):
    net, cfg = make(T, seed=5, **size)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, cfg.n, cfg.n, 4)).astype(np.float32)
    t = rng.standard_normal((2, cfg.n, cfg.n)).astype(np.float32)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    loss, g = net.loss_grad(xd.data_ptr(), td.data_ptr(), 2, want_grad=True)
    L0, gr = F.loss_and_grad(cfg, oracle_theta(cfg, net.get_params()), x.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(L0, rel=TOL)
    o = 0
    for name, shp in F.param_shapes(cfg):
        k = int(np.prod(shp))
        assert rel(g[o:o + k], gr[o:o + k]) <= TOL, name
        o += k
    # deterministic reductions: a second call gives the same bits
    _, g2 = net.loss_grad(xd.data_ptr(), td.data_ptr(), 2, want_grad=True)
    assert np.array_equal(g, g2)


def test_adam_step_matches_oracle(T, torch):
    net, cfg = make(T, seed=7)
    rng = np.random.default_rng(2)
    x = torch.tensor(rng.standard_normal((1, cfg.n, cfg.n, 4)).astype(np.float32), device="cuda")
    t = torch.tensor(rng.standard_normal((1, cfg.n, cfg.n)).astype(np.float32), device="cuda")
    th0 = net.get_params()
    _, g = net.loss_grad(x.data_ptr(), t.data_ptr(), 1, want_grad=True)
    net.adam_step(1e-3)
    th1 = net.get_params()
    ref, _, _ = F.adam_update(th0.astype(np.float64), g.astype(np.float64), 0 * th0, 0 * th0, 1, 1e-3)
    np.testing.assert_allclose(th1, ref, atol=2e-6)


def test_training_reduces_loss_teacher_student(T, torch):
    teacher, cfg = make(T, seed=11, max_batch=2)
    student, _ = make(T, seed=12, max_batch=2)
    rng = np.random.default_rng(3)
    x = torch.tensor(rng.standard_normal((2, cfg.n, cfg.n, 4)).astype(np.float32), device="cuda")
    y = torch.zeros((2, cfg.n, cfg.n), device="cuda")
    teacher.forward(x.data_ptr(), y.data_ptr(), 2)
    torch.cuda.synchronize()
    first, _ = student.loss_grad(x.data_ptr(), y.data_ptr(), 2)
    for _ in range(150):
        loss, _ = student.loss_grad(x.data_ptr(), y.data_ptr(), 2)
        student.adam_step(3e-3)
    assert loss < 0.2 * first


def test_restrict_samples_band_limited_field(T):
    nf, nc, L = 128, 64, 16.0
    X, Y = ti.grid_coords(nf, L / nf)
    dk = 2 * np.pi / L
    th = dk * (3 * X + 2 * Y) + 0.2
    vx, vy = -2 * dk * np.sin(th), 3 * dk * np.sin(th)
    fine = T.Domain(np.zeros((nf, nf), np.uint8), nf, L / nf, precision=32)
    fine.set_velocity(vx + 0.01, vy)
    coarse = T.Domain(np.zeros((nc, nc), np.uint8), nc, L / nc, precision=32)
    T.ttsh_restrict(fine.h, coarse.h)
    fx, fy, fw = fine.fields()
    cx, cy, cw = coarse.fields()
    assert rel(cw, fw[::2, ::2]) <= 1e-6
    assert rel(np.stack([cx, cy]), np.stack([fx[::2, ::2], fy[::2, ::2]])) <= 1e-6


def test_correct_adds_projected_network_output(T, torch):
    n, dx = 32, 0.5
    mask = ti.circle_mask(n, dx, 5.0)
    dom = T.Domain(mask, n, dx, precision=32)
    vx, vy = ti.noise_velocity(mask, 3, 0.3)
    dom.set_velocity(vx, vy)
    net, cfg = make(T, seed=9, n=n, max_batch=1)
    scales = np.array([0.5, 2.0, 2.0, 1.0], np.float32)
    net.set_scales(scales, 4.0)
    bx, by, bw = dom.fields()
    K = dom.mask()
    scratch = torch.zeros(5 * n * n, device="cuda")
    net.correct(dom, scratch.data_ptr())
    ax, ay, aw = dom.fields()
    x = np.stack([bw * scales[0], bx * scales[1], by * scales[2], K * scales[3]], axis=-1)[None]
    delta = F.forward(cfg, oracle_theta(cfg, net.get_params()), x)[0] / 4.0
    p = O.Params(n=n, dx=dx)
    _, _, M2 = O.wavenumbers(p)
    D = O.dft2(delta)
    D[(M2 == 0) | (M2 > (n // 4) ** 2)] = 0
    expect = np.real(O.idft2(D))
    assert rel(aw - bw, expect) <= TOL
    # zero weights except the output bias: a constant correction is removed by the projection
    th = np.zeros(net.nparams, np.float32)
    th[-1] = 3.0
    net.set_params(th)
    w_before, v_before = dom.spectral_state()
    net.correct(dom, scratch.data_ptr())
    w_after, v_after = dom.spectral_state()
    assert np.abs(w_after - w_before).max() <= 1e-5 * max(1.0, np.abs(w_before).max())
    assert np.array_equal(v_after, v_before)


def test_rollout_graph_equals_manual_loop(T, torch):
    n, dx = 64, 0.32
    mask = ti.circle_mask(n, dx, 5.4)
    vx, vy = ti.noise_velocity(mask, 5, 0.3)
    net, _ = make(T, seed=13, n=n, max_batch=1)
    net.set_scales(np.array([0.5, 2.0, 2.0, 1.0], np.float32), 8.0)
    scratch = torch.zeros(5 * n * n, device="cuda")
    a = T.Domain(mask, n, dx, precision=32, dt=0.04)
    b = T.Domain(mask, n, dx, precision=32, dt=0.04)
    a.set_velocity(vx, vy)
    b.set_velocity(vx, vy)
    net.rollout(a, 23, scratch.data_ptr(), correct_every=2)
    for _ in range(11):
        b.step(2)
        net.correct(b, scratch.data_ptr())
    b.step(1)
    b.synchronize()
    assert a.steps == b.steps == 23
    wa, va = a.spectral_state()
    wb, vb = b.spectral_state()
    assert np.array_equal(wa, wb) and np.array_equal(va, vb)


def test_corrector_workflow_small(T, torch):
    from paper_2304_03306_gb300 import corrector as Cr
    net = T.FNO(n=256, width=32, modes=8, layers=2, max_batch=4, seed=1)
    X, Y = Cr.generate(net, ntraj=3, samples=2, spacing=8, transient=40, amplitude=0.3, seed=2)
    assert X.shape == (6, 256, 256, 4) and Y.shape == (6, 256, 256)
    assert bool(torch.isfinite(X).all()) and bool(torch.isfinite(Y).all())
    Cr.normalise(net, X, Y)
    losses = Cr.train(net, X, Y, iters=20, batch=4, lr=1e-3, log_every=19)
    assert losses[-1][1] < losses[0][1]
    r = Cr.evaluate(net, 6.3, coarse_steps=40, sample_every=20, transient=40)
    assert r["nonfinite"] == 0 and r["t_fno"] > 0 and 0 <= r["spectrum_error_plain"] < 10
