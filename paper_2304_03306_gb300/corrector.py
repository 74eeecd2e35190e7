"""Learned-corrector workflow: training data generated by the solver itself, training on the
GPU with the library's FNO kernels, and evaluation against the plain solver.

Every arithmetic step runs in libttsh.so (solver steps, restriction, features, residuals,
network forward/backward, Adam, corrections).  PyTorch only provides device memory for the
sample tensors and the gather of mini-batches.

Setup (same physical box L = 20.48): fine grid 512^2, dx = 0.04, dt = 0.01; coarse grid
256^2, dx = 0.08, dt_c = 4 dt.  A sample is (features of the coarse state one coarse step
after restricting the fine state, target = restricted fine vorticity four fine steps later
minus that coarse vorticity).  Training shapes: circles with R ~ U[5, 7] outside windows
around the held-out radii, and dumbbells R ~ U[2.8, 3.5], D/R ~ U[1, 1.9].
"""
from __future__ import annotations

import time

import numpy as np

from . import ttsh

FINE = dict(n=512, dx=0.04, dt=0.01)
COARSE = dict(n=256, dx=0.08, dt=0.04)
HELD_OUT = (5.5, 6.3, 6.9)
NBINS = COARSE["n"] // 4 + 1


def _inputs():
    import ttsh_inputs
    return ttsh_inputs


def mask_for(shape, grid):
    ti = _inputs()
    if shape[0] == "circle":
        return ti.circle_mask(grid["n"], grid["dx"], shape[1])
    return ti.dumbbell_mask(grid["n"], grid["dx"], shape[1], shape[2])


def training_shapes(ntraj, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < ntraj:
        if rng.random() < 0.75:
            R = float(rng.uniform(5.0, 7.0))
            if min(abs(R - h) for h in HELD_OUT) < 0.1:
                continue
            out.append(("circle", R))
        else:
            R = float(rng.uniform(2.8, 3.5))
            out.append(("dumbbell", R, float(rng.uniform(1.0, 1.9)) * R))
    return out


def _domain(shape, grid, stream=None):
    return ttsh.Domain(mask_for(shape, grid), grid["n"], grid["dx"], precision=32, dt=grid["dt"], stream=stream)


def generate(net, ntraj=64, samples=16, spacing=40, transient=3000, amplitude=0.3, seed=0):
    """Return device tensors X (S, n, n, 4) and Y (S, n, n) with S = ntraj * samples."""
    import torch
    ti = _inputs()
    shapes = training_shapes(ntraj, seed)
    fines, cas, cbs = [], [], []
    for i, sh in enumerate(shapes):
        f = _domain(sh, FINE)
        m = mask_for(sh, FINE)
        f.set_velocity(*ti.noise_velocity(m, 1000 * seed + i, amplitude))
        fines.append(f)
        cas.append(_domain(sh, COARSE))
        cbs.append(_domain(sh, COARSE))
    batch = ttsh.Batch(fines)
    batch.step(transient)
    batch.synchronize()
    n = COARSE["n"]
    S = ntraj * samples
    X = torch.empty((S, n, n, 4), device="cuda")
    Y = torch.empty((S, n, n), device="cuda")
    k = 0
    for _ in range(samples):
        for i in range(ntraj):
            ttsh.ttsh_restrict(fines[i].h, cas[i].h)
            cas[i].step(1)
        batch.step(4)
        batch.synchronize()
        for i in range(ntraj):
            ttsh.ttsh_restrict(fines[i].h, cbs[i].h)
            net.features(cas[i], X[k].data_ptr())
            net.residual(cbs[i], cas[i], Y[k].data_ptr())
            cas[i].synchronize()
            k += 1
        batch.step(spacing - 4)
        batch.synchronize()
    batch.close()
    for d in fines + cas + cbs:
        d.close()
    return X, Y


def normalise(net, X, Y):
    """Per-channel input scales and an output scale from the data (applied in place and
    stored in the network, so features/residuals of new states use the same scaling)."""
    sx = [1.0 / max(float(X[..., c].std()), 1e-12) for c in range(4)]
    sy = 1.0 / max(float(Y.std()), 1e-12)
    for c in range(4):
        X[..., c] *= sx[c]
    Y *= sy
    net.set_scales(np.array(sx, np.float32), sy)
    return sx, sy


def train(net, X, Y, iters=600, batch=8, lr=1e-3, seed=0, log_every=100):
    import torch
    rng = np.random.default_rng(seed)
    S = X.shape[0]
    xb = torch.empty((batch,) + tuple(X.shape[1:]), device="cuda")
    yb = torch.empty((batch,) + tuple(Y.shape[1:]), device="cuda")
    losses = []
    for it in range(iters):
        idx = torch.as_tensor(rng.choice(S, size=batch, replace=False), device="cuda")
        torch.index_select(X, 0, idx, out=xb)
        torch.index_select(Y, 0, idx, out=yb)
        loss, _ = net.loss_grad(xb.data_ptr(), yb.data_ptr(), batch)
        lr_t = lr * 0.5 * (1 + np.cos(np.pi * it / iters))
        net.adam_step(lr_t)
        if it % log_every == 0 or it == iters - 1:
            losses.append((it, loss))
    return losses


def _spectrum_stats(samples):
    spec = np.mean([s["spectrum"][:NBINS] for s in samples], axis=0)
    psi = np.array([s["psi"] for s in samples])
    return spec, float(psi.mean()), float(psi.std())


def spectrum_error(spec, ref):
    return float(np.sum(np.abs(spec - ref)) / np.sum(ref))


def evaluate(net, radius, coarse_steps=2000, sample_every=50, transient=3000, amplitude=0.3, seed=7,
             correct_every=1):
    """Fine 512^2 solver vs coarse 256^2 (dt x4) with and without the corrector, from the same
    spun-up state; time-averaged shell spectra over s <= 64 and the order parameter."""
    import torch
    ti = _inputs()
    shape = ("circle", radius)
    fine = _domain(shape, FINE)
    fine.set_velocity(*ti.noise_velocity(mask_for(shape, FINE), seed, amplitude))
    fine.step(transient)
    cp, cf = _domain(shape, COARSE), _domain(shape, COARSE)
    ttsh.ttsh_restrict(fine.h, cp.h)
    ttsh.ttsh_restrict(fine.h, cf.h)
    fine_state = fine.spectral_state()
    coarse_state = cp.spectral_state()
    scratch = torch.zeros(5 * COARSE["n"] ** 2, device="cuda")
    res = {"radius": radius}
    runs = {"fine": [], "plain": [], "fno": []}
    for _ in range(coarse_steps // sample_every):
        fine.step(4 * sample_every)
        cp.step(sample_every)
        net.rollout(cf, sample_every, scratch.data_ptr(), correct_every)
        runs["fine"].append(fine.diagnostics(nbins=NBINS))
        runs["plain"].append(cp.diagnostics(nbins=NBINS))
        runs["fno"].append(cf.diagnostics(nbins=NBINS))
    ref, pf, sf = _spectrum_stats(runs["fine"])
    for key in ("plain", "fno"):
        spec, pm, ps = _spectrum_stats(runs[key])
        res[f"spectrum_error_{key}"] = spectrum_error(spec, ref)
        res[f"psi_{key}"] = (pm, ps)
    res["psi_fine"] = (pf, sf)
    res["nonfinite"] = int(sum(s["nonfinite"] for r in runs.values() for s in r))
    # wall-clock of the same physical time from the same start, without diagnostics
    fine.set_spectral_state(*fine_state)
    cf.set_spectral_state(*coarse_state)
    cp.set_spectral_state(*coarse_state)
    fine.synchronize()
    t0 = time.perf_counter()
    fine.step(4 * coarse_steps)
    fine.synchronize()
    res["t_fine"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    cp.step(coarse_steps)
    cp.synchronize()
    res["t_plain"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    net.rollout(cf, coarse_steps, scratch.data_ptr(), correct_every)
    res["t_fno"] = time.perf_counter() - t0
    res["speedup_fno"] = res["t_fine"] / res["t_fno"]
    res["speedup_plain"] = res["t_fine"] / res["t_plain"]
    for d in (fine, cp, cf):
        d.close()
    return res


def main(argv=None):
    """Run the corrector network's forward pass on random inputs and report its time:
    python -m paper_2304_03306_gb300.corrector --passes K [--batch B] (configured network:
    256^2, width 32, 16 modes, 4 layers).  Useful for timing and profiling the network alone."""
    import argparse

    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--passes", type=int, default=3)
    ap.add_argument("--batch", type=int, default=1)
    a = ap.parse_args(argv)
    net = ttsh.FNO(n=COARSE["n"], width=32, modes=16, layers=4, max_batch=max(1, a.batch), seed=0)
    x = torch.randn((a.batch, COARSE["n"], COARSE["n"], 4), device="cuda")
    y = torch.zeros((a.batch, COARSE["n"], COARSE["n"]), device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    net.forward(x.data_ptr(), y.data_ptr(), a.batch)
    e0.record()
    for _ in range(a.passes):
        net.forward(x.data_ptr(), y.data_ptr(), a.batch)
    e1.record()
    torch.cuda.synchronize()
    print(f"forward, batch {a.batch}: {e0.elapsed_time(e1) / max(1, a.passes):.4f} ms per pass")
    net.close()


if __name__ == "__main__":
    main()
