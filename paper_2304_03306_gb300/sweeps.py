"""Radius sweeps with state continuation: the hysteresis protocol of Sec. III.C.

The paper runs its circular-domain simulations sequentially: starting from the steady state
at one radius, the radius is increased by a small step, the run continues from the previous
radius' final state until it is steady again, and the vortex order parameter Psi is measured
over several periods; the same is then done with decreasing radius.  Here each stage is a
domain of the new radius whose spectral state (omega^ and the mean flow) is set to the
previous stage's final state, stepped for `transient` steps and then for `measure` steps
while the device records E, Z and Psi every `every` steps (ttsh_step_record).  Several
independent chains (different seeds) advance together as one batch per stage.

All arithmetic runs in libttsh.so; this module only orders the calls.
"""
from __future__ import annotations

import numpy as np

from . import ttsh


def _inputs():
    import ttsh_inputs
    return ttsh_inputs


def _stage(states, radius, n, dx, precision, dt, transient, measure, every):
    """Continue every chain's state on a domain of the given radius; returns the final
    states and each chain's recorded series (rows: step, E, Z, Psi, nonfinite)."""
    import torch
    ti = _inputs()
    mask = ti.circle_mask(n, dx, radius)
    doms = []
    for w_hat, v0 in states:
        d = ttsh.Domain(mask, n, dx, precision=precision, dt=dt)
        d.set_spectral_state(w_hat, v0)
        doms.append(d)
    if transient:
        if len(doms) > 1 and n <= 1024:
            b = ttsh.Batch(doms)
            b.step(transient)
            b.synchronize()
            b.close()
        else:
            for d in doms:
                d.step(transient)
    series = []
    ns = -(-measure // every)
    buf = torch.zeros(len(doms) * ns * 5, dtype=torch.float64, device="cuda")
    for i, d in enumerate(doms):
        d.step_record(measure, every, buf.data_ptr() + i * ns * 5 * 8, ns)
    for d in doms:
        d.synchronize()
    host = buf.cpu().numpy().reshape(len(doms), ns, 5)
    out_states = []
    for i, d in enumerate(doms):
        series.append(host[i])
        out_states.append(d.spectral_state())
        d.close()
    return out_states, series


def hysteresis(radii, n, dx, seeds=(0,), precision=32, dt=0.01, transient=5000, measure=5000,
               every=10, amplitude=0.01, spin_up=None):
    """Run the protocol up through `radii` and back down to radii[0].  The first stage starts from
    seeded noise (reading c6) inside radii[0] and is spun up for `spin_up` (default:
    transient) extra steps.  Returns {"up": [...], "down": [...]}, one record per stage:
    radius, per-chain Psi mean and standard deviation over the measured samples, and the
    series themselves."""
    ti = _inputs()
    mask0 = ti.circle_mask(n, dx, radii[0])
    states = []
    for s in seeds:
        d = ttsh.Domain(mask0, n, dx, precision=precision, dt=dt)
        d.set_velocity(*ti.noise_velocity(mask0, s, amplitude))
        d.step(transient if spin_up is None else spin_up)
        states.append(d.spectral_state())
        d.close()
    result = {"up": [], "down": []}
    # going down starts from the final state at the largest radius
    for direction, seq in (("up", list(radii)), ("down", list(radii)[-2::-1])):
        for R in seq:
            states, series = _stage(states, R, n, dx, precision, dt, transient, measure, every)
            psi = np.array([s[:, 3] for s in series])
            result[direction].append({"radius": float(R), "psi_mean": psi.mean(axis=1).tolist(),
                                      "psi_std": psi.std(axis=1).tolist(), "series": series})
    return result
