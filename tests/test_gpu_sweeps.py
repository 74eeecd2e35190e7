"""The hysteresis protocol (Sec. III.C) on the GPU against the same protocol run by the oracle:
state continued across radii, Psi recorded during each stage's measurement window."""
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


def oracle_chain(radii, n, dx, seed, spin_up, transient, measure, every):
    p = O.Params(n=n, dx=dx)
    m0 = ti.circle_mask(n, dx, radii[0])
    s = O.project_velocity(*ti.noise_velocity(m0, seed, 0.3), p)
    s = O.run(s, O.process_mask(m0), p, spin_up)
    out = {}
    for direction, seq in (("up", list(radii)), ("down", list(radii)[-2::-1])):
        rows = []
        for R in seq:
            K = O.process_mask(ti.circle_mask(n, dx, R))
            s = O.run(s, K, p, transient)
            psi = []
            for j in range(measure):
                if j % every == 0:
                    psi.append(O.diagnostics(s, p)["psi"])
                s = O.step(s, K, p)
            rows.append(psi)
        out[direction] = rows
    return out


def test_hysteresis_chain_matches_oracle(T):
    from paper_2304_03306_gb300 import sweeps
    radii, n, dx = (5.0, 5.2, 5.4), 32, 0.5
    res = sweeps.hysteresis(radii, n, dx, seeds=(3, 4), precision=64, transient=20, measure=30,
                            every=10, amplitude=0.3, spin_up=25)
    assert [r["radius"] for r in res["up"]] == list(radii)
    assert [r["radius"] for r in res["down"]] == [5.2, 5.0]
    for c, seed in enumerate((3, 4)):
        ref = oracle_chain(radii, n, dx, seed, 25, 20, 30, 10)
        for direction in ("up", "down"):
            for stage, want in zip(res[direction], ref[direction]):
                got = stage["series"][c][:, 3]
                np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12)
                assert np.all(stage["series"][c][:, 4] == 0)
