"""Host-side order of the hysteresis protocol (Sec. III.C), with the device work replaced by
fakes: the chains are spun up once at the first radius, go up through every radius and come
back down to the first, each stage continuing from the previous stage's final states."""
import numpy as np

from paper_2304_03306_gb300 import sweeps


class FakeDomain:
    made = []

    def __init__(self, mask, n, dx, precision=32, dt=0.01):
        self.steps = 0
        FakeDomain.made.append(self)

    def set_velocity(self, vx, vy):
        self.v = float(np.abs(vx).sum() + np.abs(vy).sum())

    def step(self, n):
        self.steps += n

    def spectral_state(self):
        return ("spun", self.steps), np.zeros(2)

    def close(self):
        pass


def test_hysteresis_visits_radii_up_then_down_and_continues_states(monkeypatch):
    calls = []

    def fake_stage(states, radius, n, dx, precision, dt, transient, measure, every):
        calls.append((radius, [s[0] for s in states], transient, measure, every))
        ns = -(-measure // every)
        series = [np.column_stack([np.arange(ns) * every, np.ones(ns), np.ones(ns),
                                   np.full(ns, radius), np.zeros(ns)]) for _ in states]
        return [(("after", radius), s[1]) for s in states], series

    monkeypatch.setattr(sweeps, "_stage", fake_stage)
    monkeypatch.setattr(sweeps.ttsh, "Domain", FakeDomain)
    radii = [5.20, 5.22, 5.24, 5.26]
    r = sweeps.hysteresis(radii, 64, 0.25, seeds=(1, 2), transient=7, measure=25, every=10,
                          spin_up=11)
    assert [c[0] for c in calls] == [5.20, 5.22, 5.24, 5.26, 5.24, 5.22, 5.20]
    # spin-up once per seed at the first radius, then every stage starts from the last one's states
    assert calls[0][1] == [("spun", 11), ("spun", 11)]
    for prev, cur in zip(calls, calls[1:]):
        assert cur[1] == [("after", prev[0])] * 2
    assert all(c[2:] == (7, 25, 10) for c in calls)
    assert [s["radius"] for s in r["up"]] == radii
    assert [s["radius"] for s in r["down"]] == radii[-2::-1]
    for d in ("up", "down"):
        for s in r[d]:
            assert s["psi_mean"] == [s["radius"]] * 2 and s["psi_std"] == [0.0, 0.0]
            assert len(s["series"]) == 2 and s["series"][0].shape == (3, 5)
