"""The adaptive choice of preconditioner (Sec. 3), host logic on the CPU with
fake contexts and a fake clock."""
import pytest

from paper_1810_12437_gb300.adaptive import AdaptivePreconditioner


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def test_compares_every_period_and_keeps_the_faster():
    clock = FakeClock()
    cost = {"prior": 3.0, "jacobi": 1.0}
    calls = []

    def draw(ctx):
        calls.append(ctx)
        clock.t += cost[ctx]
        return f"beta by {ctx}"

    ad = AdaptivePreconditioner(lambda name: name, period=100, clock=clock)
    assert ad.run(0, draw) == "beta by jacobi"             # comparison step: both ran
    assert calls == ["prior", "jacobi"] and ad.current == "jacobi"
    for step in range(1, 100):
        assert ad.run(step, draw) == "beta by jacobi"      # the winner serves the others
    assert calls.count("prior") == 1
    cost["jacobi"] = 5.0                                   # the posterior changed
    assert ad.run(100, draw) == "beta by prior" and ad.current == "prior"
    assert [h[2] for h in ad.history] == ["jacobi", "prior"]


def test_period_checked():
    with pytest.raises(ValueError):
        AdaptivePreconditioner(lambda name: name, period=0)
