"""Selection logic of the launch-shape tuner, on the host: candidate caps,
the choice among timings, and the measuring protocol (a fresh batch per cap,
warmed to t_warm, timed from t_warm to t_warm + t_span, always closed)."""
import pytest

from paper_1905_08717_gb300 import autotune


def test_candidate_caps():
    assert autotune.candidate_caps(152) == [0, 304, 152, 76, 38]
    assert autotune.candidate_caps(2) == [0, 4, 2, 1]
    assert autotune.candidate_caps(1) == [0, 2, 1]
    assert autotune.candidate_caps(0) == [0, 2, 1]


def test_choose():
    assert autotune.choose({0: 1.0, 152: 0.5, 38: 0.7}) == 152
    assert autotune.choose({0: 0.5, 152: 0.5}) == 0          # a tie keeps the default
    assert autotune.choose({76: 0.5, 152: 0.5, 38: 0.9}) == 152  # else the larger cap
    with pytest.raises(ValueError):
        autotune.choose({})


class _Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def test_tune_batch_protocol():
    clock = _Clock()
    cost = {0: 3.0, 64: 1.0, 16: 2.0}  # seconds of the timed span per cap
    log = []

    class FakeBatch:
        def __init__(self, problems, q0s, stream=None, grid_cap=0):
            assert problems == ["p"] and q0s == ["q"]
            self.cap, self.t, self.closed = grid_cap, 0.0, False
            log.append(self)

        def step(self, t):
            assert t > self.t and not self.closed
            if self.t > 0.0:  # the timed span (after the warm-up step)
                assert (self.t, t) == (0.5, 0.75)
                clock.t += cost[self.cap]
            self.t = t

        def close(self):
            self.closed = True

    r = autotune.tune_batch(["p"], ["q"], 0.5, 0.25, caps=[0, 64, 16], batch_cls=FakeBatch, clock=clock)
    assert r["best"] == 64
    assert r["seconds"] == cost and r["caps"] == [0, 64, 16]
    assert [b.cap for b in log] == [0, 64, 16]
    assert all(b.closed and b.t == 0.75 for b in log)


def test_tune_batch_closes_on_error():
    seen = []

    class Failing:
        def __init__(self, problems, q0s, stream=None, grid_cap=0):
            self.closed = False
            seen.append(self)

        def step(self, t):
            raise RuntimeError("step failed")

        def close(self):
            self.closed = True

    with pytest.raises(RuntimeError):
        autotune.tune_batch(["p"], ["q"], 0.1, 0.1, caps=[0, 8], batch_cls=Failing)
    assert len(seen) == 1 and seen[0].closed
    with pytest.raises(ValueError):
        autotune.tune_batch(["p"], ["q"], 0.1, 0.0, caps=[0], batch_cls=Failing)
