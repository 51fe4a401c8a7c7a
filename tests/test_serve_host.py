"""Host logic of the serving loop (admission against the HBM budget, continuous batching,
release of finished simulations), run on the CPU against a fake library: every call the loop
makes into the native layer is replaced by a stand-in that only keeps counts."""
import pytest

import paper_2311_05170_gb300.serve as serve
from paper_2311_05170_gb300.native import TPNS_EBUDGET, TpnsError


class FakeWorkload:
    def __init__(self, name, nbytes, dofs):
        self.name, self.nbytes, self.dofs = name, nbytes, dofs


class FakeSolver:
    live = []
    created = []

    def __init__(self, w, precision="fp32", hbm_budget_bytes=0, stream=None):
        if w.nbytes > hbm_budget_bytes:
            raise TpnsError(TPNS_EBUDGET, "over budget")
        self.w, self.steps, self.closed = w, 0, False
        FakeSolver.live.append(self)
        FakeSolver.created.append(w.name)

    def stats(self):
        return {"n_fine_dofs": self.w.dofs, "device_bytes": self.w.nbytes, "last_step_ms": 1.0 + self.steps}

    def fields(self):
        return {"steps": self.steps}

    def close(self):
        self.closed = True
        FakeSolver.live.remove(self)


def fake_batch_step(solvers):
    assert len({id(s) for s in solvers}) == len(solvers)
    assert sum(s.w.nbytes for s in solvers) <= fake_batch_step.budget
    fake_batch_step.max_live = max(fake_batch_step.max_live, len(solvers))
    for s in solvers:
        assert not s.closed
        s.steps += 1


@pytest.fixture
def fake(monkeypatch):
    FakeSolver.live, FakeSolver.created = [], []
    fake_batch_step.max_live = 0
    monkeypatch.setattr(serve, "Solver", FakeSolver)
    monkeypatch.setattr(serve, "batch_step", fake_batch_step)
    return FakeSolver


def test_every_request_runs_its_steps_within_the_budget(fake):
    budget = 100
    fake_batch_step.budget = budget
    reqs = [(0.0, FakeWorkload("a", 60, 10), 3), (0.0, FakeWorkload("b", 50, 20), 2),
            (0.0, FakeWorkload("c", 30, 5), 4)]
    stats, done = serve.run_serving(reqs, budget, keep_fields=True, time_scale=0.0, background=False)
    assert stats["requests"] == 3 and not fake.live
    by = {r.w.name: r for r in done}
    for name, n in (("a", 3), ("b", 2), ("c", 4)):
        assert by[name].done_steps == n and by[name].fields == {"steps": n}
        assert by[name].latencies_ms == [1.0 + k for k in range(1, n + 1)]
    # a and c fit together (90), b (50) waits for a to finish: b was refused while a held 60
    assert stats["refused_for_budget"] >= 1
    assert fake.created[:2] == ["a", "c"] and fake.created[2] == "b"
    assert stats["ticks"] == 3 + 2        # a's 3 ticks (c beside it), then b with c's last step
    assert stats["max_concurrency"] == 2 and fake_batch_step.max_live == 2
    assert stats["step_latency_ms_p50"] is not None and stats["tick_ms_p99"] is not None


def test_max_live_caps_the_batch(fake):
    fake_batch_step.budget = 10 ** 9
    reqs = [(0.0, FakeWorkload(str(i), 1, 1), 2) for i in range(7)]
    stats, done = serve.run_serving(reqs, 10 ** 9, max_live=3, time_scale=0.0, background=False)
    assert stats["requests"] == 7 and fake_batch_step.max_live == 3
    assert all(r.done_steps == 2 for r in done)
    assert stats["dof_steps_per_s"] > 0


def test_other_errors_are_not_swallowed(fake, monkeypatch):
    class Broken(FakeSolver):
        def __init__(self, *a, **k):
            raise TpnsError(1, "invalid")

    monkeypatch.setattr(serve, "Solver", Broken)
    with pytest.raises(TpnsError):
        serve.run_serving([(0.0, FakeWorkload("x", 1, 1), 1)], 10, time_scale=0.0, background=False)
    with pytest.raises(TpnsError):
        serve.run_serving([(0.0, FakeWorkload("x", 1, 1), 1)], 10, time_scale=0.0, background=True)
