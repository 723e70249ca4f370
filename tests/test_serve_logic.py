"""Host-side scheduling logic of the continuous-batching server (no GPU: fake engines)."""
import numpy as np

from paper_1807_00086_gb300.serve import Request, Server, serving_workload


class FakeEngine:
    created = []

    def __init__(self, shape, R, nbytes):
        self.shape, self.R = shape, R
        self.slots = [None] * R
        self.left = [0] * R
        self.bytes = nbytes
        self.dofs_per_column = 10
        self.closed = False
        FakeEngine.created.append(self)

    def free_slot(self):
        for j, r in enumerate(self.slots):
            if r is None:
                return j
        return None

    def active(self):
        return any(r is not None for r in self.slots)

    def admit(self, req, j):
        self.slots[j] = req
        self.left[j] = req.nsteps

    def step(self):
        fin = []
        for j, r in enumerate(self.slots):
            if r is not None:
                self.left[j] -= 1
                if self.left[j] == 0:
                    r.result = np.array([r.rid])
                    fin.append(r)
                    self.slots[j] = None
        return fin

    def close(self):
        self.closed = True


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001          # every query advances time a little
        return self.t

    def sleep(self, dt):
        self.t += dt


def _run(reqs, budget, R=2, per_engine=100):
    FakeEngine.created = []
    srv = Server(budget, R=R, engine_factory=lambda sh: FakeEngine(sh, R, per_engine),
                 estimate=lambda d, N, k, R, p: per_engine)
    stats = srv.run(reqs)
    srv.close()
    return stats


def test_every_request_completes_and_latency_is_positive():
    reqs = [Request(i, 0.0005 * i, 2 + i % 2, 8, 1 + i % 3, 3 + i % 5, np.zeros(2)) for i in range(20)]
    stats = _run(reqs, budget=10_000)
    assert stats["requests"] == 20
    assert all(r.result is not None and r.finished >= r.arrival for r in reqs)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["dof_steps"] == 10 * sum(r.nsteps for r in reqs)


def test_budget_limits_resident_contexts_and_idle_ones_are_evicted():
    # 6 shapes, budget for two contexts at a time
    reqs = [Request(i, 0.0, 2, 8 + i % 6, 1, 4, np.zeros(2)) for i in range(12)]
    stats = _run(reqs, budget=250, per_engine=100)
    assert stats["requests"] == 12
    assert len(FakeEngine.created) >= 6
    evicted = [e for e in FakeEngine.created if e.closed]
    assert len(evicted) >= 4        # contexts were recycled to stay under the budget


def test_same_shape_requests_share_a_context_in_slots():
    reqs = [Request(i, 0.0, 3, 4, 2, 5, np.zeros(3)) for i in range(5)]
    _run(reqs, budget=10_000, R=4)
    assert len(FakeEngine.created) == 1


def test_serving_workload_shapes():
    reqs = serving_workload(n_req=300, rate=20.0, seed=5)
    assert len(reqs) == 300
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) >= 0) and 10 < arr[-1] < 20       # ~ 300 / 20 s
    for r in reqs:
        ne = 2 * r.N ** 2 if r.dim == 2 else 6 * r.N ** 3
        assert 500 <= ne <= 2e5 and 1 <= r.k <= 4 and 20 <= r.nsteps <= 200
        assert np.all((r.source >= 0.1) & (r.source <= 0.9))
    assert len({r.shape for r in reqs}) < 80                    # shapes repeat: batching is possible
