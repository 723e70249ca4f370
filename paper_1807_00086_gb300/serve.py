"""Continuous-batching server for implicit HDG wave-solve requests.

A request asks for `nsteps` implicit BDF2 steps of an acoustic wave on a structured simplex
mesh (dimension, mesh size N, degree k) driven by one Ricker point source at a given
position, starting from rest. Requests of the same shape share the element operators
(the factored local blocks and every S_K of Sec. 2.4, Eq. LS), so the server keeps one
resident context per shape with R slots: each admitted request occupies one right-hand-side
column, and one `hdg_step` advances every request of that shape in the same launches.

Continuous batching: requests are admitted whenever a slot of their shape is free, even
while other requests of that shape are mid-solve (a slot is reset to rest and its source is
delayed to the slot's start time); a context is created only when the device-memory budget
allows it, after evicting idle contexts. Contexts of different shapes run on their own CUDA
streams from worker threads, so their work overlaps on the device. Each request's result
depends only on its own column (per-column Krylov recurrences and convergence tests), so it
is the same alone and in a mix, within the solver tolerance.

The engine is injectable (`engine_factory`) so the scheduling logic can run without a GPU.
"""
import threading
import time
from collections import OrderedDict, deque
from dataclasses import dataclass

import numpy as np

from . import inputs

F0, T0 = 10.0, 0.12        # Ricker wavelet of every request (relative to its own start)


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    dim: int
    N: int
    k: int
    nsteps: int
    source: np.ndarray
    admitted: float = None
    finished: float = None
    result: np.ndarray = None

    @property
    def shape(self):
        return (self.dim, self.N, self.k)


def mesh_for(dim, N):
    return inputs.unit_square_tri(N) if dim == 2 else inputs.unit_cube_tet(N)


def estimate_bytes(dim, N, k, R, prec="mixed"):
    """Device bytes of one context (upper estimate of the library's allocations)."""
    from math import comb
    ne = 2 * N * N if dim == 2 else 6 * N ** 3
    nf = (3 * N * N + 2 * N) if dim == 2 else (12 * N ** 3 + 6 * N * N)
    Np, Nf = comb(k + dim, dim), comb(k + dim - 1, dim - 1)
    n, m = (dim + 1) * Np, (dim + 1) * Nf
    p4 = (m * (m + 1) // 2 + 3) // 4
    per_elem = m * m * 8 + Np * Np * 8 + 320 + m * 8 + 7 * n * 8 * R + m * 8 * R
    if prec == "mixed":
        per_elem += p4 * 16 + m * 4 * R
        if R > 1:
            per_elem += m * m * 8          # FP32 pairs of S_K for the double-float residual
        per_elem += Np * Np * 8 + 256      # double-float H^-1 and geometry (local solves)
        if R == 1:
            per_elem += p4 * 32         # double-float copy for the refinement apply
    per_face = Nf * R * (9 * 8 + 8 * 4 + 8) + 16
    per_face += Nf * R * 8 * 2 * 8          # least-squares guess: 8 stored (b, lam) pairs
    return int(ne * per_elem + nf * per_face + (1 << 20))


class Engine:
    """Resident context of one request shape with R slots (right-hand-side columns)."""

    def __init__(self, shape, R, prec="mixed", dt=2e-3, rtol=1e-12):
        import torch
        from . import hdg
        dim, N, k = shape
        self.shape, self.R, self.dt = shape, R, dt
        self.stream = hdg.own_stream()          # never shared with another context
        vert, elem = mesh_for(dim, N)
        with torch.cuda.stream(self.stream):
            self.s = hdg.Solver(vert, elem, k, 1.0, 1.0, 1.0, prec=prec, rtol=rtol, nrhs=R, use_graphs=True,
                                stream=self.stream)
            self.s.hdg_set_dirichlet(None)
            self.s.hdg_set_state(self.s.empty_fields(), 0.0)
            self.u_buf, self.lam_buf = self.s.empty_fields(), self.s.empty_traces()   # reused read-back buffers
        self.t = 0.0
        self.slots = [None] * R
        self.done_steps = [0] * R
        self.pos = np.full((R, dim), 0.5)
        self.amp = np.zeros(R)
        self.delay = np.zeros(R)
        self.bytes = self.s.sizes.device_bytes
        self.dofs_per_column = self.s.n_elem * self.s.n

    def free_slot(self):
        for j, r in enumerate(self.slots):
            if r is None:
                return j
        return None

    def active(self):
        return any(r is not None for r in self.slots)

    def admit(self, req, j):
        self.slots[j] = req
        self.done_steps[j] = 0
        self.pos[j] = req.source
        self.amp[j] = 1.0
        self.delay[j] = self.t            # the request's clock starts now
        self.s.hdg_reset_column(j)
        self._upload_sources()

    def _upload_sources(self):
        live = [j for j in range(self.R) if self.slots[j] is not None]
        if live:
            self.s.hdg_set_sources(self.pos[live], self.amp[live], F0, T0, col=np.array(live, dtype=np.int32),
                                   delay=self.delay[live])
        else:
            self.s.hdg_set_sources(np.zeros((0, self.shape[0])), np.zeros(0), F0, T0)

    def step(self):
        """One BDF2 step of every slot; returns the requests that completed."""
        import torch
        with torch.cuda.stream(self.stream):
            self.s.hdg_step(self.dt, "bdf2", 1)
        self.t += self.dt
        finished = []
        for j, r in enumerate(self.slots):
            if r is None:
                continue
            self.done_steps[j] += 1
            if self.done_steps[j] >= r.nsteps:
                finished.append(j)
        if finished:
            with torch.cuda.stream(self.stream):
                u, lam, t = self.s.hdg_get_state(u=self.u_buf, lam=self.lam_buf)
                out = [(j, u[:, :, j].cpu().numpy()) for j in finished]
            for j, arr in out:
                self.slots[j].result = arr
            done = [self.slots[j] for j in finished]
            for j in finished:
                self.slots[j] = None
                self.amp[j] = 0.0
            self._upload_sources()
            return done
        return []

    def close(self):
        from . import hdg
        self.s.close()
        self.stream.synchronize()
        hdg.release_stream(self.stream)


class Server:
    """Continuous batching: one worker thread per resident context keeps stepping while the
    context has active slots; the scheduler thread admits arrivals into free slots (taking the
    context's lock between two steps) and creates or evicts contexts under the budget."""

    def __init__(self, budget_bytes, R=4, prec="mixed", dt=2e-3, engine_factory=None, max_workers=None,
                 estimate=estimate_bytes):
        self.budget = budget_bytes
        self.R, self.prec, self.dt = R, prec, dt
        self.factory = engine_factory or (lambda shape: Engine(shape, R, prec, dt))
        self.estimate = estimate
        self.engines = OrderedDict()      # shape -> engine, least recently used first
        self.locks = {}
        self.workers = {}
        self.cv = threading.Condition()
        self.done = []
        self.dof_steps = 0
        self.error = None

    def used_bytes(self):
        return sum(e.bytes for e in self.engines.values())

    def _engine_for(self, shape):
        if shape in self.engines:
            self.engines.move_to_end(shape)
            return self.engines[shape]
        need = self.estimate(shape[0], shape[1], shape[2], self.R, self.prec)
        for sh in list(self.engines):
            if self.used_bytes() + need <= self.budget:
                break
            w = self.workers.get(sh)
            if not self.engines[sh].active() and (w is None or not w.is_alive()):
                self.engines.pop(sh).close()
                self.locks.pop(sh, None)
                self.workers.pop(sh, None)
        if self.used_bytes() + need > self.budget:
            return None
        eng = self.factory(shape)
        self.engines[shape] = eng
        self.locks[shape] = threading.Lock()
        return eng

    def _work(self, shape, clock, t_start):
        eng, lock = self.engines[shape], self.locks[shape]
        try:
            while True:
                with lock:
                    if not eng.active():
                        return
                    active_before = sum(1 for r in eng.slots if r is not None)
                    fin = eng.step()
                now = clock() - t_start
                with self.cv:
                    self.dof_steps += eng.dofs_per_column * active_before
                    for r in fin:
                        r.finished = now
                        self.done.append(r)
                    self.cv.notify_all()
        except Exception as ex:          # surfaced by run()
            with self.cv:
                self.error = ex
                self.cv.notify_all()

    def run(self, requests, clock=time.perf_counter, sleep=None):
        """Serves `requests` (arrival times in seconds from the start); returns statistics."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting = deque()
        total = len(pending)
        t_start = clock()
        with self.cv:
            self.done, self.dof_steps, self.error = [], 0, None
        while True:
            with self.cv:
                if self.error is not None:
                    raise self.error
                if len(self.done) == total:
                    break
            now = clock() - t_start
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            still = deque()
            while waiting:
                r = waiting.popleft()
                eng = self._engine_for(r.shape)
                if eng is None:
                    still.append(r)
                    continue
                with self.locks[r.shape]:
                    j = eng.free_slot()
                    if j is None:
                        still.append(r)
                        continue
                    r.admitted = clock() - t_start
                    eng.admit(r, j)
                w = self.workers.get(r.shape)
                if w is None or not w.is_alive():
                    w = threading.Thread(target=self._work, args=(r.shape, clock, t_start), daemon=True)
                    self.workers[r.shape] = w
                    w.start()
            waiting = still
            # wait for an arrival or a completion
            timeout = 0.02
            if pending:
                timeout = max(0.0, min(timeout, pending[0].arrival - (clock() - t_start)))
            with self.cv:
                if len(self.done) < total and self.error is None:
                    self.cv.wait(timeout=timeout if (pending or waiting) else 0.05)
        for w in list(self.workers.values()):
            w.join()
        wall = clock() - t_start
        lat = np.array([r.finished - r.arrival for r in self.done]) if self.done else np.zeros(1)
        # latency = waiting for a slot (and a context) + being stepped in the slot
        wait = np.array([r.admitted - r.arrival for r in self.done]) if self.done else np.zeros(1)
        serv = lat - wait
        return {"requests": len(self.done), "wall_s": wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                "wait_p50_ms": float(np.percentile(wait, 50) * 1e3), "wait_p99_ms": float(np.percentile(wait, 99) * 1e3),
                "service_p50_ms": float(np.percentile(serv, 50) * 1e3),
                "service_p99_ms": float(np.percentile(serv, 99) * 1e3),
                "dof_steps": self.dof_steps, "dof_steps_per_s": self.dof_steps / wall if wall > 0 else 0.0,
                "contexts_created": len(self.engines)}

    def close(self):
        for w in list(self.workers.values()):
            w.join()
        for e in self.engines.values():
            e.close()
        self.engines.clear()


def serving_workload(n_req=1000, rate=20.0, seed=inputs.DEFAULT_SEED, ne_lo=1e3, ne_hi=1e5):
    """Poisson arrivals at `rate`/s; 2D or 3D (p = 1/2); element count log-uniform in
    [ne_lo, ne_hi] snapped to a ladder of structured meshes (so requests share shapes);
    k uniform in {1..4}; 20..200 steps; source uniform in [0.1, 0.9]^d."""
    rng = np.random.default_rng(seed)
    ladder2 = np.array([24, 32, 45, 64, 90, 128, 181, 224])      # 2 N^2 triangles
    ladder3 = np.array([6, 8, 11, 14, 18, 22, 26])                # 6 N^3 tetrahedra
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    reqs = []
    for i in range(n_req):
        dim = int(rng.choice([2, 3]))
        ne = float(np.exp(rng.uniform(np.log(ne_lo), np.log(ne_hi))))
        if dim == 2:
            lad = ladder2[(2 * ladder2 ** 2 >= ne_lo * 0.5) & (2 * ladder2 ** 2 <= ne_hi * 2)]
            N = int(lad[np.argmin(np.abs(np.log(2 * lad ** 2) - np.log(ne)))])
        else:
            lad = ladder3[(6 * ladder3 ** 3 >= ne_lo * 0.5) & (6 * ladder3 ** 3 <= ne_hi * 2)]
            N = int(lad[np.argmin(np.abs(np.log(6 * lad ** 3) - np.log(ne)))])
        reqs.append(Request(i, float(t[i]), dim, N, int(rng.integers(1, 5)), int(rng.integers(20, 201)),
                            rng.uniform(0.1, 0.9, size=dim)))
    return reqs
