#!/usr/bin/env python
"""Benchmark: HDG DOF-steps/s of the implicit acoustic wave solver on GB300.

Workload (one step = one implicit BDF2 step through the whole hot path: element
right-hand sides, condensed right-hand side, Krylov trace solve with the matrix-free
S_K apply, local recovery): 3D acoustic wave on the unit cube, structured mesh of
32^3 cubes x 6 = 196,608 tetrahedra, degree k = 3 (80 field DOFs per element), tau = 1,
c ~ logU[1, 3] per element (seeded), rho = 1, BDF2 dt = 2e-3, Ricker point source
f0 = 10. Inputs are seeded and synthetic; the per-element operators (S_K: 2.5 GB FP64)
are far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|mixed|mixed16] [--impl ours|reference]

`--impl reference` times the CPU oracle on a bounded sample of the same workload.
Under torchrun (N > 1) every rank runs an independent replica (the path does not shard
across GPUs; no collective on the data path); value = units of all ranks / max time.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")
if "--serve" in sys.argv:
    # many resident contexts, each on its own stream: give them separate hardware queues
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "HDG DOF-steps/s on 1 GB300, mixed vs FP64 at <=1e-9 rel err; serve p50/p99 ms"
UNIT = "DOF-steps/s"
DT = 2e-3
SAMPLE_N = 4          # oracle sample: 4^3 x 6 = 384 tetrahedra, same k, same recipe
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a kernel, from an
# ncu capture of that kernel at that element count; keyed by (kernel, n_elem). An entry is
# removed whenever the kernel changes.
MEASURED_TRAFFIC = {
    ("apply16_kernel<3,3>", 196608): (346971264, "ncu dram__bytes_read.sum + dram__bytes_write.sum, mean of 3 launches "
                                                  "at this size (profiles/apply16_acoustic3d_k3_196608tets_dram.md)"),
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi during the timed region (SM clock, max clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------- oracle legs
def oracle_sample(steps=None, budget_s=None, warmup=0):
    """Times the CPU oracle on the bounded sample: BDF2 steps of the 384-tet workload."""
    from oracle import acoustic as ac
    from paper_1807_00086_gb300 import inputs
    w = inputs.acoustic_3d_workload(N=SAMPLE_N)
    prob = ac.build_problem(w["vert"], w["elem"], w["k"], w["tau"], w["rho"], w["c"])
    ac.add_point_source(prob, w["sources"][0], w["f0"], w["t0"])
    ne = w["elem"].shape[0]
    nloc = 4 * prob.Np
    u = np.zeros((ne, nloc))
    cond = ac.condense(prob, 1.5 / DT)
    hist = [u, u]
    t = 0.0
    times = []

    def one_step():
        nonlocal hist, t
        t += DT
        h = (4.0 / 3.0) * hist[1] - (1.0 / 3.0) * hist[0]
        un, lam = ac.solve_stage(prob, cond, h, t)
        hist = [hist[1], un]

    for _ in range(warmup):
        one_step()
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        one_step()
        times.append(time.perf_counter() - t0)
        if steps is not None and len(times) >= steps:
            break
        if budget_s is not None and time.perf_counter() - t_start >= budget_s:
            break
    total = sum(times)
    dofs = ne * nloc
    return {"value": dofs * len(times) / total, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": "%d BDF2 steps of the same workload on a %d^3x6 = %d-tet mesh (k=3, %d field DOFs); "
                      "oracle = numpy/scipy FP64, per-element LU + sparse direct trace solve" % (len(times), SAMPLE_N,
                                                                                                ne, dofs),
            "ms_per_step": 1e3 * total / len(times), "steps": len(times)}


def _oracle_worker(budget_s):
    return oracle_sample(budget_s=budget_s)["value"]


def oracle_all_cores(budget_s):
    """The same oracle sample run as one single-threaded process per host core at once
    (replicas, as the GPU runs replicas): the aggregate DOF-steps/s of the host. The pool is
    started with spawn, so no worker inherits the parent's CUDA context."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    with mp.get_context("spawn").Pool(n) as pool:
        vals = pool.map(_oracle_worker, [budget_s] * n)
    return {"value": float(sum(vals)), "processes": n, "per_process_min": float(min(vals)),
            "per_process_max": float(max(vals))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    r = oracle_sample(steps=args.steps, warmup=args.warmup)
    out = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "acoustic3d_k3_32cube_bdf2 (bounded sample: %d^3x6 tets)" % SAMPLE_N},
           "cpu_baseline": {k: r[k] for k in ("value", "unit", "cores", "host_cores", "kind", "sample")},
           "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def max_over_ranks(dist, x, device):
    """The largest x over all ranks (x itself without a process group): the replicas' job
    time is that of the slowest rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------- GPU leg
def run_ours(args):
    import torch
    from paper_1807_00086_gb300 import hdg, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    R = args.nrhs
    elastic = args.physics == "elastic"
    scheme, dt = ("dirk3", 1e-3) if elastic else ("bdf2", DT)
    vardeg = elastic and args.mixed_degree
    if vardeg:
        w = inputs.elastic_3d_mixed_workload(N=args.N if args.N != 32 else 24)
    elif elastic:
        w = inputs.elastic_3d_workload(N=args.N if args.N != 32 else 24, k=args.k)
    elif R > 1:
        w = inputs.acoustic_3d_multisource_workload(N=args.N, k=args.k, nsrc=R)
    else:
        w = inputs.acoustic_3d_workload(N=args.N, k=args.k)
    ne = w["elem"].shape[0]
    u_init = None

    def make_solver(prec):
        nonlocal u_init
        if elastic:
            sv = hdg.Solver(w["vert"], w["elem"], w["k"], 1.0, w["rho"], lam=w["lam"], mu=w["mu"], prec=prec,
                            rtol=args.rtol, inner_rtol=args.inner_rtol, elem_k=w.get("elem_k"),
                            guess_history=args.guess_history, device_loops=not args.host_loops)
            if u_init is None:
                xq = sv.hdg_quadrature_points(0)
                u_init = sv.hdg_project_volume(inputs.gaussian_velocity_values(xq, w["center"], w["width"], 9))
            sv.hdg_set_state(u_init, 0.0)
            return sv
        sv = hdg.Solver(w["vert"], w["elem"], w["k"], w["tau"], w["rho"], w["c"], prec=prec, rtol=args.rtol,
                        inner_rtol=args.inner_rtol, nrhs=R, guess_history=args.guess_history,
                        device_loops=not args.host_loops, trace_space=args.trace_space, solver=args.solver,
                        precond=args.precond if args.solver == "gmres" else "jacobi")
        sv.hdg_set_sources(w["sources"], np.ones(len(w["sources"])), w["f0"], w["t0"], col=w.get("source_cols"))
        sv.hdg_set_dirichlet(None)
        sv.hdg_set_state(sv.empty_fields(), 0.0)
        return sv

    s = make_solver(args.prec)
    dofs = int(np.prod(s._fshape))
    stream = s.stream
    total = args.total_steps if args.total_steps is not None else (100 if elastic else 200)
    preroll = args.preroll if args.preroll is not None else (0 if elastic else 60)
    run = {"iters": 0, "sweeps": 0, "steps": 0, "ms": 0.0}

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def advance(solver, n, tally=None):
        """n untimed steps, device time and Krylov counts added to tally."""
        if n <= 0:
            return
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(n):
            info = solver.hdg_step(dt, scheme, 1)
            if tally is not None:
                tally["iters"] += info["iterations"]
                tally["sweeps"] += info["sweeps"]
        b.record(stream)
        b.synchronize()
        if tally is not None:
            tally["steps"] += n
            tally["ms"] += a.elapsed_time(b)

    # pre-roll to the source's peak (t0 = 0.12 at 60 steps of 2e-3), so that the timed window lies
    # in the wave-propagation phase of the run rather than in the quiet start from rest; then the
    # warm-up (the condensation for alpha = 3/(2 dt) happens in the first step)
    advance(s, preroll, run)
    advance(s, args.warmup, run)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    s.hdg_get_stats(reset=True)
    ev0, ev1 = ev(), ev()
    ev0.record(stream)
    iters = 0
    sweeps = 0
    for _ in range(args.steps):
        info = s.hdg_step(dt, scheme, 1)
        iters += info["iterations"]
        sweeps += info["sweeps"]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    st_timed = s.hdg_get_stats(reset=True)
    launches_timed = st_timed["kernel_launches"]
    run["iters"] += iters
    run["sweeps"] += sweeps
    run["steps"] += args.steps
    run["ms"] += ms
    ms_max = max_over_ranks(dist, ms, "cuda")
    value = world * dofs * args.steps / (ms_max / 1e3)
    window = {"first_step": preroll + args.warmup + 1, "last_step": preroll + args.warmup + args.steps,
              "t_start": (preroll + args.warmup) * dt, "t_end": (preroll + args.warmup + args.steps) * dt}

    # per-launch kernel durations for the roofline: the same number of steps again, each launch of
    # the trace applies bracketed by CUDA events on the context stream (the timed window above
    # runs without these events)
    s.hdg_enable_stats(True)
    s.hdg_get_stats(reset=True)
    a_i, b_i = ev(), ev()
    a_i.record(stream)
    for _ in range(args.steps):
        info = s.hdg_step(dt, scheme, 1)
        run["iters"] += info["iterations"]
        run["sweeps"] += info["sweeps"]
    b_i.record(stream)
    b_i.synchronize()
    run["steps"] += args.steps
    run["ms"] += a_i.elapsed_time(b_i)
    st = s.hdg_get_stats(reset=True)
    s.hdg_enable_stats(False)
    instrumented_ms_per_step = a_i.elapsed_time(b_i) / args.steps

    # end to end through the public API with host buffers: the state (u^n, u^{n-1}, lambda) goes
    # host -> device, one step, and u^{n+1}, u^n, lambda come back device -> host, every step
    # (the state calls copy straight between the page-locked host buffers and the context)
    u_h = torch.empty(s._fshape, dtype=torch.float64).pin_memory()
    up_h = torch.empty(s._fshape, dtype=torch.float64).pin_memory()
    l_h = torch.empty(s._tshape, dtype=torch.float64).pin_memory()
    _, _, _, t_now = s.hdg_get_state(u=u_h, uprev=up_h, lam=l_h, want_prev=True)
    torch.cuda.synchronize()
    barrier()
    e2e_steps = max(1, min(args.steps, 10 if R == 1 else 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.hdg_set_state(u_h, t_now, uprev=up_h, lam=l_h)
        info = s.hdg_step(dt, scheme, 1)
        run["iters"] += info["iterations"]
        run["sweeps"] += info["sweeps"]
        _, _, _, t_now = s.hdg_get_state(u=u_h, uprev=up_h, lam=l_h, want_prev=True)
    e2e_s = time.perf_counter() - t0
    run["steps"] += e2e_steps
    e2e_value = world * dofs * e2e_steps / max_over_ranks(dist, e2e_s, "cuda")
    field_bytes = int(np.prod(s._fshape)) * 8
    trace_bytes = int(np.prod(s._tshape)) * 8
    nschur, nslot = s.sizes.schur_entries, s.sizes.slot_entries
    # the rest of the configured run (Krylov counts over every step of it)
    advance(s, total - run["steps"], run)
    full_run = {"steps": run["steps"], "krylov_iters_per_step": run["iters"] / max(1, run["steps"]),
                "refinement_sweeps_per_step": run["sweeps"] / max(1, run["steps"]) if args.prec != "fp64" else None,
                "device_ms_excluding_e2e_steps": run["ms"],
                "dof_steps_per_s_excluding_e2e_steps": dofs * (run["steps"] - e2e_steps) / (run["ms"] / 1e3)
                if run["ms"] > 0 else None}

    # roofline of the dominant kernel (matrix-free trace apply). Algorithmic bytes of one apply
    # y = sum_K P_K^T S_K P_K x: every element's packed symmetric S_K at the operator's
    # precision (plus its scale for FP16), x read once per interior trace entry and y written once.
    peaks, src = load_peaks()
    m = s.m
    P = m * (m + 1) // 2
    n_int = (s.n_faces - s.n_bnd) * s.Nf if not vardeg else None

    def alg_bytes(s_bytes, scale_bytes, vec_bytes, cols=1):
        return ne * (P * s_bytes + scale_bytes) + 2 * n_int * cols * vec_bytes

    def hbm_line(kernel, byt, launch_ms, launches, extra=None):
        ach = byt / (launch_ms / 1e3) / 1e9 if launch_ms > 0 else None
        d = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
             "frac": ach / peaks["hbm_gbs"] if ach else None, "traffic": None, "kernel": kernel,
             "peak_source": src + " hbm_gbs (copy)", "bytes_per_launch": byt, "bytes_per_elem": byt / ne,
             "launch_ms": launch_ms, "launches": launches}
        if extra:
            d.update(extra)
        return d

    def dev_or_event(st_t, st_i, key):
        """Mean launch duration of the FP32/FP16 apply: from the kernels' own device timers over
        the uninstrumented timed window (the launches inside the solve graphs) when they ran there,
        else from the CUDA events of the instrumented window; both figures are reported."""
        ev_ms = st_i[key + "_ms"] / max(1, st_i[key + "_launches"])
        extra = {"event_launch_ms": ev_ms if st_i[key + "_launches"] else None,
                 "event_launches": st_i[key + "_launches"]}
        if st_i.get("dev_" + key + "_launches"):
            extra["device_timer_launch_ms_same_launches"] = st_i["dev_" + key + "_ms"] / st_i["dev_" + key + "_launches"]
        if st_t.get("dev_" + key + "_launches"):
            n = st_t["dev_" + key + "_launches"]
            extra["launch_ms_source"] = ("%globaltimer stamps taken by the kernel (first CTA start to last CTA end), "
                                         "mean over the launches of the timed window")
            return st_t["dev_" + key + "_ms"] / n, n, extra
        extra["launch_ms_source"] = "CUDA events around each launch on the context stream (instrumented window)"
        return ev_ms, st_i[key + "_launches"], extra

    apply_avg_ms = st["apply_ms"] / max(1, st["apply_launches"])
    if R > 1:
        if args.prec != "fp64":
            a32 = st["apply32_ms"] / max(1, st["apply32_launches"])
            if R in (32, 64):
                kname = ("apply_tc_pq_kernel<3,3,%d> (S_K x the %d-column trace block on the tensor cores, TF32 "
                         "mma.sync with split X; p.q and alpha in its epilogue)" % (R, R))
            elif R > 64:
                kname = "apply_tc_kernel<3,3,64> (S_K x the %d-column trace block on the tensor cores)" % R
            else:
                kname = "apply_multi_kernel<3,3,float> (FP32 packed S_K, %d columns)" % R
            roof_multi = hbm_line(kname, alg_bytes(4, 0, 4, R), a32,
                                  st["apply32_launches"],
                                  {"implementation_bytes_per_elem": ((P + 3) // 4) * 16 + 2 * m * R * 4,
                                   "flops_per_elem": 2 * m * m * R})
        else:
            roof_multi = hbm_line("apply_multi_kernel<3,3,double> (%d columns)" % R, ne * m * m * 8 + 2 * n_int * R * 8,
                                  apply_avg_ms, st["apply_launches"], {"flops_per_elem": 2 * m * m * R})
    fp64_view = {"kernel": "apply_kernel<3,3> (FP64 S_K x lambda_K)", "launches": st["apply_launches"],
                 "launch_ms": apply_avg_ms,
                 "achieved_tflops": 2 * m * m * ne / (apply_avg_ms / 1e3) / 1e12 if st["apply_launches"] else None}
    if vardeg:
        roof = {}   # set below from the compact per-element-degree blocks
    elif args.prec == "fp64":
        ach = fp64_view["achieved_tflops"]
        roof = {"bound": "alu", "achieved": ach, "peak": 1.25, "unit": "TFLOP/s", "frac": ach / 1.25,
                "traffic": None, "kernel": fp64_view["kernel"],
                "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (probe measured 1.20)",
                "flops_per_elem": 2 * m * m, "launch_ms": apply_avg_ms, "launches": st["apply_launches"]}
    else:
        a32, n32, t32 = dev_or_event(st_timed, st, "apply32")
        roof = hbm_line("apply32_kernel<3,3> (FP32 packed-symmetric S_K x lambda_K)", alg_bytes(4, 0, 4) if n_int else 0,
                        a32, n32, t32)
        if st.get("apply16_launches"):
            a16, n16, t16 = dev_or_event(st_timed, st, "apply16")
            fp32_view = {k: roof[k] for k in ("kernel", "bytes_per_launch", "launch_ms", "launches", "achieved")}
            t16.update({"implementation_bytes_per_elem": ((P + 7) // 8) * 16 + 4 + 2 * m * 4,
                        "fp32_apply": fp32_view})
            roof = hbm_line("apply16_kernel<3,3> (FP16 packed-symmetric S_K, per-element FP32 scale)",
                            alg_bytes(2, 4, 4), a16, n16, t16)
            tr = MEASURED_TRAFFIC.get(("apply16_kernel<3,3>", ne))
            if tr:
                roof["traffic"] = tr[0]
                roof["traffic_source"] = tr[1]
        if st.get("applydf_launches"):
            adf = st["applydf_ms"] / st["applydf_launches"]
            byt = alg_bytes(8, 0, 8)
            roof["df_refinement_apply"] = {
                "kernel": "apply_df_kernel<3,3> (double-float hi + lo packed S_K)", "launches": st["applydf_launches"],
                "launch_ms": adf, "bytes_per_launch": byt, "achieved_gbs": byt / (adf / 1e3) / 1e9,
                "frac": byt / (adf / 1e3) / 1e9 / peaks["hbm_gbs"]}
        roof["fp64_refinement_apply"] = fp64_view
    # element-local post-processing of the final state into P_{k+1}, timed on its own (outside
    # the steps' timed region); FP64-ALU bound, algorithmic flops per element as counted here
    post = None
    if args.postprocess and not elastic and R == 1:
        u_f, lam_f, _ = s.hdg_get_state()
        ps = s.hdg_postprocess(u_f, lam_f)
        for _ in range(2):
            s.hdg_postprocess(u_f, lam_f, ps)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(5):
            s.hdg_postprocess(u_f, lam_f, ps)
        ev1.record(stream)
        ev1.synchronize()
        pm = ev0.elapsed_time(ev1) / 5
        d, Np, Nf = s.dim, s.Np, s.Nf
        na = math.comb(s.k + 1 + d, d) - 1
        fl = (2 * d * Np * (d * Np + (d + 1) * Nf) + 2 * na * d * d * Np + d * d * na * (na + 1)
              + na ** 3 / 3 + 2 * na * na)
        ach_p = fl * ne / (pm / 1e3) / 1e12
        post = {"kernel": "post_kernel<%d,%d> (p* in P_%d: discrete gradient, local Neumann problem, Cholesky)"
                % (d, s.k, s.k + 1), "launch_ms": pm, "flops_per_elem": fl, "achieved_tflops": ach_p,
                "peak_tflops": 1.25, "frac": ach_p / 1.25, "peak_source": "nominal GB300 FP64",
                "bytes_per_elem": (Np + (d + 1) * Nf + 32 + na + 1) * 8}
        del ps, u_f, lam_f

    # the plain FP64 GPU path on the same workload and steps, for the mixed-vs-FP64 comparison
    fp64 = None
    tiles = s.hdg_get_tuning() if vardeg else None
    if args.prec != "fp64" and not args.no_fp64_compare:
        u_mixed = s.hdg_get_state()[0]
        tiles = s.hdg_get_tuning() if vardeg else None
        s.close()
        torch.cuda.empty_cache()
        s64 = make_solver("fp64")
        advance(s64, preroll + args.warmup)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            s64.hdg_step(dt, scheme, 1)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms64 = ev0.elapsed_time(ev1)
        # the rest of the same run from the same start, to the same final step as the mixed run
        advance(s64, run["steps"] - preroll - args.warmup - args.steps)
        u64 = s64.hdg_get_state()[0]
        rel = float((u_mixed - u64).abs().max() / u64.abs().max().clamp_min(1e-300))
        fp64 = {"value": dofs * args.steps / (ms64 / 1e3), "ms_per_step": ms64 / args.steps,
                "speedup_mixed_over_fp64": ms64 / ms_max,
                "max_rel_diff_fields_after_%d_steps" % run["steps"]: rel}
        s64.close()

    if R > 1:
        roof = roof_multi
    if vardeg:
        # per launch: every compact S_K (FP32, or FP64 for the plain path), the trace gather and
        # the slot products
        if args.prec != "fp64":
            f16 = st.get("apply16_launches", 0) > 0
            a32 = (st["apply16_ms"] / st["apply16_launches"]) if f16 else \
                st["apply32_ms"] / max(1, st["apply32_launches"])
            byt = (nschur * 2 + ne * 4 if f16 else nschur * 4) + 2 * nslot * 4
            ach = byt / (a32 / 1e3) / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": None,
                    "kernel": ("apply_vd_kernel<float, __half> (compact FP16 S_K, per-element scale)" if f16 else
                               "apply_vd_kernel<float> (compact FP32 S_K, per-element m_K)"),
                    "peak_source": src + " (hbm_gbs: copy)",
                    "bytes_per_launch": byt, "launch_ms": a32,
                    "launches": st["apply16_launches"] if f16 else st["apply32_launches"],
                    "fp64_refinement_apply": {"launch_ms": apply_avg_ms, "launches": st["apply_launches"],
                                              "achieved_tflops": 2 * nschur / (apply_avg_ms / 1e3) / 1e12
                                              if st["apply_launches"] else None}}
            if st.get("applydf_launches"):
                adf = st["applydf_ms"] / st["applydf_launches"]
                roof["df_refinement_apply"] = {
                    "kernel": "apply_vd_df_kernel (double-float hi + lo compact S_K)", "launches": st["applydf_launches"],
                    "launch_ms": adf, "bytes_per_launch": nschur * 8 + nslot * 16,
                    "achieved_gbs": (nschur * 8 + nslot * 16) / (adf / 1e3) / 1e9}
        else:
            ach = 2 * nschur / (apply_avg_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": 1.25, "unit": "TFLOP/s", "frac": ach / 1.25,
                    "traffic": None, "kernel": "apply_vd_kernel<double> (compact FP64 S_K)",
                    "peak_source": "nominal GB300 FP64 1.25 TFLOP/s", "flops_per_launch": 2 * nschur,
                    "launch_ms": apply_avg_ms, "launches": st["apply_launches"]}
    elif elastic and args.prec != "fp64":
        a32 = st["apply32_ms"] / max(1, st["apply32_launches"])
        bytes_el = m * m * 4 + 2 * m * 4
        ach = bytes_el * ne / (a32 / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                "traffic": None, "kernel": "apply32f_kernel<ElDims<3,%d>> (FP32 S_K %dx%d)" % (args.k, m, m),
                "bytes_per_elem": bytes_el, "launch_ms": a32, "launches": st["apply32_launches"],
                "fp64_refinement_apply": fp64_view}

    if str(roof.get("launch_ms_source", "")).startswith("%globaltimer"):
        roof["timing"] = ("launch_ms: the kernel's own %%globaltimer stamps over the launches of the timed window "
                          "(inside the solve graphs); event_launch_ms: CUDA events around every launch on the context "
                          "stream during %d instrumented steps that follow the timed window (%.3f ms/step with the "
                          "events, host-driven loops)" % (args.steps, instrumented_ms_per_step))
    else:
        roof["timing"] = ("CUDA events around every launch on the context stream during %d instrumented steps that "
                          "follow the timed window (%.3f ms/step with the events); the timed window runs without them"
                          % (args.steps, instrumented_ms_per_step))
    # bounded serving leg (the serve p50/p99 half of the metric): the first requests of the
    # Poisson(20/s) serving workload through the continuous-batching server, after the solver
    # above has released its memory
    serve = None
    if args.serve_leg > 0 and not elastic and R == 1:
        from paper_1807_00086_gb300.serve import Server, serving_workload
        try:
            s.close()
        except Exception:
            pass
        torch.cuda.empty_cache()
        reqs = serving_workload(n_req=args.serve_leg, rate=args.serve_rate)
        srv = Server(budget_bytes=int(args.serve_budget_gb * (1 << 30)), R=args.serve_slots, prec="mixed")
        st_srv = srv.run(reqs)
        srv.close()
        serve = {"requests": st_srv["requests"], "arrival_rate_per_s": args.serve_rate, "p50_ms": st_srv["p50_ms"],
                 "p99_ms": st_srv["p99_ms"], "mean_ms": st_srv["mean_ms"], "dof_steps_per_s": st_srv["dof_steps_per_s"],
                 "wait_p50_ms": st_srv["wait_p50_ms"], "wait_p99_ms": st_srv["wait_p99_ms"],
                 "service_p50_ms": st_srv["service_p50_ms"], "service_p99_ms": st_srv["service_p99_ms"],
                 "wall_s": st_srv["wall_s"], "slots_per_context": args.serve_slots,
                 "contexts": st_srv["contexts_created"],
                 "workload": "first %d requests of the seeded serving workload (2D/3D acoustic, 1e3-1e5 elements, "
                             "k in 1..4, 20-200 BDF2 steps)" % args.serve_leg}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_sample(budget_s=args.cpu_budget)
        cpu = {k: r[k] for k in ("value", "unit", "cores", "host_cores", "kind", "sample")}
        if not args.no_all_cores:
            cpu["all_cores"] = oracle_all_cores(args.cpu_budget)
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32+f64", "mixed16": "f16+f32+f64"}[args.prec],
               "data": "synthetic",
               "config": {"workload": ("elastic3d_k%s_%dcube_dirk3" % ("mix1to4" if vardeg else args.k,
                                                                    round((ne / 6) ** (1 / 3))) if elastic else
                                       "acoustic3d_k3_32cube_bdf2" + ("_%dsrc" % R if R > 1 else "") +
                                       ("_" + args.trace_space if args.trace_space != "hdg" else "")), "n_elem": ne,
                          "k": "U{1..4} per element" if vardeg else args.k, "dofs": dofs, "nrhs": R,
                          "trace_dofs": int(s.sizes.trace_entries) * R, "dt": dt, "scheme": scheme.upper(),
                          "precision": args.prec, "rtol": args.rtol, "parallelism": "replicas",
                          "l2": "inputs larger than L2 (S_K %.2f GB)" % (nschur * 8 / 1e9),
                          "timed_window": window, "preroll_steps": preroll,
                          "krylov_iters_per_step": iters / args.steps,
                          "refinement_sweeps_per_step": sweeps / args.steps if args.prec != "fp64" else None,
                          "inner_rtol": args.inner_rtol if args.prec != "fp64" else None,
                          "guess_history": args.guess_history if R == 1 else None,
                          "trace_space": args.trace_space, "solver": args.solver,
                          "precond": args.precond if args.solver == "gmres" else "jacobi",
                          "trace_unknowns": int(s.sizes.trace_unknowns) * R,
                          "trace_solve": "host-driven loops" if (args.host_loops or R > 1) else
                          "one CUDA-graph launch per trace solve (device-side loop conditions)"},
               "roofline": roof, "cpu_baseline": cpu, "fp64_gpu": fp64,
               "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * field_bytes + trace_bytes,
                       "d2h_bytes_per_step": 2 * field_bytes + trace_bytes, "steps": e2e_steps},
               "gpu_launches": launches_timed, "clocks": clk, "full_run": full_run}
        if post is not None:
            out["postprocess"] = post
        if serve is not None:
            out["serve"] = serve
        if vardeg:
            out["config"]["autotuned_tiles"] = tiles
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def svk_condense_flops(k):
    """FP64 flops of one element of svk_condense_kernel<k> (an FMA counts 2): the residual on the
    (2k+2)^3 rule, the deformation gradient on the (2k+1)^3 rule, per Jacobian point the tangent
    and the three outer-product accumulations (Dx T Dx^T upper triangle, Dx T BH, BH^T T BH
    upper triangle) with their per-point precomputes, the Cholesky of S_v, Z = L^{-1} W, Z^T Z
    and the two tangent applies."""
    NP = (k + 1) * (k + 2) * (k + 3) // 6
    NFP = (k + 1) * (k + 2) // 2
    NV, M, N = 3 * NP, 12 * NFP, 21 * NP
    NQR, NQJ = (2 * k + 2) ** 3, (2 * k + 1) ** 3
    ea, eb, ec = NV * (NV + 1) // 2, NV * M, M * (M + 1) // 2
    per_point = 3 * (60 + 81 * 8 + 3 * NP * 6 + 4 * NFP)           # stress, tangent, g_J, psi per pass
    per_point += 27 * NP * 6 + ea * 8                                  # (a)
    per_point += 108 * 6 + 36 * NP * 6 + eb * 4                        # (b)
    per_point += 144 * 18 + ec * 5                                     # (c)
    f = NQJ * per_point
    f += NQR * (18 * NP + 80) + 9 * NP * NQR * 2 + NQJ * 9 * NP * 2    # residual, F at the Jacobian points
    f += NV ** 3 // 3 + NV * NV * M + ec * NV * 2                      # Cholesky, Z, Z^T Z
    f += 2 * NQJ * (9 * NP * 4 + 81 * 2 + 700)                         # two tangent applies
    f += N * (4 * (NP + NFP) * 2 + 6 * NP)                             # volume / face terms of R
    return f


def run_svk(args):
    """Nonlinear SVK elastodynamics (Sec. 4.4-4.5): free large-amplitude vibration of the clamped
    plate (n x n x 1 cubes of 6 tets, one element through the 0.01 thickness, traction-free top
    and bottom, clamped sides), DIRK3 with a Newton solve per stage, each Newton iteration
    condensing every element with its tangent at the quadrature points. Initial state: the
    plate solution's velocity 0.4 pi sin(pi x) sin(pi y) e_z, F = I, P = 0."""
    import torch
    from paper_1807_00086_gb300 import hdg, inputs
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.N
    k = args.k
    dt = 2e-3
    vert, elem = inputs.plate_tet(n)
    ne = elem.shape[0]

    prec = args.prec if args.prec in ("fp64", "mixed") else "mixed"

    def make(prec=prec):
        sv = hdg.Solver(vert, elem, k, 1.0, np.ones(ne), lam=np.full(ne, 1.5), mu=np.ones(ne), svk=True, rtol=1e-10,
                        prec=prec)
        zb = sv.hdg_quadrature_points(1)[:, :, 2]
        sv.hdg_svk_set_traction_faces(np.all(np.abs(zb - 0.01) < 1e-13, axis=1) | np.all(np.abs(zb) < 1e-13, axis=1))
        xv = sv.hdg_quadrature_points(0)
        vals = np.zeros(xv.shape[:2] + (21,))
        vals[:, :, 2] = 0.4 * np.pi * np.sin(np.pi * xv[:, :, 0]) * np.sin(np.pi * xv[:, :, 1])
        sv.hdg_set_state(sv.hdg_project_volume(vals), 0.0)
        return sv

    s = make()
    dofs = ne * s.n
    stream = s.stream
    for _ in range(args.warmup):
        s.hdg_step(dt, "dirk3", 1)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    s.hdg_get_stats(reset=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    newton, cg = 0, 0
    a.record(stream)
    for _ in range(args.steps):
        info = s.hdg_step(dt, "dirk3", 1)
        newton += info["sweeps"]
        cg += info["iterations"]
    b.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = a.elapsed_time(b)
    launches = s.hdg_get_stats(reset=True)["kernel_launches"]
    ms_max = max_over_ranks(dist, ms, "cuda")
    value = world * dofs * args.steps / (ms_max / 1e3)
    # kernel times: one more step with CUDA events around every condensation and recovery
    s.hdg_enable_stats(True)
    s.hdg_get_stats(reset=True)
    s.hdg_step(dt, "dirk3", 1)
    st = s.hdg_get_stats(reset=True)
    s.hdg_enable_stats(False)
    cms = st["svk_condense_ms"] / max(1, st["svk_condense_launches"])
    rms = st["svk_recover_ms"] / max(1, st["svk_recover_launches"])
    fl = svk_condense_flops(k) * ne
    ach = fl / (cms / 1e3) / 1e12
    peak, psrc = ((1.25, "nominal GB300 FP64 1.25 TFLOP/s (the FP64 pipe; no FP64 tensor path is used)")
                  if prec == "fp64" else
                  (80.5, "GB300 FP32 CUDA cores: 152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s (the "
                         "Jacobian arithmetic; the FP64 residual is a few percent of the flops)"))
    roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
            "kernel": "svk_condense_kernel<%d, %s> (FP64 residual; tangent at (2k+1)^3 points and condensation in %s)"
                      % (k, "double" if prec == "fp64" else "float", "FP64" if prec == "fp64" else "FP32"),
            "peak_source": psrc,
            "flops_per_elem": svk_condense_flops(k), "launch_ms": cms, "launches": st["svk_condense_launches"],
            "timing": "CUDA events around every launch during one instrumented step after the timed window",
            "recover_kernel": {"kernel": "svk_recover_kernel<%d>" % k, "launch_ms": rms,
                               "launches": st["svk_recover_launches"]}}
    # end to end through the public API with host buffers: fields and traces in, one step, out
    u_h = torch.empty(s._fshape, dtype=torch.float64).pin_memory()
    l_h = torch.empty(s._tshape, dtype=torch.float64).pin_memory()
    _, _, t_now = s.hdg_get_state(u=u_h, lam=l_h)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.hdg_set_state(u_h, t_now, lam=l_h)
        s.hdg_step(dt, "dirk3", 1)
        _, _, t_now = s.hdg_get_state(u=u_h, lam=l_h)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * dofs * e2e_steps / max_over_ranks(dist, e2e_s, "cuda")
    fb, tb = int(np.prod(s._fshape)) * 8, int(np.prod(s._tshape)) * 8
    trace_dofs, schur_entries = s.sizes.trace_entries, s.sizes.schur_entries
    # the FP64 form on the same trajectory: warm-up + timed steps from the same initial state,
    # its rate and the largest field difference after them
    fp64 = None
    if prec != "fp64" and not args.no_fp64_compare:
        u_m, _, _ = s.hdg_get_state()
        s.close()
        torch.cuda.empty_cache()
        ref = make("fp64")
        mix = make(prec)
        nst = args.warmup + args.steps
        mix.hdg_step(dt, "dirk3", nst)
        ref.hdg_step(dt, "dirk3", args.warmup)
        torch.cuda.synchronize()
        a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a2.record(ref.stream)
        ref.hdg_step(dt, "dirk3", args.steps)
        b2.record(ref.stream)
        torch.cuda.synchronize()
        ms64 = a2.elapsed_time(b2)
        u64, _, _ = ref.hdg_get_state()
        um, _, _ = mix.hdg_get_state()
        fp64 = {"value": dofs * args.steps / (ms64 / 1e3), "ms_per_step": ms64 / args.steps,
                "speedup_mixed_over_fp64": ms64 / ms,
                "max_rel_diff_fields_after_%d_steps" % nst: float((um - u64).abs().max() / u64.abs().max())}
        ref.close()
        mix.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import elastic_svk as nl
        vs, es = inputs.plate_tet(2)

        def tb_face(Y):
            z = Y[:, 2]
            return bool(np.all(np.abs(z - z[0]) < 1e-14) and (abs(z[0]) < 1e-14 or abs(z[0] - 0.01) < 1e-14))
        prob = nl.build_problem(vs, es, k, 1.0, 1.5, 1.0, neumann_face=tb_face)

        def v0(x, t):
            v = np.zeros((x.shape[0], 3))
            v[:, 2] = 0.4 * np.pi * np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])
            return v
        u0 = nl.project(prob, v0, lambda x, t: np.zeros((x.shape[0], 9)), lambda x, t: np.zeros((x.shape[0], 9)), 0.0)
        t0 = time.perf_counter()
        nst = 0
        while nst < 1 or time.perf_counter() - t0 < min(args.cpu_budget, 20.0):
            u0, _, _ = nl.run_dirk3(prob, u0 + 0.0, dt, 1)
            nst += 1
        el = time.perf_counter() - t0
        cpu = {"value": es.shape[0] * 21 * prob.Np * nst / el, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
               "kind": "oracle",
               "sample": "%d DIRK3 steps of the SVK plate on a 2x2x1 = %d-tet plate (k=%d, %d field DOFs); oracle = "
                         "numpy/scipy FP64, per-element LU of the 21 N_p Newton system + sparse direct trace solve"
                         % (nst, es.shape[0], k, es.shape[0] * 21 * prob.Np)}
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32+f64",
               "data": "synthetic",
               "config": {"workload": "svk3d_plate_k%d_%dx%dx1_dirk3" % (k, n, n), "n_elem": ne, "k": k, "dofs": dofs,
                          "trace_dofs": int(trace_dofs), "dt": dt, "scheme": "DIRK3",
                          "precision": prec + (" (FP32 Jacobian, FP64 residual)" if prec != "fp64" else ""),
                          "newton_tol": 1e-11, "cg_rtol": 1e-10, "parallelism": "replicas",
                          "newton_iters_per_stage": newton / (3 * args.steps),
                          "cg_iters_per_newton": cg / max(1, newton),
                          "l2": "inputs larger than L2 (S_K %.2f GB)" % (schur_entries * 8 / 1e9)},
               "roofline": roof, "cpu_baseline": cpu, "fp64_gpu": fp64,
               "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": fb + tb, "d2h_bytes_per_step": fb + tb,
                       "steps": e2e_steps},
               "gpu_launches": launches, "clocks": clk}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_apply_only(args):
    """Profiling driver: condense the workload at size N and run `steps` trace applies."""
    import torch
    from paper_1807_00086_gb300 import hdg, inputs
    w = inputs.acoustic_3d_workload(N=args.N, k=args.k)
    s = hdg.Solver(w["vert"], w["elem"], w["k"], w["tau"], w["rho"], w["c"], prec=args.prec)
    s.hdg_condense(1.5 / DT)
    x = torch.tensor(inputs.random_traces(s.n_faces, s.Nf, 1), device="cuda")
    for _ in range(args.steps):
        y = s.hdg_trace_apply(x)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "apply", "n_elem": s.n_elem, "applies": args.steps, "max_abs": float(y.abs().max())}))


def run_serve(args):
    """Serving workload: Poisson arrivals (20/s), 2D/3D acoustic requests of mixed mesh size,
    degree and step count, continuous batching under a device-memory budget."""
    import torch
    from paper_1807_00086_gb300.serve import Server, serving_workload
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    reqs = serving_workload(n_req=args.serve_requests, rate=args.serve_rate)
    srv = Server(budget_bytes=int(args.serve_budget_gb * (1 << 30)), R=args.serve_slots, prec=args.prec)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    stats = srv.run(reqs)
    clk = clocks.stop()
    srv.close()
    out = {"metric": METRIC, "mode": "serve", "value": stats["dof_steps_per_s"], "unit": UNIT,
           "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"], "mean_ms": stats["mean_ms"],
           "wait_p50_ms": stats["wait_p50_ms"], "wait_p99_ms": stats["wait_p99_ms"],
           "service_p50_ms": stats["service_p50_ms"], "service_p99_ms": stats["service_p99_ms"],
           "higher_is_better": True, "dtype": {"fp64": "f64", "mixed": "f32+f64", "mixed16": "f16+f32+f64"}[args.prec], "data": "synthetic",
           "config": {"workload": "serve_acoustic_2d3d_poisson%g" % args.serve_rate, "requests": stats["requests"],
                      "slots_per_context": args.serve_slots, "budget_gb": args.serve_budget_gb,
                      "contexts_resident_at_end": stats["contexts_created"], "wall_s": stats["wall_s"],
                      "precision": args.prec},
           "clocks": clk}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default=None, choices=["fp64", "mixed", "mixed16"],
                    help="default: mixed16 for the single-source acoustic and the mixed-degree elastic workloads, "
                         "else mixed")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the plain FP64 comparison run that follows a mixed-precision measurement")
    ap.add_argument("--rtol", type=float, default=1e-12)
    ap.add_argument("--inner-rtol", type=float, default=None,
                    help="default: 1e-3 (FP16 operator: its rounding bounds a sweep near 4e-4), "
                         "3e-6 (FP32 operator, one right-hand side), 1e-4 (FP32, many)")
    ap.add_argument("--N", type=int, default=32)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--physics", default="acoustic", choices=["acoustic", "elastic", "svk"],
                    help="elastic: the 3D linear elastodynamics workload (24^3 x 6 tets, DIRK3); svk: nonlinear "
                         "elastodynamics, free vibration of the clamped plate (--N x --N x 1 cubes, k = --k)")
    ap.add_argument("--guess-history", type=int, default=8,
                    help="earlier stage solutions spanning the least-squares initial guess (0: extrapolation)")
    ap.add_argument("--mixed-degree", action="store_true",
                    help="elastic: per-element degree uniform in {1..4} (the mixed-degree workload)")
    ap.add_argument("--nrhs", type=int, default=1,
                    help="right-hand-side columns solved together (64: the multi-source workload)")
    ap.add_argument("--preroll", type=int, default=None,
                    help="untimed steps before the warm-up (default: 60 for the acoustic workloads, i.e. to the "
                         "Ricker source's peak at t0 = 0.12; 0 for elastic)")
    ap.add_argument("--total-steps", type=int, default=None,
                    help="steps of the whole run whose Krylov counts are reported (default: 200 acoustic, 100 elastic)")
    ap.add_argument("--solver", default="cg", choices=["cg", "gmres"],
                    help="gmres: restarted GMRES with two-pass classical Gram-Schmidt (FP64, the paper's Krylov method)")
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "bilu0"],
                    help="with --solver gmres: right preconditioner, Jacobi or block ILU(0) (the paper's)")
    ap.add_argument("--trace-space", default="hdg", choices=["hdg", "iedg", "edg"],
                    help="acoustic, one column: continuous traces on the interior (iedg) or all (edg) faces")
    ap.add_argument("--host-loops", action="store_true",
                    help="host-driven Krylov and refinement loops (polled) instead of one graph launch per trace solve")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-all-cores", action="store_true",
                    help="skip the all-cores oracle timing (one oracle process per host core)")
    ap.add_argument("--postprocess", action="store_true",
                    help="acoustic, one column: also time the local post-processing into P_{k+1} on the final "
                         "state (outside the steps' timed region; reported under \"postprocess\")")
    ap.add_argument("--mode", default="step", choices=["step", "apply"],
                    help="apply: profiling driver that only condenses and applies K (no JSON bench line)")
    ap.add_argument("--serve", action="store_true", help="run the continuous-batching serving workload")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-leg", type=int, default=100,
                    help="requests of the serving workload run after the step benchmark (0: none)")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    args = ap.parse_args()
    if args.prec is None:
        args.prec = "mixed16" if ((args.physics == "acoustic" and args.nrhs == 1 and not args.serve) or
                                  (args.physics == "elastic" and args.mixed_degree)) else "mixed"
    if args.inner_rtol is None:
        args.inner_rtol = 1e-3 if args.prec == "mixed16" else (1e-4 if args.nrhs > 1 else 3e-6)
    if args.physics == "svk":
        if args.N == 32 and "--N" not in sys.argv:
            args.N = 16
        if args.k == 3 and "--k" not in sys.argv:
            args.k = 2
        run_svk(args)
    elif args.serve:
        run_serve(args)
    elif args.mode == "apply":
        run_apply_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
