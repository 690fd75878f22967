#!/usr/bin/env python3
"""Benchmark of the MPLP++ Handshake solver on one GB300.

Workload (default): the pose-shaped dense model -- complete graph K_60, 300
labels per node, truncated-quadratic distance costs, 500 iterations of the
round-robin schedule (59 matchings of 30 edges).  One step = reset the
reparametrization, run all 500 iterations, compute the exact dual bound and
the primal rounding with its energy: every row of the hot path.

Reported: edge updates/s (whole job), the persistent Handshake kernel's
algorithmic HBM GB/s against the measured copy bandwidth, the same workload
through the looped (one launch per matching) driver at equal final bound,
the end-to-end rate through the public API with host buffers, and the FP64
oracle on the host cores.  Multi-GPU runs (torchrun) are replicas: every rank
solves its own seeded copy (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

CONFIGS = {
    1: ("K20_L8_uniform_T200", 200),
    2: ("pose_K60_L300_T500", 500),
    3: ("knn_n2000_k50_L64_T300", 300),
    4: ("batch256_K10-80_L16-128_T100", 100),
    5: ("batch16_K50_L64_T50", 50),
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def models_for(cfg: int, seed: int, count: int = 0):
    """The models of a configuration; count > 0 with configuration 4: that
    many models of the batch recipe instead of 256 (a smaller case of the
    same kernel, for profiling); with configuration 1: that many seeded
    replicas of the K_20 model solved together."""
    from paper_2004_08227_gb300 import workloads as W
    if cfg == 4 and count > 0:
        return W.batch(count, seed=seed), CONFIGS[4][1]
    if cfg == 1 and count > 0:
        return [W.config(1, seed=seed * count + k)[0] for k in range(count)], CONFIGS[1][1]
    models, T = W.config(cfg, seed=seed)
    if not isinstance(models, list):
        models = [models]
    return models, T


def algorithmic_bytes(models):
    """Algorithmic HBM bytes of one iteration: per edge update the FP32 table
    read once (4 L_u L_v) and the FP32 node vectors and messages of both ends
    read and written (16 (L_u + L_v))."""
    total = 0
    for m in models:
        L = np.asarray(m.labels, np.int64)
        Lu, Lv = L[np.asarray(m.edge_u)], L[np.asarray(m.edge_v)]
        total += int(np.sum(4 * Lu * Lv + 16 * (Lu + Lv)))
    return total


def host_cpu():
    """CPU model and logical core count of the host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"model": model, "nproc": os.cpu_count()}


def kernel_traffic(iterations):
    """DRAM bytes per launch of the Handshake kernel from the committed ncu
    summary, scaled from its 500-iteration figure; None when the kernel
    sources changed since the capture (recorded SHA-1 of the sources)."""
    import hashlib
    import re
    prof = os.path.join(ROOT, "profiles", "hs_persistent_kernel_pose_K60_L300.md")
    try:
        txt = open(prof).read()
        h = hashlib.sha1()
        for f in ("handshake.cu", "common.cuh"):
            h.update(open(os.path.join(ROOT, "paper_2004_08227_gb300", "csrc", f), "rb").read())
        if re.search(r"source_sha1: ([0-9a-f]+)", txt).group(1) != h.hexdigest():
            return None
        return float(re.search(r"dram_bytes_per_launch: ([0-9.]+)", txt).group(1)) * iterations / 500.0
    except Exception:
        return None


def load_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_rate(models, T_full, budget_s: float):
    """The FP64 oracle as it stands, single thread, on a bounded sample: the
    first model of the workload for as many iterations as fit the budget."""
    import oracle
    from oracle import schedule as osched
    m = models[0]
    order = osched.build(m.schedule, m.n, m.edge_u, m.edge_v)[1]
    t0 = time.perf_counter()
    st = oracle.run(m, order, 1)
    t1 = time.perf_counter() - t0
    iters = int(max(1, min(T_full - 1, budget_s / max(t1, 1e-9) - 1)))
    t0 = time.perf_counter()
    oracle.run(m, order, iters, state=st)
    dt = time.perf_counter() - t0
    total_iters = iters + 1
    rate = total_iters * m.E / (t1 + dt)
    return rate, {"value": rate, "unit": "edge_updates/s", "cores": 1, "kind": "oracle",
                  "sample": f"{m.name}: {total_iters} of {T_full} iterations, single-thread FP64 C oracle, "
                            f"{t1 + dt:.1f} s"}


def cpu_oracle_rate_parallel(models, T_full, budget_s: float):
    """The FP64 oracle with the edges of each matching updated on every host
    core (oracle.run_parallel: OpenMP, equal to the sequential oracle bit for
    bit) on a bounded sample: the first model for as many iterations as fit
    the budget."""
    import oracle
    from oracle import schedule as osched
    m = models[0]
    off, order = osched.build(m.schedule, m.n, m.edge_u, m.edge_v)
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    st = oracle.run_parallel(m, off, order, 1, threads=threads)
    t1 = time.perf_counter() - t0
    iters = int(max(1, min(T_full - 1, budget_s / max(t1, 1e-9) - 1)))
    t0 = time.perf_counter()
    oracle.run_parallel(m, off, order, iters, state=st, threads=threads)
    dt = time.perf_counter() - t0
    total_iters = iters + 1
    rate = total_iters * m.E / (t1 + dt)
    cpu = host_cpu()
    return rate, {"value": rate, "unit": "edge_updates/s", "cores": threads, "kind": "oracle",
                  "cpu": cpu["model"], "nproc": cpu["nproc"],
                  "sample": f"{m.name}: {total_iters} of {T_full} iterations, FP64 C oracle, edges of each "
                            f"matching on {threads} threads (OpenMP), {t1 + dt:.1f} s"}


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = args.config
    models, T = models_for(cfg, seed=0)
    import oracle
    from oracle import schedule as osched
    m = models[0]
    off, order = osched.build(m.schedule, m.n, m.edge_u, m.edge_v)
    threads = oracle.max_threads()
    st = None
    per = max(1, args.ref_iters)
    for _ in range(args.warmup):
        st = oracle.run_parallel(m, off, order, per, state=st, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st = oracle.run_parallel(m, off, order, per, state=st, threads=threads)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = per * m.E / (ms / 1e3)
    name = CONFIGS[cfg][0]
    cpu = host_cpu()
    line = {"impl": "reference", "metric": "edge_updates_per_s", "value": value, "unit": "edge_updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "sample": f"{per} iteration(s) of {m.name} per step"},
            "cpu_baseline": {"value": value, "unit": "edge_updates/s", "cores": threads, "kind": "oracle",
                             "cpu": cpu["model"], "nproc": cpu["nproc"],
                             "sample": f"{per} of {T} iterations of {m.name} per step, FP64 C oracle, edges of "
                                       f"each matching on {threads} threads (OpenMP)"},
            "e2e": {"value": value, "unit": "edge_updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(ms: float, world: int, device: str) -> float:
    """The slowest rank's time per step: the whole job ends when it does."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(updates_per_rank: float, world: int, ms: float) -> float:
    """Edge updates per second of the whole job: every rank solves its own
    replica (the same workload, its own seed), timed by the slowest rank."""
    return updates_per_rank * world / (ms / 1e3)


def _timed(stream, fn, n):
    import torch
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    out = None
    for _ in range(n):
        out = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / n, out


def looped_baseline(Solver, models, T, stream, step, D_ref, ms_ref, n):
    """The plain driver: one launch per matching.  One model: the same model
    looped; several models: a loop of per-model solves (each its own solver)."""
    if len(models) == 1:
        sl = Solver(models, mode="looped")
        step(sl)
        lms, D = _timed(stream, lambda: step(sl), n)
        launches = T * sl.info()["phases"]
        sl.close()
    else:
        solvers = [Solver([m], mode="looped") for m in models]

        def loop():
            return np.concatenate([step(s) for s in solvers])
        loop()
        lms, D = _timed(stream, loop, n)
        launches = T * sum(s.info()["phases"] for s in solvers)
        for s in solvers:
            s.close()
    return {"ms_per_step": lms, "launches_per_step": launches, "models": len(models),
            "final_bound_sum": float(np.sum(D)), "bound_equal": bool(np.array_equal(D, D_ref)),
            "persistent_speedup": lms / ms_ref}


def batched_vs_looped(Solver, stream, args):
    models, T = models_for(4, seed=0)
    s = Solver(models, mode="persistent")
    tune = s.autotune(2) if args.autotune > 0 else None
    info = s.info()

    def step_b(sol):
        sol.reset()
        sol.run(T)
        return sol.bound(exact=True)
    step_b(s)
    bms, D = _timed(stream, lambda: step_b(s), 2)
    s.close()
    lp = looped_baseline(Solver, models, T, stream, step_b, D, bms, 1)
    # the same batch through each persistent driver: one kernel launch per solve
    # (the fastest of a few block sizes per driver)
    persistent = {}
    for name, mode, sizes in (("cluster", "persistent", (128, 256, 512)), ("warp", "warp", (32, 64, 128)),
                              ("queue", "queue", (128,))):
        best = None
        for nt in sizes:
            try:
                sp = Solver(models, mode=mode, threads=nt, cluster=1)
            except Exception as e:  # a mapping the shapes do not admit
                best = best or {"unavailable": str(e)}
                continue
            step_b(sp)
            pms, Dp = _timed(stream, lambda: step_b(sp), 1)
            pin = sp.info()
            if best is None or "ms" not in best or pms < best["ms"]:
                best = {"ms": pms, "run_launches": 2, "bound_equal": bool(np.array_equal(Dp, D)),
                        "speedup_vs_per_model_loop": lp["ms_per_step"] / pms,
                        "mapping": {k: pin[k] for k in ("cluster", "threads", "grid")}}
            sp.close()
        persistent[name] = best
    upd = T * info["edges"]
    return {"workload": CONFIGS[4][0], "models": len(models), "edges": info["edges"], "iterations": T,
            "batched_ms": bms, "batched_edge_updates_per_s": upd / (bms / 1e3),
            "batched_gbs": T * algorithmic_bytes(models) / (bms / 1e3) / 1e9,
            "batched_frac_of_peak": T * algorithmic_bytes(models) / (bms / 1e3) / 1e9 / load_peak()[0],
            "batched_gbs_state32": T * info["bytes_per_iteration"] / (bms / 1e3) / 1e9,
            "per_model_looped_ms": lp["ms_per_step"], "per_model_launches": lp["launches_per_step"],
            "bound_equal": lp["bound_equal"], "speedup": lp["ms_per_step"] / bms,
            "mapping": {k: info[k] for k in ("mode", "cluster", "threads", "grid")},
            "autotune": tune.get("best") if tune else None, "persistent_drivers": persistent}


def replicas_study(Solver, stream, args, peak):
    """The K_20, L = 8 workload (200 iterations): one model, whose chain of 3,800
    dependent matchings of 10 small edges is latency-bound, and many seeded
    replicas solved together through the batched path (autotuned mapping), so
    that the Handshake kernel's HBM throughput shows."""
    from paper_2004_08227_gb300 import workloads as W
    T = 200
    rows = []
    for nrep in (1, args.replicas):
        models = [W.config(1, seed=k)[0] for k in range(nrep)]
        s = Solver(models)
        tune = s.autotune(2) if args.autotune > 0 else None

        def run(sol=s):
            sol.reset()
            sol.run(T)
        run()
        ms, _ = _timed(stream, run, 2)
        inf = s.info()
        gbs = T * algorithmic_bytes(models) / (ms / 1e3) / 1e9
        rows.append({"models": nrep, "edges": inf["edges"], "ms": ms, "us_per_iteration": 1e3 * ms / T,
                     "edge_updates_per_s": T * inf["edges"] / (ms / 1e3), "gbs": gbs, "frac_of_peak": gbs / peak,
                     "mapping": {k: inf[k] for k in ("mode", "cluster", "threads", "grid")},
                     "autotune": tune.get("best") if tune else None})
        s.close()
    return {"workload": CONFIGS[1][0], "iterations": T, "rows": rows}


def knn_study(Solver, stream, args, peak):
    """The semi-dense kNN model (n = 2000, 50 nearest neighbours, L = 64,
    greedy colouring, 300 iterations): the Handshake run alone, autotuned."""
    models, T = models_for(3, seed=0)
    s = Solver(models)
    tune = s.autotune(2) if args.autotune > 0 else None

    def run():
        s.reset()
        s.run(T)
    run()
    ms, _ = _timed(stream, run, 2)
    inf = s.info()
    gbs = T * algorithmic_bytes(models) / (ms / 1e3) / 1e9
    s.close()
    return {"workload": CONFIGS[3][0], "edges": inf["edges"], "matchings": inf["phases"], "iterations": T, "ms": ms,
            "edge_updates_per_s": T * inf["edges"] / (ms / 1e3), "gbs": gbs, "frac_of_peak": gbs / peak,
            "mapping": {k: inf[k] for k in ("mode", "cluster", "threads", "grid")},
            "autotune": tune.get("best") if tune else None}


def differentiation_study(Solver, stream, args):
    """16 x K_50, L = 64, T = 50 with a state checkpoint every 10 iterations:
    the forward run (with the bound) and the backward (mplpp_backward) timed
    separately, with host gradients and with device gradients; device memory
    the solver holds afterwards, and the peak including the backward's
    transient gradient buffers (host-gradient path)."""
    import types
    import torch
    models, T = models_for(5, seed=0)
    s = Solver(models, record_every=10)

    def fwd(sol=s):
        sol.reset()
        sol.run(T)
        sol.bound(exact=True)

    def bwd():
        s.backward()
    fwd()
    bwd()
    fms, _ = _timed(stream, fwd, 3)
    fwd()
    bms, _ = _timed(stream, bwd, 2)
    inf = s.info()
    transient = 4 * sum(int(np.sum(np.asarray(m.labels, np.int64))) for m in models)
    transient += 4 * sum(int(np.sum(np.asarray(m.labels, np.int64)[m.edge_u] *
                                    np.asarray(m.labels, np.int64)[m.edge_v])) for m in models)
    s.close()
    # the same with the costs and the gradients in device memory (the
    # autograd path): no gradient buffers allocated and copied back per call
    dev = []
    for m in models:
        d = types.SimpleNamespace(labels=m.labels, edge_u=m.edge_u, edge_v=m.edge_v, schedule=m.schedule)
        d.unary = torch.as_tensor(np.ascontiguousarray(m.unary, np.float32)).cuda()
        d.pairwise = torch.as_tensor(np.ascontiguousarray(m.pairwise, np.float32)).cuda()
        dev.append(d)
    sd = Solver(dev, record_every=10, device_inputs=True)
    gu = torch.empty(sum(sd.unary_sizes), dtype=torch.float32, device="cuda")
    gp = torch.empty(max(1, sum(sd.pair_sizes)), dtype=torch.float32, device="cuda")

    def bwd_dev():
        sd.backward(None, gu, gp)
    fwd(sd)
    bwd_dev()
    fwd(sd)
    dms, _ = _timed(stream, bwd_dev, 2)
    sd.close()
    return {"workload": CONFIGS[5][0], "iterations": T, "record_every": 10, "forward_ms": fms, "backward_ms": bms,
            "backward_over_forward": bms / fms, "backward_device_gradients_ms": dms,
            "backward_device_gradients_over_forward": dms / fms, "solver_device_bytes": inf["device_bytes"],
            "peak_device_bytes": inf["device_bytes"] + transient}


def rules_comparison(Solver, stream, args):
    """The dense pose model and the semi-dense kNN model under the Handshake
    (H), MPLP (M) and uniform (U) updates (Sec. 4, eqs. (H), (M), (U)) from
    phi = 0 with the same schedule: the bound after one iteration (Thm. 2:
    H >= M >= U) and after 50, and the device time of the 50-iteration run
    (H: the autotuned mapping; M, U: one CTA per edge, one launch per
    matching)."""
    T = 50
    res = {}
    for cfg, name in ((2, "pose_K60_L300"), (3, "knn_n2000_k50_L64")):
        models, _ = models_for(cfg, seed=0)
        out = {"iterations": T}
        for rule in ("H", "M", "U"):
            s = Solver(models, rule=rule)
            if rule == "H" and args.autotune > 0:
                s.autotune(2)
            s.reset()
            s.run(1)
            d1 = float(s.bound(exact=True).sum())

            def run(sol=s):
                sol.reset()
                sol.run(T)
            run()
            ms, _ = _timed(stream, run, 2)
            inf = s.info()
            out[rule] = {"ms": ms, "edge_updates_per_s": T * inf["edges"] / (ms / 1e3),
                         "bound_1": d1, "bound": float(s.bound(exact=True).sum()),
                         "mode": inf["mode"], "threads": inf["threads"]}
            s.close()
        tol = 1e-6 * max(1.0, abs(out["H"]["bound_1"]))
        out["one_iteration_H_ge_M_ge_U"] = bool(out["H"]["bound_1"] >= out["M"]["bound_1"] - tol
                                                and out["M"]["bound_1"] >= out["U"]["bound_1"] - tol)
        out["highest_bound"] = max("HMU", key=lambda r: out[r]["bound"])
        res[name] = out
    return res


def _time_run(Solver, stream, models, T, args):
    s = Solver(models)
    if args.autotune > 0:
        s.autotune(2)

    def run():
        s.reset()
        s.run(T)
    run()
    ms, _ = _timed(stream, run, 2)
    inf = s.info()
    s.close()
    return ms, inf


def sparsity_study(Solver, stream, args, peak):
    """The Handshake solver on the pose model with edges removed at random
    (the paper's density study, Sec. 7; greedy edge colouring): per density,
    edge updates/s and algorithmic GB/s of the run (autotuned mapping)."""
    from paper_2004_08227_gb300 import workloads as W
    T = 100
    rows = []
    for keep in (1.0, 0.4, 0.1, 0.05, 0.01):
        ms, inf = _time_run(Solver, stream, [W.pose_sparse(keep, 60, 300, seed=0)], T, args)
        gbs = T * inf["bytes_per_iteration"] / (ms / 1e3) / 1e9
        rows.append({"keep": keep, "edges": inf["edges"], "matchings": inf["phases"], "ms": ms,
                     "edge_updates_per_s": T * inf["edges"] / (ms / 1e3), "gbs": gbs, "frac_of_peak": gbs / peak,
                     "mapping": {k: inf[k] for k in ("mode", "cluster", "threads", "grid")}})
    return {"workload": "pose_K60_L300, every edge kept with probability keep", "iterations": T, "rows": rows}


def pose_dense_study(Solver, stream, args):
    """The shape of the paper's pose dataset: fully connected, L = 13, n in the
    hundreds to thousands (round robin: n - 1 matchings of n / 2 edges)."""
    from paper_2004_08227_gb300 import workloads as W
    T = 20
    rows = []
    for n in (600, 1200):
        ms, inf = _time_run(Solver, stream, [W.pose_dense(n, 13, seed=0)], T, args)
        rows.append({"n": n, "edges": inf["edges"], "matchings": inf["phases"], "ms": ms,
                     "edge_updates_per_s": T * inf["edges"] / (ms / 1e3),
                     "gbs": T * inf["bytes_per_iteration"] / (ms / 1e3) / 1e9,
                     "mapping": {k: inf[k] for k in ("mode", "cluster", "threads", "grid")}})
    return {"workload": "pose_dense_Kn_L13", "iterations": T, "rows": rows}


def structured_study(Solver, stream, args):
    """Stereo-like grids with truncated-linear, Potts and truncated-quadratic
    costs: the structured Handshake path (no table reads) against the dense
    drivers on the same costs given as tables (autotuned), equal iterations."""
    from paper_2004_08227_gb300 import workloads as W
    T = 50
    rows = []
    for name, kw in (("truncated_linear_tau4", dict(weight=1.0, tau=4.0)), ("potts", dict(weight=1.0, tau=1.0)),
                     ("truncated_quadratic_tau16", dict(weight=0.1, tau=16.0, quad=True))):
        m = W.grid_trunc_linear(128, 128, 64, seed=0, **kw)
        row = {"costs": name}
        for key, structured in (("structured", True), ("dense", False)):
            s = Solver([m], structured=structured)
            if args.autotune > 0:
                s.autotune(2)

            def run(sol=s):
                sol.reset()
                sol.run(T)
            run()
            ms, _ = _timed(stream, run, 2)
            inf = s.info()
            row[key] = {"ms": ms, "edge_updates_per_s": T * inf["edges"] / (ms / 1e3),
                        "bound": float(s.bound(exact=True)[0]), "mode": inf["mode"]}
            s.close()
        row["speedup"] = row["dense"]["ms"] / row["structured"]["ms"]
        rows.append(row)
    return {"workload": "grid128x128_L64", "edges": int(m.E), "iterations": T, "rows": rows}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2004_08227_gb300.solver import Solver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev_index = local
    cfg = args.config
    name, T = CONFIGS[cfg]
    if args.iters:
        T = args.iters
    if cfg == 4 and args.models > 0:
        name = f"batch{args.models}_K10-80_L16-128_T{T}"
    if cfg == 1 and args.models > 0:
        name = f"K20_L8_uniform_x{args.models}_T{T}"
    # cpu baseline first (before any GPU work), rank 0 only
    cpu = cpu1 = None
    models, _ = models_for(cfg, seed=rank, count=args.models)
    if rank == 0 and world == 1 and not args.no_cpu:
        log("timing the oracle on the host ...")
        _, cpu = cpu_oracle_rate_parallel(models, T, args.cpu_budget)
        _, cpu1 = cpu_oracle_rate(models, T, args.cpu_budget)
    stream = torch.cuda.current_stream()
    s = Solver(models, mode=args.mode, cluster=args.cluster, threads=args.threads)
    tune = None
    if args.autotune > 0 and args.mode == "auto" and not (args.cluster or args.threads):
        tune = s.autotune(args.autotune)
        log("autotune:", tune.get("best"))
    info = s.info()
    E_total = info["edges"]
    log("solver:", info)

    def step(sol):
        sol.reset()
        sol.run(T)
        D = sol.bound(exact=True)
        sol.labeling()
        return D

    kern_ms = []

    def timed_step(sol):
        sol.reset()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sol.run(T)
        b.record(stream)
        D = sol.bound(exact=True)
        sol.labeling()
        kern_ms.append(a.elapsed_time(b))
        return D

    for _ in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev_index)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    D_persist = None
    for _ in range(args.steps):
        D_persist = timed_step(s)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    value = whole_job_rate(T * E_total, world, ms)
    bytes_iter = algorithmic_bytes(models)
    bytes_iter32 = info["bytes_per_iteration"]
    kms = statistics.mean(kern_ms)
    achieved = T * bytes_iter / (kms / 1e3) / 1e9
    achieved32 = T * bytes_iter32 / (kms / 1e3) / 1e9
    peak, peak_kind = load_peak()
    kernel = {"persistent": "hs_persistent_kernel", "queue": "hs_queue_kernel", "resident": "hs_resident_kernel",
              "warp": "hs_warp_kernel", "structured": "struct_kernel",
              "structured_queue": "struct_queue_kernel"}.get(info["mode"], "hs_looped_kernel")

    # the looped driver (one launch per matching) on the same workload, equal bound
    looped = None
    if not args.no_looped:
        looped = looped_baseline(Solver, models, T, stream, step, D_persist, ms, max(1, min(args.steps, 3)))

    # the batched workload (256 uneven models): one persistent solve of the
    # batch against a loop of plain per-model solves, equal final bounds
    batched = None
    if args.batched and cfg != 4:
        batched = batched_vs_looped(Solver, stream, args)

    # K_20 replicas, the kNN model and the differentiation batch
    replicas = knn = diff = None
    if args.extra and rank == 0:
        replicas = replicas_study(Solver, stream, args, peak)
        if cfg != 3:
            knn = knn_study(Solver, stream, args, peak)
        diff = differentiation_study(Solver, stream, args)

    # the M and U updates beside H (equal iterations)
    rules = None
    if args.rules and rank == 0:
        rules = rules_comparison(Solver, stream, args)

    # the pose model sparsified, and the pose dataset's dense small-L shape
    sparsity = dense13 = structured = None
    if args.studies and rank == 0:
        sparsity = sparsity_study(Solver, stream, args, peak)
        dense13 = pose_dense_study(Solver, stream, args)
        structured = structured_study(Solver, stream, args)

    # end to end through the public API with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        class _M:
            pass
        pinned = []
        h2d = 0
        for m in models:
            pm = _M()
            pm.labels, pm.edge_u, pm.edge_v, pm.schedule = m.labels, m.edge_u, m.edge_v, m.schedule
            pm.unary = torch.from_numpy(m.unary).pin_memory()
            pm.pairwise = torch.from_numpy(m.pairwise).pin_memory()
            h2d += pm.unary.numel() * 4 + pm.pairwise.numel() * 4
            pinned.append(pm)
        d2h = 8 * len(models) + 4 * sum(m.n for m in models) + 8 * len(models)
        # one solver (created untimed); every timed step copies that step's
        # costs from pinned host memory (mplpp_update_costs), solves, and reads
        # the bound, labels and energies back to the host
        se = Solver(pinned, mode=info["mode"], cluster=info["cluster"], threads=info["threads"])
        times = []
        for i in range(1 + max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            se.update_costs([pm.unary for pm in pinned], [pm.pairwise for pm in pinned])
            se.run(T)
            se.bound(exact=True)
            se.labeling()
            torch.cuda.synchronize()
            if i > 0:
                times.append(time.perf_counter() - t0)
        se.close()
        et = max_over_ranks(statistics.mean(times) * 1e3, world, "cuda") / 1e3
        e2e = {"value": whole_job_rate(T * E_total, world, et * 1e3), "unit": "edge_updates/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": et * 1e3,
               "step_ms": [round(t * 1e3, 2) for t in times], "timer": "host wall clock"}

    # per step: reset (1), the run (restamp + one persistent launch, or one
    # launch per matching and iteration), exact bound (3), rounding + energy
    launches_per_step = (1 + (2 if info["mode"] in ("persistent", "warp", "queue") else T * info["phases"]) + 3
                         + info["labeling_launches"])
    line = {
        "metric": "edge_updates_per_s", "value": value, "unit": "edge_updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": name, "models": len(models), "edges": E_total, "iterations": T,
                   "matchings": info["phases"], "mode": info["mode"], "cluster": info["cluster"],
                   "threads": info["threads"], "grid": info["grid"], "parallelism": f"replicas{world}",
                   "autotuned": bool(tune), 
                   "l2": "inputs larger than L2 (tables %.0f MB per model)" % (bytes_iter / 1e6)},
        "hbm_gbs": achieved,
        "roofline": {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind,
                     "traffic": kernel_traffic(T) if (cfg == 2 and info["mode"] == "persistent") else None,
                     "algorithmic_bytes_per_launch": T * bytes_iter,
                     "bytes_formula": "per edge update 4 L_u L_v + 16 (L_u + L_v)",
                     "achieved_state32": achieved32, "frac_state32": achieved32 / peak,
                     "bytes_formula_state32": "per edge update 4 L_u L_v + 32 (L_u + L_v) (double-float state)",
                     "launch_ms": kms},
        "config1_replicas": replicas,
        "knn": knn,
        "differentiation": diff,
        "looped": looped,
        "batched": batched,
        "rules": rules,
        "sparsity": sparsity,
        "pose_dense_L13": dense13,
        "structured": structured,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "cpu_baseline_single_thread": cpu1,
        "clocks": ck,
        "gpu_launches": launches_per_step * args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


def make_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=sorted(CONFIGS))
    ap.add_argument("--iters", type=int, default=0, help="override the iteration count")
    ap.add_argument("--mode", default="auto", choices=["auto", "looped", "persistent", "queue", "resident", "warp"])
    ap.add_argument("--models", type=int, default=0,
                    help="with --config 4: models of the batch recipe (0: the 256 of the workload); "
                         "with --config 1: replicas of the K_20 model")
    ap.add_argument("--cluster", type=int, default=0, help="CTAs per edge (0: chosen; set: no autotuning)")
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0: chosen; set: no autotuning)")
    ap.add_argument("--no-looped", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batched", type=int, default=1, help="also time the 256-model batch against per-model loops")
    ap.add_argument("--studies", type=int, default=1, help="also run the sparsified pose, dense L=13 and structured-cost workloads")
    ap.add_argument("--rules", type=int, default=1, help="also run the M and U updates beside H (pose and kNN)")
    ap.add_argument("--autotune", type=int, default=3, help="iterations per candidate of the mapping autotuner (0: off)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--extra", type=int, default=1,
                    help="also run K_20 replicas, the kNN model and the differentiation batch")
    ap.add_argument("--replicas", type=int, default=4096, help="K_20 replicas solved together")
    ap.add_argument("--ref-iters", type=int, default=10,
                    help="--impl reference: oracle iterations per step (amortizes the copy of the FP64 state)")
    return ap


def main():
    args = make_parser().parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
