"""Writes the full-size expected values used by the GPU tests.

Calls only the FP64 oracle (oracle/) on the seeded workloads of
paper_2004_08227_gb300.workloads: for each workload shape, the dual bound
after the full iteration count, the rounded labeling and its energy; for the
differentiation shape also central finite differences (h = 1e-4) of D_T at
sampled entries.  The oracle is plain IEEE double C built without FP
contraction, so the values do not depend on the machine that writes them.

The states file (full_size_config<c>_states.json) holds the oracle's
reparametrized unaries theta^phi_u after the full iteration count at a seeded
sample of nodes (of a seeded sample of models for the batches), computed with
oracle.run_parallel (bit-identical to oracle.run).

usage: python tests/golden/make_golden.py [--states] {1,2,3,4,5} [...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle import schedule as osched  # noqa: E402
from paper_2004_08227_gb300 import workloads as W  # noqa: E402


def _order(m):
    return osched.build(m.schedule, m.n, m.edge_u, m.edge_v)[1]


def _digest(m):
    h = hashlib.sha256()
    for a in (m.labels, m.edge_u, m.edge_v, m.unary, m.pairwise):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]


def solve_entry(m, T):
    sol = oracle.solve(m, _order(m), T)
    return {"name": m.name, "inputs_sha256_16": _digest(m), "iterations": T, "bound": sol["bound"],
            "labels": sol["labels"].tolist(), "margins_min": float(np.min(sol["margins"])),
            "margins": [float(x) for x in sol["margins"]], "energy": sol["energy"]}


def fd_entries(m, T, count, seed=0, steps=(1e-4, 1e-5, 1e-6)):
    """Central differences of D_T at sampled entries.  D_T is piecewise linear:
    where the one-sided differences at step h disagree (a kink within h) the
    next smaller step is tried; `h` records the step used (None: kink at all)."""
    order = _order(m)
    D, gu, gp = oracle.grad(m, order, T)
    rng = np.random.default_rng(seed)
    nz = np.flatnonzero(gp)
    picks = [("p", int(i)) for i in rng.choice(nz, size=count // 2, replace=False)]
    picks += [("p", int(i)) for i in rng.choice(gp.size, size=count // 4, replace=False)]
    picks += [("u", int(i)) for i in rng.choice(gu.size, size=count - len(picks), replace=False)]
    un0 = m.unary.astype(np.float64)
    pw0 = m.pairwise.astype(np.float64)

    def DT(which, i, d):
        un, pw = un0.copy(), pw0.copy()
        (un if which == "u" else pw)[i] += d
        th_u, th_uv = oracle.run(m, order, T, state=(un, pw))
        return oracle.bound(m, th_u, th_uv)

    out = []
    for which, i in picks:
        f0 = DT(which, i, 0.0)
        rec = {"which": which, "index": i, "oracle_grad": float((gu if which == "u" else gp)[i]), "h": None}
        for h in steps:
            fp, fm = DT(which, i, h), DT(which, i, -h)
            fd = (fp - fm) / (2 * h)
            right, left = (fp - f0) / h, (f0 - fm) / h
            rec.update({"fd": fd, "right": right, "left": left})
            if abs(right - left) <= 1e-4 * max(abs(fd), 1e-3):
                rec["h"] = h
                break
        out.append(rec)
    return {"D": D, "steps": list(steps), "entries": out}


# sampled nodes per model and models per workload of the states file
STATE_SAMPLE = {1: (20, 1), 2: (32, 1), 3: (128, 1), 4: (8, 16), 5: (8, 16)}


def states_entry(c, models, T):
    """theta^phi_u of the oracle at sampled nodes of sampled models."""
    nodes_per, models_per = STATE_SAMPLE[c]
    rng = np.random.default_rng(1000 + c)
    picks = sorted(rng.choice(len(models), size=min(models_per, len(models)), replace=False).tolist())
    out = []
    for i in picks:
        m = models[i]
        off, order = osched.build(m.schedule, m.n, m.edge_u, m.edge_v)
        th_u, _ = oracle.run_parallel(m, off, order, T)
        nodes = sorted(rng.choice(m.n, size=min(nodes_per, m.n), replace=False).tolist())
        uoff = np.concatenate([[0], np.cumsum(m.labels.astype(np.int64))])
        vals = np.concatenate([th_u[uoff[u]:uoff[u + 1]] for u in nodes])
        out.append({"model": int(i), "name": m.name, "inputs_sha256_16": _digest(m), "nodes": nodes,
                    "theta_u": [float(v) for v in vals]})
    return out


def main_states(cfgs):
    for c in cfgs:
        t0 = time.time()
        models, T = W.config(c)
        if not isinstance(models, list):
            models = [models]
        res = {"workload_config": c, "iterations": T,
               "writer": "tests/golden/make_golden.py --states (FP64 oracle only)",
               "samples": states_entry(c, models, T)}
        res["seconds"] = time.time() - t0
        with open(os.path.join(HERE, f"full_size_config{c}_states.json"), "w") as f:
            json.dump(res, f)
        print(f"config {c} states: {time.time() - t0:.0f} s", flush=True)


def main(cfgs):
    for c in cfgs:
        t0 = time.time()
        models, T = W.config(c)
        if not isinstance(models, list):
            models = [models]
        res = {"workload_config": c, "iterations": T,
               "writer": "tests/golden/make_golden.py (FP64 oracle only)",
               "models": [solve_entry(m, T) for m in models]}
        if c == 5:
            res["finite_differences_model0"] = fd_entries(models[0], T, 200)
        res["seconds"] = time.time() - t0
        with open(os.path.join(HERE, f"full_size_config{c}.json"), "w") as f:
            json.dump(res, f)
        print(f"config {c}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    args = sys.argv[1:]
    if args and args[0] == "--states":
        main_states([int(a) for a in args[1:]] or [1, 2, 3, 4, 5])
    else:
        main([int(a) for a in args] or [1, 2, 3, 4, 5])
