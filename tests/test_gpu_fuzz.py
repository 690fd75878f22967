"""Seeded randomized parity sweep: small models of random shape (complete
graphs with uneven label counts, kNN graphs with greedy edge colouring,
batches of several models), random iteration counts, solved by every driver
that takes the shapes (looped, persistent, warp, queue and, for label counts
up to 32, resident) with varied block sizes, each checked against the FP64
oracle entry by entry: the reparametrized unaries, the implied reparametrized
tables, the bound, and the labels (the conditional check of _parity).

The cases are drawn from a fixed seed, so the sweep is the same on every run;
it complements the hand-picked cases of the other parity tests with shapes
nobody chose.
"""
import numpy as np
import pytest

import oracle
from oracle import schedule as osched
from paper_2004_08227_gb300 import workloads as W
from paper_2004_08227_gb300.solver import Solver

import _parity as P

pytestmark = pytest.mark.gpu


def _order(m):
    return osched.build(m.schedule, m.n, m.edge_u, m.edge_v)[1]


def _model(rng, k):
    kind = rng.choice(["complete", "knn"], p=[0.65, 0.35])
    lmax = int(rng.choice([2, 5, 8, 13, 24, 32, 48, 96, 140]))
    lmin = int(rng.integers(1, lmax + 1))
    seed = int(rng.integers(1 << 30))
    if kind == "complete":
        return W.uneven_complete(int(rng.integers(2, 13)), lmin, lmax, seed=seed)
    n = int(rng.integers(8, 41))
    return W.knn(n, int(rng.integers(2, 7)), lmax, seed=seed)


def _cases(count=48, seed=20261204):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        models = [_model(rng, k) for _ in range(int(rng.choice([1, 1, 2, 3])))]
        T = int(rng.integers(1, 7))
        lmax = max(int(np.max(m.labels)) for m in models)
        modes = ["looped", "persistent", "queue"]
        if lmax <= 128:  # the warp driver's label bound
            modes.append("warp")
        mode = str(rng.choice(modes))
        if lmax <= 32 and rng.random() < 0.5:
            mode = "resident"
        threads = 0
        if mode in ("looped", "persistent"):
            threads = int(rng.choice([0, 128, 256, 512]))
        elif mode == "resident":
            threads = int(rng.choice([0, 64, 96]))
        out.append((k, models, T, mode, threads))
    return out


CASES = _cases()


@pytest.mark.parametrize("k", range(len(CASES)))
def test_random_shapes_every_driver_matches_oracle(k):
    _, models, T, mode, threads = CASES[k]
    what = f"case {k} ({mode}, threads {threads}, T {T})"
    s = Solver(models, mode=mode, threads=threads)
    assert s.info()["mode"] == mode, what
    s.run(T)
    D = s.bound(exact=True)
    xs, en = s.labels_per_model()
    for i, m in enumerate(models):
        sol = oracle.solve(m, _order(m), T)
        agg, msg = P.model_state(s, models, i)
        P.check_state(m, agg, sol["th_u"], what=f"{what} model {i}")
        P.check_tables(m, msg, sol["th_uv"], agg, what=f"{what} model {i}")
        assert abs(D[i] - sol["bound"]) <= P.RTOL_STATE * max(1.0, abs(sol["bound"])), (what, D[i], sol["bound"])
        P.check_labels(m, sol["th_u"], sol["th_uv"], xs[i], sol["labels"], what=f"{what} model {i}")
        assert abs(en[i] - oracle.energy(m, xs[i])) <= 1e-9 * max(1.0, abs(en[i])), what
    s.close()
