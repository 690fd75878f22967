"""Seeded randomized parity sweeps of the two paths the dense sweep
(test_gpu_fuzz.py) does not reach:

- structured costs (Sec. 4, message passing with truncated-linear, Potts and
  truncated-quadratic costs, no table reads): random grid sizes, label counts
  (equal or ragged), weights and truncations, including untruncated costs and
  the quadratic lower envelope, one or two models per solver, solved by the
  looped structured driver or the structured queue driver;
- the MPLP and uniform updates (eqs. (M) and (U)) on random complete and kNN
  models, one to three per solver.

Every case is checked against the FP64 oracle entry by entry, as the other
parity tests do: the reparametrized unaries, the implied reparametrized
tables, the bound and the labels (the conditional check of _parity).  The
cases are drawn from fixed seeds, so the sweeps are the same on every run.
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


def _grid(rng):
    quad = bool(rng.random() < 0.4)
    L = int(rng.choice([1, 2, 5, 16, 33, 64, 100, 128] + ([] if quad else [200, 256])))
    Lmin = int(rng.integers(1, L + 1)) if (L > 2 and rng.random() < 0.4) else 0
    if quad:
        tau = float(rng.choice([1.0, 4.0, 16.0, 90.0, 400.0, 1e6]))
        weight = float(rng.choice([0.002, 0.01, 0.05, 0.3]))
    else:
        tau = float(rng.choice([1.0, 2.0, 4.0, 9.0, 30.0, 1e4]))
        weight = float(rng.choice([0.05, 0.3, 1.0, 2.0]))
    return W.grid_trunc_linear(int(rng.integers(2, 7)), int(rng.integers(2, 7)), L, weight, tau,
                               seed=int(rng.integers(1 << 30)), Lmin=Lmin, quad=quad)


def _structured_cases(count=24, seed=20261205):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        models = [_grid(rng) for _ in range(int(rng.choice([1, 1, 2])))]
        mode = str(rng.choice(["structured", "structured_queue"]))
        out.append((k, models, int(rng.integers(1, 9)), mode))
    return out


def _dense(rng):
    lmax = int(rng.choice([2, 5, 8, 13, 24, 48, 96]))
    seed = int(rng.integers(1 << 30))
    if rng.random() < 0.65:
        return W.uneven_complete(int(rng.integers(2, 11)), int(rng.integers(1, lmax + 1)), lmax, seed=seed)
    return W.knn(int(rng.integers(8, 33)), int(rng.integers(2, 6)), lmax, seed=seed)


def _rule_cases(count=16, seed=20261206):
    rng = np.random.default_rng(seed)
    return [(k, [_dense(rng) for _ in range(int(rng.choice([1, 1, 2, 3])))], int(rng.integers(1, 7)),
             str(rng.choice(["M", "U"]))) for k in range(count)]


STRUCTURED = _structured_cases()
RULES = _rule_cases()


def _check_all(s, models, sols, what):
    D = s.bound(exact=True)
    xs, en = s.labels_per_model()
    for i, (m, (th_u, th_uv)) in enumerate(zip(models, sols)):
        Do = oracle.bound(m, th_u, th_uv)
        assert abs(D[i] - Do) <= P.RTOL_STATE * max(1.0, abs(Do)), (what, i, D[i], Do)
        agg, msg = P.model_state(s, models, i)
        P.check_state(m, agg, th_u, what=f"{what} model {i}")
        P.check_tables(m, msg, th_uv, agg, what=f"{what} model {i}")
        P.check_labels(m, th_u, th_uv, xs[i], oracle.round_labels(m, th_u, th_uv), what=f"{what} model {i}")
        assert abs(en[i] - oracle.energy(m, xs[i])) <= 1e-9 * max(1.0, abs(en[i])), what


@pytest.mark.parametrize("k", range(len(STRUCTURED)))
def test_random_structured_costs_match_oracle(k):
    _, models, T, mode = STRUCTURED[k]
    what = f"structured case {k} ({mode}, T {T}, {[m.name for m in models]})"
    s = Solver(models, mode=mode)
    assert s.info()["mode"] == mode, what
    s.run(T)
    _check_all(s, models, [oracle.run(m, _order(m), T) for m in models], what)
    s.close()


@pytest.mark.parametrize("k", range(len(RULES)))
def test_random_rule_updates_match_oracle(k):
    _, models, T, rule = RULES[k]
    what = f"rule case {k} ({rule}, T {T})"
    s = Solver(models, rule=rule)
    assert s.info()["mode"] == "looped", what
    s.run(T)
    _check_all(s, models, [oracle.run(m, _order(m), T, rule=rule) for m in models], what)
    s.close()
