"""GPU parity of the MPLP update (Sec. 4, eq. (M)) and the uniform update
(Sec. 4, eq. (U)) against the FP64 oracle, and the paper's dominance results
(Prop. 2, Thm. 2) reproduced on the GPU.

Tolerances as in test_gpu_parity.py: D within 1e-5 relative of max(|D|, 1);
theta^phi_u and the implied reparametrized tables entry by entry within 1e-5
of their scales; every label within twice the FP32 error bound of the minimum
of the oracle's rounding objective conditioned on the GPU's earlier labels
(tests/_parity.py).
"""
import numpy as np
import pytest

import oracle
from oracle import schedule as osched
from paper_2004_08227_gb300 import workloads as W
from paper_2004_08227_gb300._lib import MplppError
from paper_2004_08227_gb300.solver import Solver

import _parity as P

pytestmark = pytest.mark.gpu

RTOL_D = 1e-5


def _order(m):
    return osched.build(m.schedule, m.n, m.edge_u, m.edge_v)[1]


def _check_D(Dg, Do):
    assert abs(Dg - Do) <= RTOL_D * max(abs(Do), 1.0), (Dg, Do)


def _check_state_labels(s, m, xg, th_u, th_uv):
    agg, msg = P.model_state(s, [m], 0)
    P.check_state(m, agg, th_u, what=m.name)
    P.check_tables(m, msg, th_uv, agg, what=m.name)
    P.check_labels(m, th_u, th_uv, xg, oracle.round_labels(m, th_u, th_uv), what=m.name)


def _model(case):
    if case == "K20_L8":
        m, _ = W.config(1)
        return m, 60
    if case == "uneven_1_70":
        return W.uneven_complete(9, 1, 70, seed=3), 20
    if case == "knn":
        return W.knn(240, 8, 20, seed=3), 20
    if case == "wide_rows":  # rows longer than a warp's 32 float4 chunks
        return W.uneven_complete(4, 100, 300, seed=8), 6
    raise ValueError(case)


@pytest.mark.parametrize("rule", ["M", "U"])
@pytest.mark.parametrize("case", ["K20_L8", "uneven_1_70", "knn", "wide_rows"])
def test_rule_parity_with_oracle(rule, case):
    m, T = _model(case)
    th_u, th_uv = oracle.run(m, _order(m), T, rule=rule)
    Do = oracle.bound(m, th_u, th_uv)
    for graph in (True, False):
        s = Solver([m], rule=rule, use_graph=graph)
        assert s.info()["mode"] == "looped"
        s.run(T)
        _check_D(s.bound(exact=True)[0], Do)
        xs, _ = s.labels_per_model()
        _check_state_labels(s, m, xs[0], th_u, th_uv)


def test_rule_batch_of_uneven_models():
    models = [W.uneven_complete(n, 3, 40, seed=60 + n) for n in (3, 5, 8, 11)]
    T = 15
    for rule in ("M", "U"):
        s = Solver(models, rule=rule)
        s.run(T)
        D = s.bound(exact=True)
        for i, m in enumerate(models):
            _check_D(D[i], oracle.bound(m, *oracle.run(m, _order(m), T, rule=rule)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_one_iteration_dominance_on_gpu(seed):
    """Thm. 2: from the same start and schedule, one iteration of H gives a
    bound at least that of one M-iteration, which is at least that of one
    U-iteration (with FP32 slack)."""
    m = W.uneven_complete(12, 5, 40, seed=20 + seed)
    D = {}
    for rule in "HMU":
        s = Solver([m], rule=rule, mode="looped")
        s.run(1)
        D[rule] = float(s.bound(exact=True)[0])
    tol = 1e-6 * max(1.0, abs(D["H"]))
    assert D["H"] >= D["M"] - tol and D["M"] >= D["U"] - tol, D


@pytest.mark.parametrize("rule", ["M", "U"])
def test_single_edge_update_entrywise(rule):
    """One update of a single 37 x 53 edge: the new node vectors equal the
    oracle's eq. (M) / eq. (U) update entry by entry (FP32 table minima:
    absolute error ~1e-6 at these magnitudes)."""
    rng = np.random.default_rng(4)
    m = W.Model(labels=np.array([37, 53], np.int32), edge_u=np.array([0], np.int32),
                edge_v=np.array([1], np.int32), unary=rng.random(90).astype(np.float32),
                pairwise=rng.standard_normal(37 * 53).astype(np.float32), schedule="greedy_color")
    s = Solver([m], rule=rule)
    s.run(1)
    _, agg, _ = s.state_arrays()
    tu, tv, _ = oracle.update_edge(rule, m.unary[:37], m.unary[37:], m.pairwise.reshape(37, 53))
    np.testing.assert_allclose(agg[:37], tu, rtol=0, atol=1e-5)
    np.testing.assert_allclose(agg[37:], tv, rtol=0, atol=1e-5)


@pytest.mark.parametrize("kw", [{"mode": "persistent"}, {"mode": "warp"}])
def test_rules_only_in_the_looped_driver(kw):
    m = W.complete(5, 3, seed=0)
    for rule in ("M", "U"):
        with pytest.raises(MplppError) as ei:
            Solver([m], rule=rule, **kw)
        assert ei.value.status == -7


def test_rules_have_no_backward():
    m = W.complete(5, 3, seed=0)
    with pytest.raises(MplppError) as ei:
        Solver([m], rule="M", record_every=5)
    assert ei.value.status == -1
