"""GPU parity of the warp driver (one warp per edge, persistent) against the
FP64 oracle, and bit-identity with the cluster and looped drivers.

Every driver performs the same operations in the same order per element
(Sec. 4, eq. (H) in message form), so their states must agree bit for bit;
against the oracle the tolerances are those of test_gpu_parity.py.
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


def _check_labels(s, models, i, xg, sol):
    """State, tables and conditional labels of model i (tests/_parity.py)."""
    m = models[i]
    agg, msg = P.model_state(s, models, i)
    P.check_state(m, agg, sol["th_u"], what=m.name)
    P.check_tables(m, msg, sol["th_uv"], agg, what=m.name)
    P.check_labels(m, sol["th_u"], sol["th_uv"], xg, sol["labels"], what=m.name)


def _solve(models, T, **kw):
    s = Solver(models, **kw)
    s.run(T)
    D = s.bound(exact=True)
    xs, _ = s.labels_per_model()
    return s, D, xs


@pytest.mark.parametrize("graph", [True, False])
def test_warp_parity_complete_K20_L8(graph):
    m, T = W.config(1)
    sol = oracle.solve(m, _order(m), T)
    s, D, xs = _solve([m], T, mode="warp", use_graph=graph)
    assert s.info()["mode"] == "warp"
    _check_D(D[0], sol["bound"])
    _check_labels(s, [m], 0, xs[0], sol)


@pytest.mark.parametrize("threads", [32, 64, 128])
def test_warp_parity_uneven_labels(threads):
    """Ragged label counts 1..70 (rows not multiples of 32, columns not of 4)."""
    m = W.uneven_complete(9, 1, 70, seed=threads % 13)
    T = 25
    sol = oracle.solve(m, _order(m), T)
    s, D, xs = _solve([m], T, mode="warp", threads=threads)
    assert s.info()["threads"] == threads
    _check_D(D[0], sol["bound"])
    _check_labels(s, [m], 0, xs[0], sol)


@pytest.mark.parametrize("threads", [32, 128])
def test_warp_parity_streamed_tables(threads):
    """Label counts 65..128: tables larger than a warp's buffer (32 rows of the
    widest table) stream through both buffers in 32-row chunks, once per pass;
    several row groups per table."""
    m = W.uneven_complete(6, 65, 128, seed=5)
    T = 8
    sol = oracle.solve(m, _order(m), T)
    sw, D, xs = _solve([m], T, mode="warp", threads=threads)
    _check_D(D[0], sol["bound"])
    _check_labels(sw, [m], 0, xs[0], sol)
    ref = Solver([m], mode="persistent")
    ref.run(T)
    s = Solver([m], mode="warp", threads=threads)
    s.run(T)
    a, b = s.state_arrays(), ref.state_arrays()
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_warp_parity_knn_and_batch():
    models = [W.knn(240, 8, 20, seed=3)]
    models += [W.uneven_complete(n, 3, 40, seed=50 + n) for n in (3, 5, 8, 11, 2)]
    T = 20
    s, D, xs = _solve(models, T, mode="warp")
    for i, m in enumerate(models):
        sol = oracle.solve(m, _order(m), T)
        _check_D(D[i], sol["bound"])
        _check_labels(s, models, i, xs[i], sol)


def test_warp_bitwise_equal_to_cluster_and_looped_drivers():
    models = [W.uneven_complete(10, 4, 90, seed=9), W.uneven_complete(7, 16, 128, seed=2)]
    states = []
    for kw in ({"mode": "warp"}, {"mode": "warp", "threads": 128}, {"mode": "persistent"}, {"mode": "looped"},
               {"mode": "persistent", "cluster": 3}):
        s = Solver(models, **kw)
        s.run(17)
        states.append(s.state_arrays())
    for st in states[1:]:
        assert np.array_equal(st[1], states[0][1]) and np.array_equal(st[2], states[0][2])


def test_warp_resume_bitwise():
    m, _ = W.config(1)
    a = Solver([m], mode="warp")
    a.run(60)
    b = Solver([m], mode="warp")
    b.run(30)
    c = Solver([m], mode="warp")
    c.load_state(b.save_state())
    c.run(30)
    sa, sc = a.state_arrays(), c.state_arrays()
    assert np.array_equal(sa[1], sc[1]) and np.array_equal(sa[2], sc[2])


def test_warp_bounded_wait_times_out_without_hanging():
    m = W.complete(10, 8, seed=0)
    s = Solver([m], mode="warp", test_unreachable_wait=True, spin_limit=2000)
    s.run(3)
    with pytest.raises(MplppError) as ei:
        s.sync()
    assert ei.value.status == -4
    s.close()
    m2, T = W.config(1)
    sol = oracle.solve(m2, _order(m2), T)
    _, D, _ = _solve([m2], T, mode="warp")
    _check_D(D[0], sol["bound"])


def test_warp_rejects_labels_beyond_its_limit():
    m = W.complete(4, 130, seed=1)
    with pytest.raises(MplppError):
        Solver([m], mode="warp")


def test_autotune_measures_the_warp_driver():
    models = [W.uneven_complete(n, 16, 64, seed=n) for n in (12, 20, 9)]
    s = Solver(models)
    rep = s.autotune(2)
    assert any(c[2] == "warp" for c in rep["candidates"])
    assert s.info()["mode"] == rep["best"]["mode"]
