"""GPU parity of the structured Handshake path (truncated-linear costs
w min(|s - t|, tau), Potts for tau = 1: O(L) minimizations by prefix, suffix
and global minima or a window; truncated-quadratic w min((s - t)^2, tau): a
window) against the FP64 oracle on the same costs given as dense tables, and
against the dense GPU drivers.  Tolerances as in test_gpu_parity.py."""
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


def _check(m, T, s):
    sol = oracle.solve(m, _order(m), T)
    s.run(T)
    D = s.bound(exact=True)[0]
    assert abs(D - sol["bound"]) <= RTOL_D * max(abs(sol["bound"]), 1.0), (D, sol["bound"])
    xs, _ = s.labels_per_model()
    agg, msg = P.model_state(s, [m], 0)
    P.check_state(m, agg, sol["th_u"], what=m.name)
    P.check_tables(m, msg, sol["th_uv"], agg, what=m.name)
    P.check_labels(m, sol["th_u"], sol["th_uv"], xs[0], sol["labels"], what=m.name)
    return D


CASES = {
    "potts_L16": dict(rows=6, cols=7, L=16, weight=1.0, tau=1.0),
    "tl_L40": dict(rows=5, cols=6, L=40, weight=0.7, tau=4.0),
    "tl_L200": dict(rows=4, cols=5, L=200, weight=0.5, tau=12.0),
    "tl_L256_untruncated": dict(rows=3, cols=4, L=256, weight=0.05, tau=1000.0),
    "ragged_1_33": dict(rows=6, cols=6, L=33, weight=1.0, tau=3.0, Lmin=1),
    "ragged_2_70": dict(rows=5, cols=5, L=70, weight=0.3, tau=8.0, Lmin=2),
    "quad_L40_tau16": dict(rows=5, cols=6, L=40, weight=0.1, tau=16.0, quad=True),
    "quad_L64_untruncated": dict(rows=4, cols=4, L=64, weight=0.002, tau=1e6, quad=True),
    "quad_ragged_tau30": dict(rows=5, cols=5, L=50, weight=0.05, tau=30.0, Lmin=3, quad=True),
    "quad_L80_tau400": dict(rows=4, cols=5, L=80, weight=0.01, tau=400.0, quad=True),
    "quad_ragged_env": dict(rows=4, cols=4, L=120, weight=0.004, tau=2000.0, Lmin=17, quad=True),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_structured_parity_with_oracle(case):
    m = W.grid_trunc_linear(seed=3, **CASES[case])
    s = Solver([m])
    assert s.info()["mode"] == "structured"
    _check(m, 15, s)


@pytest.mark.parametrize("case,exact", [("potts_L16", True), ("tl_L40", True), ("ragged_2_70", True),
                                        ("quad_L40_tau16", True), ("quad_ragged_tau30", True),
                                        ("quad_L64_untruncated", False), ("quad_L80_tau400", False),
                                        ("quad_ragged_env", False), ("tl_L200", False),
                                        ("tl_L256_untruncated", False)])
def test_structured_equals_dense_drivers(case, exact):
    """Short truncation (linear radius <= 7, Potts included; quadratic radius
    <= 16): the window of candidates plus the global minimizer give the dense
    kernel's minimum of the same rounded values, so the states agree bit for
    bit.  Longer truncation: the linear scans or the quadratic lower envelope
    pick the minimizers, which rounding may decide differently where several
    have nearly the same value (reparametrized vectors form linear ramps
    along which w|s - t| + h(t) is constant): bounds within 1e-6 relative,
    state entries within 1e-5."""
    m = W.grid_trunc_linear(seed=5, **CASES[case])
    T = 20
    a = Solver([m])
    assert a.info()["mode"] == "structured"
    a.run(T)
    b = Solver([m], structured=False)
    assert b.info()["mode"] != "structured"
    b.run(T)
    sa, sb = a.state_arrays(), b.state_arrays()
    if exact:
        assert np.array_equal(sa[1], sb[1]) and np.array_equal(sa[2], sb[2])
        return
    Da, Db = a.bound(exact=True)[0], b.bound(exact=True)[0]
    assert abs(Da - Db) <= 1e-6 * max(1.0, abs(Db)), (Da, Db)
    for x, y in ((sa[1], sb[1]), (sa[2], sb[2])):
        assert np.all(np.abs(x - y) <= 1e-5 * np.maximum(1.0, np.abs(y))), np.abs(x - y).max()


@pytest.mark.parametrize("mode", ["persistent", "looped", "warp"])
def test_materialized_tables_in_the_dense_drivers(mode):
    """Structured input, dense drivers: the tables built on the device from
    (w, tau) give the oracle's result."""
    m = W.grid_trunc_linear(seed=7, **CASES["ragged_1_33"])
    _check(m, 12, Solver([m], mode=mode))


def test_structured_device_inputs_bitwise_equal_host_inputs():
    import torch
    m = W.grid_trunc_linear(seed=9, **CASES["tl_L40"])
    a = Solver([m])
    a.run(10)
    md = W.Model(m.labels, m.edge_u, m.edge_v, torch.from_numpy(m.unary).cuda(), None, schedule=m.schedule,
                 pair_kind="trunc_linear", pair_param=torch.from_numpy(np.ascontiguousarray(m.pair_param)).cuda())
    b = Solver([md], device_inputs=True)
    b.run(10)
    sa, sb = a.state_arrays(), b.state_arrays()
    assert np.array_equal(sa[1], sb[1]) and np.array_equal(sa[2], sb[2])


def test_large_labels_fall_back_to_the_dense_drivers():
    m = W.grid_trunc_linear(rows=2, cols=3, L=300, weight=0.5, tau=10.0, seed=1)
    s = Solver([m])
    assert s.info()["mode"] != "structured"
    _check(m, 6, s)
    with pytest.raises(MplppError) as ei:
        Solver([m], mode="structured")
    assert ei.value.status == -7


def test_structured_rejections():
    m = W.grid_trunc_linear(seed=0, **CASES["potts_L16"])
    dense = W.complete(5, 3, seed=0)
    with pytest.raises(MplppError) as ei:
        Solver([dense], mode="structured")
    assert ei.value.status == -7
    bad = W.grid_trunc_linear(seed=0, **CASES["potts_L16"])
    bad.pair_param = bad.pair_param.copy()
    bad.pair_param[3, 0] = -1.0
    with pytest.raises(MplppError) as ei:
        Solver([bad])
    assert ei.value.status == -1
    with pytest.raises(MplppError) as ei:
        Solver([m], record_every=5)
    assert ei.value.status == -1
    s = Solver([m])
    with pytest.raises(MplppError) as ei:
        s.update_costs([m.unary], [m.pairwise])
    assert ei.value.status == -7


def test_autotune_measures_the_structured_driver():
    m = W.grid_trunc_linear(seed=2, **CASES["tl_L40"])
    s = Solver([m])
    rep = s.autotune(2)
    assert any(c[2] == "structured" for c in rep["candidates"])
    assert s.info()["mode"] == rep["best"]["mode"]


def test_mixed_structured_and_dense_models_in_one_solver():
    """A batch mixing a structured model with dense ones runs the dense
    drivers on the materialized tables; every model matches the oracle, and
    the M update runs on them as well."""
    ms = [W.grid_trunc_linear(seed=11, **CASES["tl_L40"]), W.uneven_complete(6, 3, 30, seed=4),
          W.grid_trunc_linear(seed=12, **CASES["quad_ragged_tau30"])]
    T = 10
    s = Solver(ms)
    assert s.info()["mode"] != "structured"
    s.run(T)
    D = s.bound(exact=True)
    for i, m in enumerate(ms):
        Do = oracle.bound(m, *oracle.run(m, _order(m), T))
        assert abs(D[i] - Do) <= RTOL_D * max(abs(Do), 1.0), (i, D[i], Do)
    r = Solver(ms, rule="M")
    r.run(T)
    D = r.bound(exact=True)
    for i, m in enumerate(ms):
        Do = oracle.bound(m, *oracle.run(m, _order(m), T, rule="M"))
        assert abs(D[i] - Do) <= RTOL_D * max(abs(Do), 1.0), (i, D[i], Do)


@pytest.mark.parametrize("case", ["potts_L16", "tl_L200", "ragged_2_70", "quad_L40_tau16"])
def test_structured_queue_driver_bitwise_equal_to_looped(case):
    """The structured update in one launch (every warp taking edges from one
    queue, versioned waits): bit for bit the looped structured driver."""
    m = W.grid_trunc_linear(seed=3, **CASES[case])
    a = Solver([m], mode="structured")
    b = Solver([m], mode="structured_queue")
    assert b.info()["mode"] == "structured_queue"
    for T in (6, 2):
        a.run(T)
        b.run(T)
        sa, sb = a.state_arrays(), b.state_arrays()
        assert np.array_equal(sa[1], sb[1]) and np.array_equal(sa[2], sb[2])


def test_structured_queue_bounded_wait_times_out():
    m = W.grid_trunc_linear(seed=1, **CASES["potts_L16"])
    s = Solver([m], mode="structured_queue", test_unreachable_wait=True, spin_limit=2000)
    s.run(2)
    with pytest.raises(MplppError) as ei:
        s.sync()
    assert ei.value.status == -4
