"""GPU parity: the CUDA solver against the FP64 oracle on seeded inputs.

After the same schedule and iterations: the dual bound within 1e-5 relative
(of max(|D|, 1)); the reparametrized unaries theta^phi_u entry by entry within
1e-5 of each node's scale and every implied reparametrized table entry within
1e-5 of its edge's scale; every label within twice the FP32 error bound of the
minimum of the oracle's rounding objective conditioned on the GPU's earlier
labels (tests/_parity.py; the number of labels that differ is printed);
energies of the returned labelings equal their FP64 definition.  Integer
outputs (schedules, labels from a given state) are compared bit for bit.
"""
import json
import os

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
GOLD = os.path.join(os.path.dirname(__file__), "golden", "prop3_counterexample.json")


def _order(m):
    return osched.build(m.schedule, m.n, m.edge_u, m.edge_v)[1]


def _energy_def(m, x):
    """E(x|theta) written out from eq. energy-min (numpy, FP64)."""
    uoff = np.concatenate([[0], np.cumsum(m.labels.astype(np.int64))])
    E = float(np.sum(m.unary.astype(np.float64)[uoff[:-1] + x]))
    Lv = m.labels[m.edge_v].astype(np.int64)
    sizes = m.labels[m.edge_u].astype(np.int64) * Lv
    poff = np.concatenate([[0], np.cumsum(sizes)])[:-1]
    E += float(np.sum(m.pairwise.astype(np.float64)[poff + x[m.edge_u] * Lv + x[m.edge_v]]))
    return E


def _check_D(Dg, Do):
    assert abs(Dg - Do) <= RTOL_D * max(abs(Do), 1.0), (Dg, Do)


def _check(s, models, i, xg, sol, eg, rtol=P.RTOL_STATE):
    """State, tables and labels of model i against the oracle's solution."""
    m = models[i]
    agg, msg = P.model_state(s, models, i)
    P.check_state(m, agg, sol["th_u"], rtol=rtol, what=m.name)
    P.check_tables(m, msg, sol["th_uv"], agg, rtol=rtol, what=m.name)
    P.check_labels(m, sol["th_u"], sol["th_uv"], xg, sol["labels"], rtol=rtol, what=m.name)
    assert abs(eg - _energy_def(m, xg)) <= 1e-9 * max(1.0, abs(eg))


def _solve_gpu(models, T, **kw):
    s = Solver(models, **kw)
    s.run(T)
    D = s.bound(exact=True)
    xs, en = s.labels_per_model()
    return s, D, xs, en


def test_worked_example_exact():
    """Appendix B, proof of Prop. 3: the printed H results, bit for bit (all
    values are exact in binary32)."""
    g = json.load(open(GOLD))
    tuv = np.asarray(g["theta_uv"], np.float32).ravel()
    for tu, tv, key in ((g["theta_u"], g["theta_v"], "H"), (g["theta_u_prime"], g["theta_v_prime"], "H_prime")):
        m = W.Model(np.asarray([2, 2], np.int32), np.asarray([0], np.int32), np.asarray([1], np.int32),
                    np.asarray(tu + tv, np.float32), tuv.copy())
        for mode in ("looped", "persistent"):
            s = Solver([m], mode=mode)
            s.run(1)
            _, agg, msg = s.state_arrays()
            assert agg[:2].tolist() == g[key]["theta_u"]
            assert agg[2:].tolist() == g[key]["theta_v"]
            # theta^phi_uv = theta_uv - phi_{v->u} - phi_{u->v}: the residual table
            res = tuv.reshape(2, 2) - msg[:2, None] - msg[2:][None, :]
            assert res.tolist() == g["derived_by_hand_not_printed"]["H_residual" if key == "H" else "H_prime_residual"]
            # single edge: D = min g = MAP energy after one update (Prop. 1)
            Dg = s.bound(exact=True)[0]
            gmat = tuv.reshape(2, 2) + np.asarray(tu, np.float32)[:, None] + np.asarray(tv, np.float32)[None, :]
            assert Dg == float(gmat.min())
            s.close()


@pytest.mark.parametrize("mode,graph", [("looped", True), ("looped", False), ("persistent", True),
                                        ("persistent", False)])
def test_parity_complete_K20_L8(mode, graph):
    m, T = W.config(1)
    sol = oracle.solve(m, _order(m), T)
    s, D, xs, en = _solve_gpu([m], T, mode=mode, use_graph=graph)
    _check_D(D[0], sol["bound"])
    _check(s, [m], 0, xs[0], sol, en[0])
    assert s.info()["mode"] == mode


@pytest.mark.parametrize("cluster,threads", [(1, 128), (1, 256), (2, 256), (3, 512), (5, 128), (8, 256)])
@pytest.mark.parametrize("mode", ["looped", "persistent"])
def test_parity_uneven_labels_clusters(cluster, threads, mode):
    """Ragged shapes: per-node L in 1..70 (not multiples of 4), tables split
    over 1..8 CTAs (rows not divisible by the cluster size)."""
    m = W.uneven_complete(9, 1, 70, seed=cluster * 10 + threads % 7)
    T = 25
    sol = oracle.solve(m, _order(m), T)
    s, D, xs, en = _solve_gpu([m], T, mode=mode, cluster=cluster, threads=threads)
    inf = s.info()
    assert inf["cluster"] == cluster and inf["threads"] == threads
    _check_D(D[0], sol["bound"])
    _check(s, [m], 0, xs[0], sol, en[0])


def test_parity_knn_greedy_colouring():
    m = W.knn(240, 8, 20, seed=3)
    T = 30
    sol = oracle.solve(m, _order(m), T)
    s, D, xs, en = _solve_gpu([m], T)
    _check_D(D[0], sol["bound"])
    _check(s, [m], 0, xs[0], sol, en[0])


def test_parity_pose_like_L300_small():
    """Config-2 shape (L = 300, truncated quadratic costs) on K_8: 4 edges per
    matching, so every table spans a cluster of CTAs."""
    m = W.pose_like(8, 300, seed=1)
    T = 12
    sol = oracle.solve(m, _order(m), T)
    for mode in ("looped", "persistent"):
        s, D, xs, en = _solve_gpu([m], T, mode=mode)
        assert s.info()["cluster"] > 1
        _check_D(D[0], sol["bound"])
        _check(s, [m], 0, xs[0], sol, en[0])


def test_parity_batch_uneven_models():
    """Several models with uneven n and L solved together (batched phases)."""
    models = [W.uneven_complete(n, 3, 40, seed=50 + n) for n in (3, 5, 8, 11, 2)]
    models.append(W.tiny(7, 9, seed=4, density=0.5, uneven=True, pairwise="normal"))
    T = 20
    for mode in ("looped", "persistent", "queue"):
        s, D, xs, en = _solve_gpu(models, T, mode=mode)
        assert s.info()["mode"] == mode
        for i, m in enumerate(models):
            sol = oracle.solve(m, _order(m), T)
            _check_D(D[i], sol["bound"])
            _check(s, models, i, xs[i], sol, en[i])


def test_dual_monotone_on_gpu():
    """Lemma B.4 on the GPU trajectory (FP32 tolerance)."""
    m = W.complete(16, 24, seed=2, pairwise="normal")
    s = Solver([m])
    prev = s.bound()[0]
    for _ in range(15):
        s.run(2)
        D = s.bound()[0]
        assert D >= prev - 1e-6 * max(1.0, abs(prev))
        prev = D


def test_looped_and_persistent_bitwise_equal_and_deterministic():
    m = W.uneven_complete(10, 4, 90, seed=9)
    states = []
    for mode in ("looped", "persistent", "persistent", "queue", "queue"):
        s = Solver([m], mode=mode)
        s.run(17)
        states.append(s.state_arrays())
    for st in states[1:]:
        assert np.array_equal(st[1], states[0][1]) and np.array_equal(st[2], states[0][2])


def test_checkpoint_resume_bitwise():
    """100 + save/load + 100 iterations == 200 iterations, bit for bit."""
    m, _ = W.config(1)
    a = Solver([m])
    a.run(200)
    b = Solver([m])
    b.run(100)
    blob = b.save_state()
    c = Solver([m])
    c.load_state(blob)
    c.run(100)
    sa, sc = a.state_arrays(), c.state_arrays()
    assert sa[0] == sc[0] == 200
    assert np.array_equal(sa[1], sc[1]) and np.array_equal(sa[2], sc[2])
    assert a.bound()[0] == c.bound()[0]


def _round_case(kind, seed):
    if kind == "complete":  # one node per level: sequential rounding
        return W.uneven_complete(12, 2, 33, seed=100 + seed)
    if kind == "knn":  # few levels: one launch per level
        return W.knn(300, 6, 12, seed=seed)
    return W.grid_trunc_linear(12, 13, 9, 1.0, 3.0, seed=seed, Lmin=2)


@pytest.mark.parametrize("kind", ["complete", "knn", "grid"])
def test_rounding_decisions_match_oracle_bit_for_bit(kind):
    """Rounding from a given state: both sides take every argmin decision in
    binary64 with the same summation order (unary, then earlier neighbours by
    increasing index), so the labels must be identical -- whether the nodes are
    decided one after another or level by level (a node's earlier neighbours
    all in earlier levels)."""
    rng = np.random.default_rng(0)
    for seed in range(4):
        m = _round_case(kind, seed)
        s = Solver([m], structured=False)
        agg = rng.standard_normal(int(m.labels.sum()))
        g = oracle.Graph.of(m)
        Lu = m.labels[m.edge_u]
        Lv = m.labels[m.edge_v]
        msg = rng.standard_normal(int((Lu + Lv).sum()))
        s.set_state(agg, msg)
        xg, _ = s.labeling()
        # theta^phi_uv = (theta_uv - phi_{v->u}) - phi_{u->v} (eq. reparametrization), binary64
        th_uv = np.empty(m.pairwise.shape, np.float64)
        k = 0
        for e in range(m.E):
            pu = msg[k:k + Lu[e]]
            pv = msg[k + Lu[e]:k + Lu[e] + Lv[e]]
            k += Lu[e] + Lv[e]
            t = g.table(m.pairwise, e).astype(np.float64)
            th_uv[g.poff[e]:g.poff[e + 1]] = ((t - pu[:, None]) - pv[None, :]).ravel()
        xo = oracle.round_labels(m, agg, th_uv)
        assert np.array_equal(xg, xo)


@pytest.mark.parametrize("case", ["ties", "large", "near_ties"])
def test_rounding_screen_matches_fp64_decisions(case):
    """The rounding kernel screens labels in double-float with an error bound
    and sums only the surviving candidates in FP64; its decisions must equal
    the all-FP64 ones (oracle, same summation order) on the solver's own
    state: exact ties (values on a 1/8 grid, lowest index wins), large
    message magnitudes, and pairs of labels whose objectives differ by 2^-40."""
    rng = np.random.default_rng(21)
    m = _tied_model() if case == "ties" else W.uneven_complete(10, 4, 40, seed=8)
    g = oracle.Graph.of(m)
    Lu, Lv = m.labels[m.edge_u], m.labels[m.edge_v]
    nagg, nmsg = int(m.labels.sum()), int((Lu + Lv).sum())
    uoff = np.concatenate([[0], np.cumsum(m.labels.astype(np.int64))])
    moff = np.concatenate([[0], np.cumsum((Lu + Lv).astype(np.int64))])
    if case == "ties":
        agg = np.floor(rng.uniform(-4, 4, nagg) * 8) / 8
        msg = np.floor(rng.uniform(-4, 4, nmsg) * 8) / 8
    elif case == "large":
        agg, msg = rng.normal(0.0, 1e4, nagg), rng.normal(0.0, 1e4, nmsg)
    else:
        # labels 0 and 1 of every node enter its objective identically except
        # for the unary, which differs by 2^-40 (sign alternating by node)
        pw = m.pairwise.copy()
        for e in range(m.E):
            t = pw[g.poff[e]:g.poff[e + 1]].reshape(int(Lu[e]), int(Lv[e]))
            t[:, 1] = t[:, 0]
        m.pairwise = pw
        agg, msg = rng.normal(0.0, 1.0, nagg), rng.normal(0.0, 1.0, nmsg)
        for e in range(m.E):
            b0 = moff[e] + Lu[e]
            msg[b0 + 1] = msg[b0]
        for u in range(m.n):
            agg[uoff[u] + 1] = agg[uoff[u]] + (1 if u % 2 else -1) * 2.0 ** -40
    s = Solver([m])
    s.set_state(agg, msg)
    _, agg, msg = s.state_arrays()  # the double-float values the device holds
    xg, _ = s.labeling()
    th_uv = np.empty(m.pairwise.shape, np.float64)
    for e in range(m.E):
        pu = msg[moff[e]:moff[e] + Lu[e]]
        pv = msg[moff[e] + Lu[e]:moff[e + 1]]
        t = g.table(m.pairwise, e).astype(np.float64)
        th_uv[g.poff[e]:g.poff[e + 1]] = ((t - pu[:, None]) - pv[None, :]).ravel()
    xo = oracle.round_labels(m, agg, th_uv)
    assert np.array_equal(xg, xo)


def test_update_costs_equals_a_new_solver_bitwise():
    """mplpp_update_costs keeps the layout, mapping and graphs and restarts from
    phi = 0: the run afterwards equals a new solver's on those costs, bit for
    bit; a second update in a row does too; non-finite costs are rejected."""
    models = [W.uneven_complete(8, 4, 40, seed=30), W.uneven_complete(6, 10, 60, seed=31)]
    new = [W.uneven_complete(8, 4, 40, seed=30), W.uneven_complete(6, 10, 60, seed=31)]
    rng = np.random.default_rng(5)
    for m in new:
        m.unary = rng.random(m.unary.shape).astype(np.float32)
        m.pairwise = rng.standard_normal(m.pairwise.shape).astype(np.float32)
    for mode in ("persistent", "looped", "warp"):
        s = Solver(models, mode=mode)
        s.run(7)
        for _ in range(2):
            s.update_costs([m.unary for m in new], [m.pairwise for m in new])
            s.run(9)
            ref = Solver(new, mode=mode)
            ref.run(9)
            a, b = s.state_arrays(), ref.state_arrays()
            assert a[0] == b[0] == 9
            assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
            assert np.array_equal(s.bound(), ref.bound())
            assert np.array_equal(s.labeling()[0], ref.labeling()[0])
            ref.close()
        bad = new[0].pairwise.copy()
        bad[3] = np.inf
        with pytest.raises(MplppError):
            s.update_costs([m.unary for m in new], [bad, new[1].pairwise])
        s.close()


def test_bound_fast_equals_exact_after_full_iteration():
    """After a full iteration every reparametrized table has minimum 0 (Def. 1),
    so the node-only bound equals the exact one up to FP32 rounding."""
    m = W.complete(12, 16, seed=5, pairwise="normal")
    s = Solver([m])
    s.run(5)
    De, Df = s.bound(exact=True)[0], s.bound(exact=False)[0]
    assert abs(De - Df) <= 1e-5 * max(1.0, abs(De))


def _bound_from_state(m, agg, msg):
    """D(phi) (eq. LP-lower-bound) evaluated entry by entry in FP64 from a
    saved state: every node's and every table's minimum, each table entry as
    (theta - phi_{v->u}(s)) - phi_{u->v}(t).  Returns (D, sum of |terms|)."""
    g = oracle.Graph.of(m)
    uoff = np.concatenate([[0], np.cumsum(m.labels.astype(np.int64))])
    terms = [float(agg[uoff[u]:uoff[u + 1]].min()) for u in range(m.n)]
    k = 0
    for e in range(m.E):
        Lu, Lv = int(m.labels[m.edge_u[e]]), int(m.labels[m.edge_v[e]])
        pu, pv = msg[k:k + Lu], msg[k + Lu:k + Lu + Lv]
        k += Lu + Lv
        th = g.table(m.pairwise.astype(np.float64), e)
        terms.append(float(((th - pu[:, None]) - pv[None, :]).min()))
    return float(np.sum(terms)), float(np.sum(np.abs(terms)))


def _tied_model():
    """Costs on a coarse grid (many equal entries and equal minima)."""
    m = W.complete(10, 12, seed=3, pairwise="uniform")
    m.pairwise = (np.floor(m.pairwise * 4.0) / 4.0).astype(np.float32)
    m.unary = (np.floor(m.unary * 2.0) / 2.0).astype(np.float32)
    return m


@pytest.mark.parametrize("case", ["normal_T0", "normal_T4", "uneven_T2", "tied_T3", "large_state"])
def test_exact_bound_equals_entrywise_fp64_definition(case):
    """The exact bound's per-table minima are decided by an FP32 screen with
    an error bound and evaluated in FP64 only for the surviving candidates;
    the result must equal the entrywise FP64 definition on the solver's own
    state (up to the order of the final sum)."""
    rng = np.random.default_rng(11)
    if case.startswith("normal"):
        m, T = W.complete(12, 16, seed=5, pairwise="normal"), int(case[-1])
    elif case == "uneven_T2":
        m, T = W.uneven_complete(8, 5, 60, seed=12), 2
    elif case == "tied_T3":
        m, T = _tied_model(), 3
    else:
        m, T = W.uneven_complete(9, 3, 70, seed=4), 0
    s = Solver([m])
    s.run(T)
    if case == "large_state":  # messages and unaries far from the costs' scale
        _, agg, msg = s.state_arrays()
        s.set_state(rng.normal(0.0, 1e3, agg.size), rng.normal(0.0, 1e3, msg.size))
    _, agg, msg = s.state_arrays()
    Dg = s.bound(exact=True)[0]
    Dd, scale = _bound_from_state(m, agg, msg)
    assert abs(Dg - Dd) <= 1e-13 * (scale + 1.0), (Dg, Dd)


def test_residual_rows_and_columns_zero_after_update():
    """Def. 1 / text after eq. (H): after an edge's update all row and column
    minima of its reparametrized table are 0 (checked from the saved state)."""
    m = W.uneven_complete(8, 5, 60, seed=12)
    s = Solver([m])
    s.run(3)
    _, agg, msg = s.state_arrays()
    g = oracle.Graph.of(m)
    k = 0
    for e in range(m.E):
        Lu, Lv = int(m.labels[m.edge_u[e]]), int(m.labels[m.edge_v[e]])
        pu, pv = msg[k:k + Lu].astype(np.float64), msg[k + Lu:k + Lu + Lv].astype(np.float64)
        k += Lu + Lv
        r = g.table(m.pairwise.astype(np.float64), e) - pu[:, None] - pv[None, :]
        tol = 1e-5 * max(1.0, np.abs(r).max())
        assert np.all(np.abs(r.min(axis=1)) <= tol) and np.all(np.abs(r.min(axis=0)) <= tol)


# ---- edge cases ----------------------------------------------------------------------
def test_single_node_no_edges():
    m = W.Model(np.asarray([5], np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32),
                np.asarray([3, 1, 4, 1.5, 9], np.float32), np.zeros(0, np.float32))
    s = Solver([m])
    s.run(10)
    assert s.bound()[0] == 1.0
    x, en = s.labeling()
    assert x.tolist() == [1] and en[0] == 1.0


def test_single_label_nodes_and_empty_run():
    m = W.uneven_complete(6, 1, 1, seed=0)
    sol = oracle.solve(m, _order(m), 3)
    s = Solver([m])
    s.run(0)
    s.run(3)
    _check_D(s.bound()[0], sol["bound"])
    assert s.labeling()[0].tolist() == [0] * 6


def test_large_labels_L600_cluster8():
    m = W.uneven_complete(4, 600, 600, seed=1)
    T = 3
    sol = oracle.solve(m, _order(m), T)
    s, D, xs, en = _solve_gpu([m], T, mode="looped", cluster=8)
    _check_D(D[0], sol["bound"])
    _check(s, [m], 0, xs[0], sol, en[0])


def test_unsupported_shape_is_an_error():
    m = W.uneven_complete(2, 3000, 3000, seed=0)
    with pytest.raises(MplppError) as ei:
        Solver([m])
    assert ei.value.status == -7


@pytest.mark.parametrize("what", ["nan", "order", "dup", "schedule"])
def test_invalid_inputs_rejected(what):
    m = W.complete(5, 3, seed=0)
    sched = None
    if what == "nan":
        m.pairwise[7] = np.nan
    elif what == "order":
        m.edge_u[0], m.edge_v[0] = m.edge_v[0], m.edge_u[0]
    elif what == "dup":
        m.edge_v[1] = m.edge_v[0]
        m.schedule = "greedy_color"
    else:
        off, order = osched.round_robin(5, m.edge_u, m.edge_v)
        order = order.copy()
        order[0] = order[1]
        sched = [(off, order)]
    with pytest.raises(MplppError) as ei:
        Solver([m], user_schedules=sched)
    assert ei.value.status == -1


@pytest.mark.parametrize("kw", [{"mode": "persistent", "threads": 32}, {"mode": "looped", "threads": 96 + 1},
                                {"threads": 544}, {"mode": "warp", "threads": 16}, {"cluster": 9},
                                {"cluster": -1}])
def test_invalid_options_rejected(kw):
    """Block sizes the drivers cannot run (a cluster-driver CTA splits its
    warps between the two node vectors: two warps at least) and cluster sizes
    outside 1..8 are argument errors, not silent misbehaviour."""
    m = W.complete(5, 3, seed=0)
    with pytest.raises(MplppError) as ei:
        Solver([m], **kw)
    assert ei.value.status == -1


def test_bounded_wait_times_out_without_hanging():
    """A wait that nothing satisfies ends with MPLPP_E_TIMEOUT (bounded spin,
    drain without waiting), and the device stays usable afterwards."""
    m = W.complete(10, 8, seed=0)
    s = Solver([m], mode="persistent", test_unreachable_wait=True, spin_limit=2000)
    s.run(3)
    with pytest.raises(MplppError) as ei:
        s.sync()
    assert ei.value.status == -4
    s.close()
    m2, T = W.config(1)
    sol = oracle.solve(m2, _order(m2), 20)
    s2, D, _, _ = _solve_gpu([m2], 20, mode="persistent")
    _check_D(D[0], sol["bound"])


# ---- full size (the benchmark's workload and launch configuration) --------------------
@pytest.fixture(scope="module")
def pose_full():
    return W.pose_like(60, 300, seed=0)


def test_full_size_pose_K60_L300_parity_first_iterations(pose_full):
    """Full-size parity where the oracle still finishes in seconds: 2 iterations."""
    m = pose_full
    T = 2
    th_u, th_uv = oracle.run(m, _order(m), T)
    Do = oracle.bound(m, th_u, th_uv)
    s = Solver([m])
    assert s.info()["mode"] == "persistent"
    s.run(T)
    _check_D(s.bound()[0], Do)


def test_full_size_pose_K60_L300_properties(pose_full):
    """At the benchmark's size (500 iterations) the oracle is too slow to run in
    a test; properties that hold at any size are checked instead: D is
    monotone, D <= E(x) of the rounding, energies match their definition,
    looped == persistent bit for bit, and every residual table sampled has
    zero row and column minima."""
    m = pose_full
    s = Solver([m])
    Ds = [s.bound()[0]]
    for T in (1, 9, 90, 400):
        s.run(T)
        Ds.append(s.bound()[0])
    assert all(b >= a - 1e-6 * max(1.0, abs(a)) for a, b in zip(Ds, Ds[1:]))
    x, en = s.labeling()
    assert en[0] >= Ds[-1] - 1e-6 * abs(Ds[-1])
    assert abs(en[0] - _energy_def(m, x)) <= 1e-9 * abs(en[0])
    _, agg, msg = s.state_arrays()
    rng = np.random.default_rng(0)
    g = oracle.Graph.of(m)
    for e in rng.choice(m.E, size=12, replace=False):
        k = int(e) * 600
        r = g.table(m.pairwise, int(e)).astype(np.float64) - msg[k:k + 300, None] - msg[k + 300:k + 600][None, :]
        assert np.all(np.abs(r.min(axis=1)) <= 1e-4) and np.all(np.abs(r.min(axis=0)) <= 1e-4)
    a = Solver([m], mode="looped")
    b = Solver([m], mode="persistent")
    a.run(3)
    b.run(3)
    sa, sb = a.state_arrays(), b.state_arrays()
    assert np.array_equal(sa[1], sb[1]) and np.array_equal(sa[2], sb[2])


def test_autotune_keeps_state_and_results():
    """The autotuner leaves the state as it was, keeps a feasible mapping, and
    every mapping gives bit-identical results (minima are exact, additions
    per element), so the run after tuning matches an untuned run."""
    m = W.uneven_complete(10, 20, 90, seed=21)
    a = Solver([m])
    a.run(3)
    before = a.state_arrays()
    rep = a.autotune(2)
    after = a.state_arrays()
    assert np.array_equal(before[1], after[1]) and np.array_equal(before[2], after[2])
    assert rep["best"]["cluster"] >= 1 and len(rep["candidates"]) >= 2
    inf = a.info()
    assert inf["cluster"] == rep["best"]["cluster"] and inf["mode"] == rep["best"]["mode"]
    a.run(5)
    b = Solver([m])
    b.run(8)
    sa, sb = a.state_arrays(), b.state_arrays()
    assert np.array_equal(sa[1], sb[1]) and np.array_equal(sa[2], sb[2])


@pytest.mark.parametrize("cluster,threads", [(3, 512), (4, 512), (4, 256)])
@pytest.mark.parametrize("mode", ["looped", "persistent"])
def test_register_resident_passes_ragged(cluster, threads, mode):
    """Rows of 130..260 labels: tables whose CTA slice has at most 5 rows per
    warp take the register-resident passes (33..96 float4 chunks per row),
    the others the shared-memory passes, in the same solve; both must match
    the oracle and each other bit for bit."""
    m = W.uneven_complete(6, 130, 260, seed=cluster + threads)
    T = 6
    sol = oracle.solve(m, _order(m), T)
    s, D, xs, en = _solve_gpu([m], T, mode=mode, cluster=cluster, threads=threads)
    # 4 CTAs of 16 warps: 15 warps hold the at most 65 rows of a slice, the
    # 16th polls node u (persistent driver)
    assert s.info()["poller_warp"] == int(mode == "persistent" and (cluster, threads) == (4, 512))
    _check_D(D[0], sol["bound"])
    _check(s, [m], 0, xs[0], sol, en[0])
    ref = Solver([m], mode="looped", cluster=8, threads=128)  # never register-resident (5 rows x 4 warps < rows)
    ref.run(T)
    a, b = s.state_arrays(), ref.state_arrays()
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("cluster,threads", [(1, 64), (1, 128), (1, 256), (1, 512), (2, 64), (3, 256)])
@pytest.mark.parametrize("mode", ["looped", "persistent"])
def test_narrow_row_passes_ragged(cluster, threads, mode):
    """Rows of 1..128 labels (1..32 float4 chunks, slots of 1, 2, 4, 8, 16 and
    32 lanes): a CTA slice with at most 8 rows per lane slot takes the
    register-resident passes for narrow rows, the others the shared-memory
    passes, in the same solve; both must match the oracle, and the warp
    driver (its own code, no such passes) bit for bit."""
    m = W.uneven_complete(9, 1, 128, seed=7 * cluster + threads)
    T = 8
    sol = oracle.solve(m, _order(m), T)
    s, D, xs, en = _solve_gpu([m], T, mode=mode, cluster=cluster, threads=threads)
    _check_D(D[0], sol["bound"])
    _check(s, [m], 0, xs[0], sol, en[0])
    ref = Solver([m], mode="warp")
    ref.run(T)
    a, b = s.state_arrays(), ref.state_arrays()
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_queue_driver_batch_bitwise_equal_to_looped():
    """The queue driver (one launch, one global queue of every model's updates)
    on a batch of uneven models: bit for bit the looped driver's state."""
    models = [W.uneven_complete(n, 2, 50, seed=70 + n) for n in (2, 3, 6, 9, 13, 4)]
    models.append(W.knn(60, 5, 12, seed=1))
    a = Solver(models, mode="looped")
    b = Solver(models, mode="queue")
    assert b.info()["mode"] == "queue" and b.info()["grid"] > 0
    a.run(9)
    b.run(9)
    sa, sb = a.state_arrays(), b.state_arrays()
    assert np.array_equal(sa[1], sb[1]) and np.array_equal(sa[2], sb[2])
    b.run(4)  # continues from the state (versions reset per launch)
    a.run(4)
    sa, sb = a.state_arrays(), b.state_arrays()
    assert np.array_equal(sa[1], sb[1]) and np.array_equal(sa[2], sb[2])


def test_queue_driver_bounded_wait_times_out():
    m = W.complete(10, 8, seed=0)
    s = Solver([m], mode="queue", test_unreachable_wait=True, spin_limit=2000)
    s.run(3)
    with pytest.raises(MplppError) as ei:
        s.sync()
    assert ei.value.status == -4
    s.close()
    m2, _ = W.config(1)
    sol = oracle.solve(m2, _order(m2), 20)
    s2, D, _, _ = _solve_gpu([m2], 20, mode="queue")
    _check_D(D[0], sol["bound"])


@pytest.mark.parametrize("threads", [0, 64, 96])
@pytest.mark.parametrize("lmax", [8, 16, 32])
def test_resident_driver_bitwise_equal_to_looped(lmax, threads):
    """The resident driver (one CTA per model, its state in shared memory, a
    block barrier between matchings, groups of 8, 16 or 32 lanes per edge):
    bit for bit the looped driver's state, on uneven small models (label
    counts 1..lmax, odd and even n, a sparse graph with greedy colouring).
    With two or three warps a matching takes several rounds of edges per group,
    and some groups sit out the last round."""
    models = [W.uneven_complete(n, 1, lmax, seed=90 + n + lmax) for n in (2, 3, 7, 12, 21)]
    models.append(W.knn(40, 4, lmax, seed=5))
    a = Solver(models, mode="looped")
    b = Solver(models, mode="resident", threads=threads)
    inf = b.info()
    assert inf["mode"] == "resident" and inf["grid"] == len(models)
    if threads:
        assert inf["threads"] == threads
    for T in (5, 3):  # continues from the state
        a.run(T)
        b.run(T)
        sa, sb = a.state_arrays(), b.state_arrays()
        assert np.array_equal(sa[1], sb[1]) and np.array_equal(sa[2], sb[2])
    np.testing.assert_array_equal(a.bound(), b.bound())


def test_resident_driver_parity_K20_L8_replicas():
    """K_20, L = 8 (the small dense workload) and seeded replicas of it solved
    together by the resident driver, against the oracle."""
    models = [W.config(1, seed=k)[0] for k in range(3)]
    T = 40
    s, D, xs, en = _solve_gpu(models, T, mode="resident")
    for i, m in enumerate(models):
        sol = oracle.solve(m, _order(m), T)
        _check_D(D[i], sol["bound"])
        _check(s, models, i, xs[i], sol, en[i])


def test_resident_driver_rejects_large_labels():
    m = W.uneven_complete(5, 30, 40, seed=1)
    with pytest.raises(MplppError) as ei:
        Solver([m], mode="resident")
    assert ei.value.status == -7


def test_solvers_of_one_process_keep_their_shared_memory_limits():
    """A solver created later with smaller tables must not lower the shared
    memory limit of the kernels an earlier solver launches (the limit belongs
    to the kernel): the earlier solver still runs, in every driver."""
    big = W.uneven_complete(6, 200, 300, seed=3)
    small = W.uneven_complete(5, 2, 4, seed=4)
    for mode in ("looped", "persistent"):
        a = Solver([big], mode=mode)
        b = Solver([small], mode="looped", threads=64)
        c = Solver([small], mode="resident", threads=64)
        b.run(2)
        c.run(2)
        a.run(3)  # raised an invalid-argument launch error when the limit was lowered
        ref = Solver([big], mode=mode)
        ref.run(3)
        np.testing.assert_array_equal(a.bound(), ref.bound())
        for s in (a, b, c, ref):
            s.close()


def test_update_costs_from_pinned_host_memory_equals_pageable():
    """mplpp_update_costs reads pinned, mapped host arrays in place and copies
    pageable ones through a staging buffer: both give the same state, bit for
    bit, as a new solver with those costs."""
    import copy
    import torch
    m0 = W.uneven_complete(9, 20, 60, seed=31)
    rng = np.random.default_rng(32)
    m1 = copy.copy(m0)  # same shapes, other costs
    m1.unary = rng.standard_normal(np.asarray(m0.unary).shape).astype(np.float32)
    m1.pairwise = rng.standard_normal(np.asarray(m0.pairwise).shape).astype(np.float32)
    a = Solver([m0])
    b = Solver([m0])
    ref = Solver([m1])
    a.update_costs([np.ascontiguousarray(m1.unary)], [np.ascontiguousarray(m1.pairwise)])
    b.update_costs([torch.from_numpy(np.ascontiguousarray(m1.unary, np.float32)).pin_memory()],
                   [torch.from_numpy(np.ascontiguousarray(m1.pairwise, np.float32)).pin_memory()])
    for s in (a, b, ref):
        s.run(7)
    sa, sb, sr = a.state_arrays(), b.state_arrays(), ref.state_arrays()
    assert np.array_equal(sa[1], sr[1]) and np.array_equal(sb[1], sr[1])
    assert np.array_equal(sa[2], sr[2]) and np.array_equal(sb[2], sr[2])
    for s in (a, b, ref):
        s.close()
