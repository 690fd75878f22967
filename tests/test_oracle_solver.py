"""Pins of the oracle's iteration, dual bound, rounding and energy."""
import numpy as np
import pytest

import oracle
from oracle import schedule as osched
from paper_2004_08227_gb300 import workloads as W

from _brute import map_energy


def _order(model):
    off, order = osched.build(model.schedule, model.n, model.edge_u, model.edge_v)
    return order


def test_energy_invariant_under_reparametrization():
    """Sec. 3 (Dual Problem): E(y|theta) = E(y|theta^phi) for every labeling."""
    m = W.tiny(6, 4, seed=1, density=0.7, uneven=True)
    th_u, th_uv = oracle.run(m, _order(m), 5)
    rng = np.random.default_rng(0)
    for _ in range(50):
        y = np.asarray([rng.integers(0, l) for l in m.labels], np.int32)
        assert abs(oracle.energy(m, y) - oracle.energy(m, y, th_u, th_uv)) < 1e-9


@pytest.mark.parametrize("seed", range(4))
def test_dual_monotone(seed):
    """Lemma B.4: D never decreases along the iterations of MPLP++."""
    m = W.complete(8, 5, seed=seed, pairwise="normal")
    D0 = oracle.bound(m, m.unary, m.pairwise)
    _, _, hist = oracle.run(m, _order(m), 30, history=True)
    seq = np.concatenate([[D0], hist])
    assert np.all(np.diff(seq) >= -1e-12 * np.abs(seq[1:]).max())
    assert seq[-1] > seq[0]


@pytest.mark.parametrize("seed", range(12))
def test_bound_below_brute_force_map(seed):
    """Eq. LP-lower-bound: D(theta^phi) <= E(y) for all y, in particular the
    MAP energy found by enumeration (n <= 5, L <= 3)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 6))
    m = W.tiny(n, 3, seed=seed, density=0.8, uneven=bool(seed % 2),
               pairwise="normal" if seed % 3 else "uniform")
    Emap, _ = map_energy(m)
    th_u, th_uv, hist = oracle.run(m, _order(m), 20, history=True)
    assert np.all(hist <= Emap + 1e-9)


@pytest.mark.parametrize("seed", range(6))
def test_single_edge_exact_after_one_update(seed):
    """Prop. 1 with a single edge: after one update D = min g = MAP energy,
    and the rounding returns a MAP labeling."""
    rng = np.random.default_rng(seed)
    Lu, Lv = int(rng.integers(1, 7)), int(rng.integers(1, 7))
    m = W.Model(np.asarray([Lu, Lv], np.int32), np.asarray([0], np.int32), np.asarray([1], np.int32),
                rng.random(Lu + Lv).astype(np.float32), rng.standard_normal(Lu * Lv).astype(np.float32))
    Emap, _ = map_energy(m)
    for rule in ("H", "M"):
        th_u, th_uv = oracle.run(m, [0], 1, rule=rule)
        assert abs(oracle.bound(m, th_u, th_uv) - Emap) < 1e-9
    th_u, th_uv = oracle.run(m, [0], 1)
    x = oracle.round_labels(m, th_u, th_uv)
    assert abs(oracle.energy(m, x) - Emap) < 1e-9


@pytest.mark.parametrize("seed", range(6))
def test_one_iteration_dominance(seed):
    """Thm. 2 (with Prop. 2, 3): from the same start and order, one H-iteration
    gives D >= one M-iteration >= one U-iteration."""
    m = W.tiny(6, 4, seed=100 + seed, density=0.8, pairwise="normal")
    order = _order(m)
    D = {r: oracle.bound(m, *oracle.run(m, order, 1, rule=r)) for r in "UMH"}
    assert D["H"] >= D["M"] - 1e-12 and D["M"] >= D["U"] - 1e-12


@pytest.mark.parametrize("kind,seed", [("path", 0), ("path", 1), ("star", 2), ("star", 3)])
def test_trees_reach_map(kind, seed):
    """Derived (not stated in the paper): on trees the LP relaxation is tight
    and node-edge agreement (Thm. 1) yields a labeling with E = D, so D
    approaches the brute-force MAP energy, and the rounding finds a MAP
    labeling."""
    m = W.tree(5, 3, seed=seed, kind=kind)
    Emap, _ = map_energy(m)
    th_u, th_uv = oracle.run(m, _order(m), 200)
    assert abs(oracle.bound(m, th_u, th_uv) - Emap) < 1e-6
    x = oracle.round_labels(m, th_u, th_uv)
    assert abs(oracle.energy(m, x) - Emap) < 1e-6


def test_rounding_without_pairwise_is_unary_argmin():
    """Special case: with zero pairwise costs the rounding objective is the
    unary alone, so x_u = argmin_s theta_u(s) (lowest index on ties)."""
    m = W.tiny(6, 5, seed=4, density=1.0, uneven=True)
    m.pairwise[:] = 0
    x = oracle.round_labels(m, m.unary, m.pairwise)
    uoff = np.concatenate([[0], np.cumsum(m.labels)])
    for u in range(m.n):
        assert x[u] == int(np.argmin(m.unary[uoff[u]:uoff[u + 1]]))


@pytest.mark.parametrize("seed", range(5))
def test_rounding_energy_above_bound(seed):
    """Any labeling, in particular the rounded one, has E >= D."""
    m = W.tiny(6, 4, seed=200 + seed, density=0.9, uneven=True, pairwise="normal")
    sol = oracle.solve(m, _order(m), 10)
    assert sol["energy"] >= sol["bound"] - 1e-9
    Emap, _ = map_energy(m)
    assert sol["energy"] >= Emap - 1e-9


def test_rounding_uses_earlier_neighbours_only():
    """Node 0 is rounded on its unary alone (it has no earlier neighbour)."""
    m = W.tiny(4, 3, seed=8, density=1.0, pairwise="normal")
    x = oracle.round_labels(m, m.unary, m.pairwise)
    assert x[0] == int(np.argmin(m.unary[:3]))


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_run_parallel_equals_run_bitwise(threads):
    """Sec. 6: the edges of one matching share no node, so updating them on
    several threads gives the sequential result exactly."""
    m = W.uneven_complete(11, 2, 9, seed=5)
    off, order = osched.build(m.schedule, m.n, m.edge_u, m.edge_v)
    a = oracle.run(m, order, 4)
    b = oracle.run_parallel(m, off, order, 4, threads=threads)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert oracle.max_threads() >= 1


def test_run_parallel_rejects_a_matching_that_repeats_a_node():
    m = W.uneven_complete(5, 2, 3, seed=1)
    off, order = osched.build(m.schedule, m.n, m.edge_u, m.edge_v)
    with pytest.raises(ValueError):
        oracle.run_parallel(m, [0, len(order)], order, 1)
