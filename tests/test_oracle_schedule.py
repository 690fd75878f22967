"""Pins of the oracle's edge schedules (Sec. 6, Alg. 1)."""
import numpy as np
import pytest

from oracle import schedule as osched
from paper_2004_08227_gb300 import workloads as W


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 19, 20, 21, 60])
def test_round_robin_is_a_one_factorization(n):
    """Even n: n-1 perfect matchings of n/2 edges; odd n: n matchings of
    (n-1)/2 edges; every edge exactly once."""
    m = W.complete(n, 1, seed=0)
    off, order = osched.round_robin(n, m.edge_u, m.edge_v)
    assert osched.is_valid(n, m.E, m.edge_u, m.edge_v, off, order)
    sizes = np.diff(off)
    if n % 2 == 0:
        assert len(sizes) == n - 1 and np.all(sizes == n // 2)
    else:
        assert len(sizes) == n and np.all(sizes == (n - 1) // 2)


@pytest.mark.parametrize("seed", range(5))
def test_greedy_color_valid_and_bounded(seed):
    m = W.tiny(30, 1, seed=seed, density=0.3)
    off, order = osched.greedy_color(m.n, m.edge_u, m.edge_v)
    assert osched.is_valid(m.n, m.E, m.edge_u, m.edge_v, off, order)
    deg = np.bincount(np.concatenate([m.edge_u, m.edge_v]), minlength=m.n)
    assert len(off) - 1 <= 2 * deg.max() - 1


def test_greedy_color_path_two_colours():
    m = W.tree(9, 1, seed=0, kind="path")
    off, order = osched.greedy_color(m.n, m.edge_u, m.edge_v)
    assert len(off) - 1 == 2


@pytest.mark.parametrize("seed", range(5))
def test_alg1_matchings_are_maximal(seed):
    """Alg. 1: each pushed matching is maximal among the edges remaining."""
    m = W.tiny(25, 1, seed=seed, density=0.4)
    off, order = osched.alg1(m.n, m.edge_u, m.edge_v)
    assert osched.is_valid(m.n, m.E, m.edge_u, m.edge_v, off, order)
    remaining = set(range(m.E))
    for k in range(len(off) - 1):
        mk = set(order[off[k]:off[k + 1]].tolist())
        busy = set(m.edge_u[list(mk)].tolist()) | set(m.edge_v[list(mk)].tolist())
        for e in remaining - mk:
            assert m.edge_u[e] in busy or m.edge_v[e] in busy
        remaining -= mk


def test_validator_rejects_bad_schedules():
    m = W.complete(4, 1, seed=0)
    off, order = osched.round_robin(4, m.edge_u, m.edge_v)
    bad = order.copy()
    bad[0], bad[2] = bad[2], bad[0]  # moves an edge into a matching that shares a node
    assert not osched.is_valid(4, m.E, m.edge_u, m.edge_v, off, bad)
    assert not osched.is_valid(4, m.E, m.edge_u, m.edge_v, off, order[:-1])
