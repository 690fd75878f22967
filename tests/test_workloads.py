"""Host-side checks of the synthetic workload generators that stand in for
the paper's density study (Sec. 7, random edge removal from the pose graphs)
and for the shape of its pose dataset (fully connected, L = 13)."""
import numpy as np
import pytest

from oracle import schedule as osched
from paper_2004_08227_gb300 import workloads as W


def _tables(m):
    L = m.labels
    off = np.concatenate([[0], np.cumsum(L[m.edge_u].astype(np.int64) * L[m.edge_v])])
    return {(int(u), int(v)): m.pairwise[off[e]:off[e + 1]] for e, (u, v) in enumerate(zip(m.edge_u, m.edge_v))}


def test_pose_sparse_keep_one_is_the_pose_model():
    a, b = W.pose_like(9, 6, seed=2), W.pose_sparse(1.0, 9, 6, seed=2)
    assert np.array_equal(a.edge_u, b.edge_u) and np.array_equal(a.edge_v, b.edge_v)
    assert np.array_equal(a.unary, b.unary) and np.array_equal(a.pairwise, b.pairwise)


@pytest.mark.parametrize("keep", [0.4, 0.1, 0.05])
def test_pose_sparse_restricts_the_complete_model(keep):
    """Every kept edge has its complete-model table; sparser models keep a
    subset of the edges of denser ones (one uniform draw per edge); the kept
    fraction is within 5 binomial standard deviations of keep."""
    n, L = 40, 5
    full = _tables(W.pose_like(n, L, seed=1))
    m = W.pose_sparse(keep, n, L, seed=1)
    sub = _tables(m)
    for k, t in sub.items():
        assert np.array_equal(t, full[k])
    denser = _tables(W.pose_sparse(min(1.0, 2 * keep), n, L, seed=1))
    assert set(sub) <= set(denser)
    E = len(full)
    assert abs(len(sub) - keep * E) <= 5 * np.sqrt(E * keep * (1 - keep)) + 1


@pytest.mark.parametrize("keep", [0.4, 0.05, 0.001])
def test_pose_sparse_greedy_schedule_is_valid(keep):
    m = W.pose_sparse(keep, 30, 3, seed=0)
    assert m.E >= 1 and m.schedule == "greedy_color"
    off, order = osched.build(m.schedule, m.n, m.edge_u, m.edge_v)
    assert osched.is_valid(m.n, m.E, m.edge_u, m.edge_v, off, order)


def test_pose_dense_shape():
    m = W.pose_dense(24, 13, seed=0)
    assert m.E == 24 * 23 // 2 and np.all(m.labels == 13) and m.schedule == "round_robin"
    assert m.pairwise.shape == (m.E * 169,)
    assert np.all((m.pairwise >= 0) & (m.pairwise <= 1))  # truncated quadratic costs
    off, _ = osched.build(m.schedule, m.n, m.edge_u, m.edge_v)
    assert len(off) - 1 == 23 and np.all(np.diff(off) == 12)


@pytest.mark.parametrize("quad", [False, True])
def test_grid_structured_costs_match_their_parameters(quad):
    """The dense tables of the stereo-like grid are w min(d, tau) (or
    w min(d^2, tau)) entry by entry, the product rounded once in float32 --
    the value the structured GPU path evaluates -- on a 4-connected grid with
    a valid greedy schedule."""
    rows, cols = 5, 7
    m = W.grid_trunc_linear(rows, cols, 9, 0.8, 5.0, seed=2, Lmin=3, quad=quad)
    assert m.pair_kind == ("trunc_quad" if quad else "trunc_linear")
    assert m.E == rows * (cols - 1) + (rows - 1) * cols and np.all(m.edge_u < m.edge_v)
    assert m.pair_param.shape == (m.E, 2) and m.pair_param.dtype == np.float32
    assert np.all(m.pair_param[:, 0] >= 0.4) and np.all(m.pair_param[:, 1] == 5.0)
    L = m.labels
    off = 0
    for e in range(m.E):
        Lu, Lv = int(L[m.edge_u[e]]), int(L[m.edge_v[e]])
        w, tau = m.pair_param[e]
        for s in range(Lu):
            for t in range(Lv):
                d = np.float32(abs(s - t))
                d = np.float32(d * d) if quad else d
                assert m.pairwise[off + s * Lv + t] == np.float32(w * np.float32(min(d, tau)))
        off += Lu * Lv
    assert off == m.pairwise.shape[0]
    off_m, order = osched.build(m.schedule, m.n, m.edge_u, m.edge_v)
    assert osched.is_valid(m.n, m.E, m.edge_u, m.edge_v, off_m, order)
