"""Pins of the oracle's reverse-mode gradient of D after T H-iterations.

D_T is piecewise linear in the costs; away from kinks FP64 central differences
are exact up to rounding, so they pin the gradient (kinks are detected by
disagreeing one-sided differences and skipped)."""
import numpy as np
import pytest

import oracle
from oracle import schedule as osched
from paper_2004_08227_gb300 import workloads as W


def _DT(model, order, T, unary, pairwise):
    m = W.Model(model.labels, model.edge_u, model.edge_v, unary, pairwise)
    # the oracle converts to FP64; pass FP64 copies so perturbations survive
    th_u, th_uv = oracle.run(m, order, T, state=(unary, pairwise))
    return oracle.bound(m, th_u, th_uv)


@pytest.mark.parametrize("seed,T", [(0, 1), (1, 3), (2, 6)])
def test_grad_matches_central_differences(seed, T):
    m = W.tiny(5, 3, seed=seed, density=0.9, uneven=True, pairwise="normal")
    _, order = osched.build(m.schedule, m.n, m.edge_u, m.edge_v)
    D, gu, guv = oracle.grad(m, order, T)
    un = m.unary.astype(np.float64)
    pw = m.pairwise.astype(np.float64)
    assert abs(D - _DT(m, order, T, un, pw)) < 1e-12
    h = 1e-6
    checked = 0
    for which, base, g in (("u", un, gu), ("p", pw, guv)):
        for i in range(base.shape[0]):
            def f(d):
                b = base.copy()
                b[i] += d
                return _DT(m, order, T, b, pw) if which == "u" else _DT(m, order, T, un, b)
            f0, fp, fm = f(0.0), f(h), f(-h)
            right, left = (fp - f0) / h, (f0 - fm) / h
            if abs(right - left) > 1e-6:
                continue  # kink
            fd = (fp - fm) / (2 * h)
            assert abs(fd - g[i]) < 1e-6, (which, i, fd, g[i])
            checked += 1
    assert checked >= 0.8 * (un.shape[0] + pw.shape[0])


@pytest.mark.parametrize("seed", range(3))
def test_grad_sums_to_one_per_factor(seed):
    """Adding a constant c to one unary vector (or one table) shifts every
    later state by constants and D_T by exactly c (each update maps g + c to
    outputs whose shifts add up to c), so the gradient sums to 1 over every
    unary vector and over every pairwise table."""
    m = W.complete(6, 4, seed=seed, pairwise="normal")
    _, order = osched.round_robin(m.n, m.edge_u, m.edge_v)
    _, gu, guv = oracle.grad(m, order, 5)
    g = oracle.Graph.of(m)
    for u in range(m.n):
        assert abs(gu[g.uoff[u]:g.uoff[u + 1]].sum() - 1.0) < 1e-12
    for e in range(m.E):
        assert abs(guv[g.poff[e]:g.poff[e + 1]].sum() - 1.0) < 1e-12


def test_grad_T0_is_argmin_indicator():
    """With no iteration, D is the plain sum of minima: its gradient is the
    indicator of each (lowest-index) argmin."""
    m = W.tiny(4, 3, seed=5, density=1.0, pairwise="normal")
    _, order = osched.build(m.schedule, m.n, m.edge_u, m.edge_v)
    D, gu, guv = oracle.grad(m, order, 0)
    g = oracle.Graph.of(m)
    for u in range(m.n):
        seg = m.unary[g.uoff[u]:g.uoff[u + 1]]
        want = np.zeros_like(seg, dtype=np.float64)
        want[np.argmin(seg)] = 1
        assert np.array_equal(gu[g.uoff[u]:g.uoff[u + 1]], want)
