"""GPU backward: gradient of the dual bound after T iterations against the FP64
oracle's reverse-mode gradient and against FP64 central finite differences.

D_T is piecewise linear, so gradients are sums of +-2^-k.  The GPU backward
replays the iterations in FP64, so its argmins are those of the FP64 oracle
up to binary64 rounding order; the gradients are returned in FP32.
Tolerance: |g - g_ref| <= 1e-4 max(|g_ref|, 1e-3) (the stated 1e-4 relative,
with an absolute floor for entries near 0).
"""
import numpy as np
import pytest

import oracle
from oracle import schedule as osched
from paper_2004_08227_gb300 import workloads as W
from paper_2004_08227_gb300._lib import MplppError
from paper_2004_08227_gb300.solver import MPLPPBound, Solver

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _order(m):
    return osched.build(m.schedule, m.n, m.edge_u, m.edge_v)[1]


def _close(g, ref):
    return np.abs(g - ref) <= TOL * np.maximum(np.abs(ref), 1e-3)


@pytest.mark.parametrize("T,k", [(0, 1), (1, 1), (6, 2), (9, 4)])
@pytest.mark.parametrize("mode", ["looped", "persistent"])
def test_grad_matches_oracle_small(T, k, mode):
    m = W.uneven_complete(7, 2, 19, seed=T * 3 + k)
    Do, gu_o, gp_o = oracle.grad(m, _order(m), T)
    s = Solver([m], record_every=k, mode=mode)
    s.run(T)
    D = s.bound()[0]
    gu, gp = s.backward()
    assert abs(D - Do) <= 1e-5 * max(1.0, abs(Do))
    assert np.all(_close(gu, gu_o)), np.abs(gu - gu_o).max()
    assert np.all(_close(gp, gp_o)), np.abs(gp - gp_o).max()


def test_grad_batch_and_weights():
    """Several models in one solver; dD weights scale each model's gradient."""
    models = [W.complete(6, 5, seed=s, pairwise="normal") for s in range(3)]
    s = Solver(models, record_every=3)
    s.run(7)
    w = np.asarray([1.0, -2.0, 0.5], np.float32)
    gu, gp = s.backward(w)
    uo = po = 0
    for i, m in enumerate(models):
        _, a, b = oracle.grad(m, _order(m), 7)
        assert np.all(_close(gu[uo:uo + a.size], w[i] * a))
        assert np.all(_close(gp[po:po + b.size], w[i] * b))
        uo += a.size
        po += b.size


def test_grad_sums_to_one_per_factor_on_gpu():
    m = W.complete(10, 12, seed=3, pairwise="normal")
    s = Solver([m], record_every=5)
    s.run(12)
    gu, gp = s.backward()
    g = oracle.Graph.of(m)
    for u in range(m.n):
        assert abs(gu[g.uoff[u]:g.uoff[u + 1]].sum() - 1.0) < 1e-5
    for e in range(m.E):
        assert abs(gp[g.poff[e]:g.poff[e + 1]].sum() - 1.0) < 1e-5


def test_autograd_function():
    import torch
    graphs = [W.complete(6, 7, seed=s, pairwise="normal") for s in range(2)]
    un = torch.tensor(np.concatenate([g.unary for g in graphs]), device="cuda", requires_grad=True)
    pw = torch.tensor(np.concatenate([g.pairwise for g in graphs]), device="cuda", requires_grad=True)
    D = MPLPPBound.apply(un, pw, graphs, 8, 3)
    (D * torch.tensor([1.0, 3.0], dtype=torch.float64, device="cuda")).sum().backward()
    uo = po = 0
    for i, m in enumerate(graphs):
        Do, a, b = oracle.grad(m, _order(m), 8)
        assert abs(D[i].item() - Do) <= 1e-5 * max(1.0, abs(Do))
        w = [1.0, 3.0][i]
        assert np.all(_close(un.grad[uo:uo + a.size].cpu().numpy(), w * a))
        assert np.all(_close(pw.grad[po:po + b.size].cpu().numpy(), w * b))
        uo += a.size
        po += b.size


def test_backward_requires_record():
    m = W.complete(5, 3, seed=0)
    s = Solver([m])
    s.run(2)
    with pytest.raises(MplppError) as ei:
        s.backward()
    assert ei.value.status == -6


def _fd3(m, order, T, which, i, h):
    """D_T at +h, -h and 0 along one coordinate (FP64 oracle)."""
    un = m.unary.astype(np.float64)
    pw = m.pairwise.astype(np.float64)
    vals = []
    for d in (h, -h, 0.0):
        u2, p2 = un.copy(), pw.copy()
        (u2 if which == "u" else p2)[i] += d
        th_u, th_uv = oracle.run(m, order, T, state=(u2, p2))
        vals.append(oracle.bound(m, th_u, th_uv))
    return vals


def test_grad_K50_L64_matches_oracle_and_central_differences():
    """Differentiation workload shape (K_50, L = 64, N(0,1) pairwise, T = 50,
    checkpoints every 10) on one model: the GPU gradient equals the oracle's
    reverse-mode gradient on every entry, and FP64 central differences
    (h = 1e-4) of the oracle's D_T on sampled entries, half of them where the
    gradient is non-zero.  Where the one-sided differences disagree there is a
    kink within h (D_T is piecewise linear) and the step shrinks to 1e-5, then
    1e-6; at most a quarter of the samples may have a kink at every step."""
    m = W.complete(50, 64, seed=0, pairwise="normal")
    T = 50
    order = _order(m)
    s = Solver([m], record_every=10)
    s.run(T)
    gu, gp = s.backward()
    _, gu_o, gp_o = oracle.grad(m, order, T)
    assert np.all(_close(gu, gu_o)), np.abs(gu - gu_o).max()
    assert np.all(_close(gp, gp_o)), np.abs(gp - gp_o).max()
    rng = np.random.default_rng(1)
    nz = np.flatnonzero(gp_o)
    picks = [("p", int(i)) for i in rng.choice(nz, size=6, replace=False)]
    picks += [("p", int(i)) for i in rng.choice(gp_o.size, size=2, replace=False)]
    picks += [("u", int(i)) for i in rng.choice(gu_o.size, size=4, replace=False)]
    checked = 0
    for which, i in picks:
        for h in (1e-4, 1e-5, 1e-6):
            fp, fm, f0 = _fd3(m, order, T, which, i, h)
            fd = (fp - fm) / (2 * h)
            if abs((fp - f0) / h - (f0 - fm) / h) > TOL * max(abs(fd), 1e-3):
                continue  # kink within h: try a smaller step
            g = (gu if which == "u" else gp)[i]
            assert abs(g - fd) <= TOL * max(abs(fd), 1e-3), (which, i, h, g, fd)
            checked += 1
            break
    assert checked >= 3 * len(picks) // 4


@pytest.mark.parametrize("case", ["uneven", "integer_ties", "pose_truncated", "wide_rows"])
def test_screened_replay_equals_all_fp64_replay_bitwise(case):
    """The backward's replay screens every minimization in FP32 and evaluates
    only the candidates its error bound admits in FP64; its argmins, and so
    the gradient, must equal those of the replay that evaluates every entry in
    FP64, bit for bit -- also with exact ties (integer costs), the truncated
    pose costs (most entries exactly 1.0) and rows wider than a warp."""
    if case == "uneven":
        m, T = W.uneven_complete(9, 1, 70, seed=12), 12
    elif case == "integer_ties":
        m, T = W.uneven_complete(8, 3, 17, seed=4), 10
        m.unary[:] = np.round(4 * m.unary)
        m.pairwise[:] = np.round(3 * m.pairwise)
    elif case == "pose_truncated":
        m, T = W.pose_like(6, 120, seed=2), 8
    else:
        m, T = W.uneven_complete(4, 150, 260, seed=3), 4
    grads = []
    for fp64 in (False, True):
        s = Solver([m], record_every=3, test_fp64_replay=fp64)
        s.run(T)
        grads.append(s.backward())
        s.close()
    assert np.array_equal(grads[0][0], grads[1][0]) and np.array_equal(grads[0][1], grads[1][1])
    _, gu_o, gp_o = oracle.grad(m, _order(m), T)
    if case in ("uneven", "wide_rows"):  # tie-free costs: the oracle's argmins too
        assert np.all(_close(grads[0][0], gu_o)) and np.all(_close(grads[0][1], gp_o))


@pytest.mark.parametrize("T,k", [(7, 3), (10, 10), (5, 1)])
def test_checkpointed_replay_equals_one_pass_replay_bitwise(T, k):
    """Records of every iteration in one replay, or state checkpoints every k
    iterations and a second replay per segment: the same gradient bit for bit."""
    m = W.uneven_complete(8, 2, 40, seed=T + 10 * k)
    grads = []
    for ck in (False, True):
        s = Solver([m], record_every=k, test_checkpoints=ck)
        s.run(T)
        grads.append(s.backward())
        s.close()
    assert np.array_equal(grads[0][0], grads[1][0]) and np.array_equal(grads[0][1], grads[1][1])
