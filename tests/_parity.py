"""Parity checks of the GPU solver's state and labels against the FP64 oracle.

State (Sec. 3, eq. reparametrization): the GPU keeps theta^phi_u per node
(``agg``) and the messages of every edge (``msg``); the oracle keeps the
reparametrized costs themselves (table form).  ``check_state`` compares
theta^phi_u entry by entry, each node against its own scale (the largest
magnitude of its oracle vector, at least 1); ``check_tables`` compares the
implied reparametrized tables theta_uv - phi_{v->u} - phi_{u->v} with the
oracle's tables entry by entry, each edge against its own scale (its table,
messages and end nodes: see check_tables).

Labels (Sec. 4, Primal Rounding): the rounding decides node u on
obj_u(s) = theta^phi_u(s) + sum over earlier neighbours v of theta^phi_vu(x_v, s).
After a first difference the two labelings condition later nodes on different
labels, so comparing labels position by position says little.
``check_labels`` therefore evaluates, for EVERY node, the oracle's objective
conditioned on the GPU's own earlier labels and requires the GPU's choice to be
within twice the FP32 error bound of that objective's minimum:
    gap_u = obj_u(x_u) - min_s obj_u(s) <= 2 eps_u,
    eps_u = RTOL_STATE * (max|theta^phi_u| + sum over the in-edges of max|row|),
the error that entries within RTOL_STATE of their scale can put into a sum of
those terms.  It reports how many labels differ from the conditional argmin and
from the oracle's own labeling.
"""
from __future__ import annotations

import numpy as np

RTOL_STATE = 1e-5


def offsets(m):
    """Per-node offsets of the unary layout and per-edge offsets of the table
    and message layouts of one model (the caller's unpadded layouts)."""
    L = np.asarray(m.labels, np.int64)
    eu, ev = np.asarray(m.edge_u), np.asarray(m.edge_v)
    uoff = np.concatenate([[0], np.cumsum(L)])
    poff = np.concatenate([[0], np.cumsum(L[eu] * L[ev])])
    moff = np.concatenate([[0], np.cumsum(L[eu] + L[ev])])
    return uoff, poff, moff


def split_state(models, agg, msg):
    """Per-model (agg, msg) views of a batched solver's saved state."""
    out, ua, mb = [], 0, 0
    for m in models:
        uoff, _, moff = offsets(m)
        out.append((agg[ua:ua + uoff[-1]], msg[mb:mb + moff[-1]]))
        ua += uoff[-1]
        mb += moff[-1]
    return out


def model_state(solver, models, i):
    """(agg, msg) of model i from the solver's saved state (FP64, exact)."""
    _, agg, msg = solver.state_arrays()
    return split_state(models, agg, msg)[i]


def check_state(m, agg, th_u, rtol=RTOL_STATE, nodes=None, what=""):
    """theta^phi_u of the GPU (agg) against the oracle's (th_u), node by node.
    nodes: restrict to these node ids, with th_u then holding only their
    vectors concatenated in that order.  Returns the largest error relative
    to the node's scale."""
    uoff, _, _ = offsets(m)
    worst = 0.0
    ids = range(m.n) if nodes is None else nodes
    k = 0
    for u in ids:
        g = agg[uoff[u]:uoff[u + 1]]
        if nodes is None:
            o = th_u[uoff[u]:uoff[u + 1]]
        else:
            o = th_u[k:k + len(g)]
            k += len(g)
        scale = max(1.0, float(np.max(np.abs(o))))
        err = float(np.max(np.abs(g - o))) / scale
        worst = max(worst, err)
        assert err <= rtol, f"{what} node {u}: theta^phi_u differs by {err:.3g} of its scale {scale:.3g}"
    return worst


def gpu_table(m, msg, e, poff=None, moff=None):
    """Reparametrized table of edge e implied by the GPU state (FP64):
    theta_uv(s, t) - phi_{v->u}(s) - phi_{u->v}(t)."""
    if poff is None:
        _, poff, moff = offsets(m)
    Lu, Lv = int(m.labels[m.edge_u[e]]), int(m.labels[m.edge_v[e]])
    tab = np.asarray(m.pairwise[poff[e]:poff[e + 1]], np.float64).reshape(Lu, Lv)
    pu = msg[moff[e]:moff[e] + Lu]
    pv = msg[moff[e] + Lu:moff[e + 1]]
    return (tab - pu[:, None]) - pv[None, :]


def check_tables(m, msg, th_uv, agg, rtol=RTOL_STATE, what=""):
    """Every implied reparametrized table entry against the oracle's table,
    each edge against its own scale, at least 1: the largest magnitude among
    the original table, the oracle's table, the edge's messages and the
    reparametrized unaries of its two end nodes.  An entry is
    theta_uv - phi_{v->u} - phi_{u->v}, and a message is the difference of two
    quantities of its end node's scale (Sec. 4: phi_{v->u} = c - uh), so the
    rounding error of an entry scales with its end nodes.  Returns the largest
    relative error."""
    uoff, poff, moff = offsets(m)
    worst = 0.0
    for e in range(m.E):
        g = gpu_table(m, msg, e, poff, moff)
        o = th_uv[poff[e]:poff[e + 1]].reshape(g.shape)
        a, b = int(m.edge_u[e]), int(m.edge_v[e])
        scale = max(1.0, float(np.max(np.abs(o))),
                    float(np.max(np.abs(np.asarray(m.pairwise[poff[e]:poff[e + 1]], np.float64)))),
                    float(np.max(np.abs(msg[moff[e]:moff[e + 1]]))),
                    float(np.max(np.abs(agg[uoff[a]:uoff[a + 1]]))),
                    float(np.max(np.abs(agg[uoff[b]:uoff[b + 1]]))))
        err = float(np.max(np.abs(g - o))) / scale
        worst = max(worst, err)
        assert err <= rtol, f"{what} edge {e}: reparametrized table differs by {err:.3g} of its scale {scale:.3g}"
    return worst


def in_edges(m):
    """For every node u its in-edges (v, e) with v < u, by increasing v."""
    ins = [[] for _ in range(m.n)]
    for e, (a, b) in enumerate(zip(np.asarray(m.edge_u).tolist(), np.asarray(m.edge_v).tolist())):
        ins[b].append((a, e))
    for lst in ins:
        lst.sort()
    return ins


def check_labels(m, th_u, th_uv, x, x_oracle=None, rtol=RTOL_STATE, what=""):
    """The conditional check described in the module docstring.  Returns
    {"nodes", "differ_conditional", "differ_oracle", "worst_gap_over_eps"}."""
    uoff, poff, _ = offsets(m)
    L = np.asarray(m.labels)
    ins = in_edges(m)
    x = np.asarray(x)
    differ = 0
    worst = 0.0
    for u in range(m.n):
        Lu = int(L[u])
        obj = np.array(th_u[uoff[u]:uoff[u + 1]], np.float64)
        scale = float(np.max(np.abs(obj)))
        for v, e in ins[u]:
            row = th_uv[poff[e] + int(x[v]) * Lu:poff[e] + (int(x[v]) + 1) * Lu]
            obj = obj + row
            scale += float(np.max(np.abs(row)))
        best = int(np.argmin(obj))
        eps = rtol * max(1.0, scale)
        gap = float(obj[int(x[u])] - obj[best])
        if int(x[u]) != best:
            differ += 1
        worst = max(worst, gap / eps)
        assert gap <= 2 * eps, (f"{what} node {u}: label {int(x[u])} is {gap:.3g} above the minimum of the "
                                f"oracle's objective (label {best}); allowed 2 x {eps:.3g}")
    res = {"nodes": int(m.n), "differ_conditional": differ, "worst_gap_over_eps": worst,
           "differ_oracle": None if x_oracle is None else int(np.sum(np.asarray(x_oracle) != x))}
    print(f"{what} labels: {res}")
    return res


def first_divergence(x, x_oracle, margins, eps, what=""):
    """Full-size form when the oracle's state is not at hand: up to the first
    differing node both labelings are decided on the same objective, so that
    node's oracle margin must be within 2 eps of it.  Returns the number of
    differing labels."""
    x, xo = np.asarray(x), np.asarray(x_oracle)
    diff = np.flatnonzero(x != xo)
    if diff.size:
        u = int(diff[0])
        assert margins[u] <= 2 * eps[u], (f"{what} first differing node {u}: oracle margin {margins[u]:.3g} "
                                          f"above 2 x {eps[u]:.3g}")
    print(f"{what} labels differing from the oracle's: {int(diff.size)} of {x.size}")
    return int(diff.size)


def objective_eps(m, agg, msg, x, rtol=RTOL_STATE):
    """eps_u (module docstring) from a state given in message form, for the
    objective conditioned on labels x."""
    uoff, poff, moff = offsets(m)
    L = np.asarray(m.labels)
    ins = in_edges(m)
    eps = np.zeros(m.n)
    for u in range(m.n):
        Lu = int(L[u])
        scale = float(np.max(np.abs(agg[uoff[u]:uoff[u + 1]])))
        for v, e in ins[u]:
            Lv_ = int(L[v])
            tab = np.asarray(m.pairwise[poff[e]:poff[e + 1]], np.float64).reshape(Lv_, Lu)
            row = tab[int(x[v])] - msg[moff[e] + int(x[v])] - msg[moff[e] + Lv_:moff[e + 1]]
            scale += float(np.max(np.abs(row)))
        eps[u] = rtol * max(1.0, scale)
    return eps
