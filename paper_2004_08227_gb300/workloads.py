"""Seeded synthetic workloads for MPLP++ (dense pairwise graphical models).

This module only draws inputs: it holds none of the method's arithmetic, and
both the CUDA path and the FP64 oracle consume what it returns.  Costs are
drawn in FP64 with ``numpy.random.default_rng(seed)`` and rounded once to FP32;
the FP32 values are what both sides see.

The paper's own datasets (protein, pose, worms; Sec. 7) are not available; the
shapes below stand in for them:

  complete(n, L)   K_n, uniform labels, unary U[0,1), pairwise U[0,1) or N(0,1)
  pose_like()      K_60, L=300; label s of node u is a point p_us in [0,1]^3,
                   edge distance D_uv ~ U[0.1, 1], pairwise
                   min(((|p_us - p_vt| - D_uv) / 0.05)^2, 1), unary U[0,1)
  knn()            n points in [0,1]^3, each linked to its k nearest neighbours
                   (union, so degrees vary), L labels, unary U, pairwise N(0,1)
  batch()          many complete graphs, n ~ U{10..80}, per-node L ~ U{16..128}
  tiny()/tree()    small random models for brute-force checks
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Model:
    """One pairwise model.  Edges satisfy u < v; unary is concatenated node by
    node; pairwise concatenates the row-major L_u x L_v tables in edge order."""
    labels: np.ndarray          # int32 [n]
    edge_u: np.ndarray          # int32 [E]
    edge_v: np.ndarray          # int32 [E]
    unary: np.ndarray           # float32 [sum L]
    pairwise: np.ndarray        # float32 [sum L_u L_v]
    schedule: str = "greedy_color"
    name: str = ""
    meta: dict = field(default_factory=dict)
    pair_kind: str = "dense"    # "trunc_linear": pairwise(s,t) = w_e min(|s - t|, tau_e); "trunc_quad":
                                # w_e min((s - t)^2, tau_e) (both also given densely in pairwise)
    pair_param: np.ndarray = None  # float32 [E, 2]: (w_e, tau_e) for the structured kinds

    @property
    def n(self) -> int:
        return int(self.labels.shape[0])

    @property
    def E(self) -> int:
        return int(self.edge_u.shape[0])

    def table_sizes(self) -> np.ndarray:
        return self.labels[self.edge_u].astype(np.int64) * self.labels[self.edge_v].astype(np.int64)

    def bytes_per_iteration(self) -> int:
        """Algorithmic HBM bytes of one iteration of the message-form update:
        each FP32 table read once (4 B/entry) + the FP64 agg and message
        vectors read and written (32 B per label of each endpoint)."""
        Lu = self.labels[self.edge_u].astype(np.int64)
        Lv = self.labels[self.edge_v].astype(np.int64)
        return int(np.sum(4 * Lu * Lv + 32 * (Lu + Lv)))


def _complete_edges(n: int):
    iu, iv = np.triu_indices(n, k=1)
    return iu.astype(np.int32), iv.astype(np.int32)


def _draw_pairwise(rng, sizes, dist: str) -> np.ndarray:
    total = int(np.sum(sizes))
    out = np.empty(total, np.float32)
    chunk = 1 << 24
    for s in range(0, total, chunk):
        m = min(chunk, total - s)
        if dist == "uniform":
            out[s:s + m] = rng.random(m)
        else:
            out[s:s + m] = rng.standard_normal(m)
    return out


def complete(n: int, L: int, seed: int = 0, pairwise: str = "uniform") -> Model:
    """K_n with L labels per node; unary U[0,1); pairwise U[0,1) or N(0,1)."""
    rng = np.random.default_rng(seed)
    eu, ev = _complete_edges(n)
    labels = np.full(n, L, np.int32)
    unary = rng.random(n * L).astype(np.float32)
    pw = _draw_pairwise(rng, labels[eu].astype(np.int64) * labels[ev], pairwise)
    return Model(labels, eu, ev, unary, pw, schedule="round_robin",
                 name=f"K{n}_L{L}_{pairwise}_s{seed}")


def pose_like(n: int = 60, L: int = 300, seed: int = 0, sigma: float = 0.05) -> Model:
    """Pose-shaped dense model: truncated quadratic distance-consistency costs."""
    rng = np.random.default_rng(seed)
    eu, ev = _complete_edges(n)
    labels = np.full(n, L, np.int32)
    unary = rng.random(n * L).astype(np.float32)
    pts = rng.random((n, L, 3))
    Duv = rng.uniform(0.1, 1.0, size=eu.shape[0])
    pw = np.empty(eu.shape[0] * L * L, np.float32)
    for e in range(eu.shape[0]):
        d = np.linalg.norm(pts[eu[e]][:, None, :] - pts[ev[e]][None, :, :], axis=2)
        c = np.minimum(((d - Duv[e]) / sigma) ** 2, 1.0)
        pw[e * L * L:(e + 1) * L * L] = c.ravel()
    return Model(labels, eu, ev, unary, pw, schedule="round_robin",
                 name=f"pose_K{n}_L{L}_s{seed}")


def _pose_tables(pts: np.ndarray, eu: np.ndarray, ev: np.ndarray, Duv: np.ndarray, sigma: float,
                 block: int = 4096) -> np.ndarray:
    """Truncated quadratic distance-consistency tables of the given edges,
    min(((|p_us - p_vt| - D_uv) / sigma)^2, 1), row-major, in blocks of edges."""
    L = pts.shape[1]
    out = np.empty(eu.shape[0] * L * L, np.float32)
    for s in range(0, eu.shape[0], block):
        e = slice(s, min(s + block, eu.shape[0]))
        d = np.linalg.norm(pts[eu[e]][:, :, None, :] - pts[ev[e]][:, None, :, :], axis=3)
        c = np.minimum(((d - Duv[e, None, None]) / sigma) ** 2, 1.0)
        out[s * L * L:e.stop * L * L] = c.ravel()
    return out


def pose_sparse(keep: float, n: int = 60, L: int = 300, seed: int = 0, sigma: float = 0.05) -> Model:
    """The pose-shaped model with every edge kept with probability `keep`
    (random sparsification, as in the paper's density study, Sec. 7), scheduled
    by greedy edge colouring.  Points, distances and unaries are drawn as in
    pose_like, so a kept edge has the table it has in the complete model."""
    rng = np.random.default_rng(seed)
    eu, ev = _complete_edges(n)
    labels = np.full(n, L, np.int32)
    unary = rng.random(n * L).astype(np.float32)
    pts = rng.random((n, L, 3))
    Duv = rng.uniform(0.1, 1.0, size=eu.shape[0])
    kept = np.random.default_rng(seed + 7919).random(eu.shape[0]) < keep
    if not kept.any():
        kept[0] = True
    eu, ev, Duv = eu[kept], ev[kept], Duv[kept]
    return Model(labels, eu.astype(np.int32), ev.astype(np.int32), unary, _pose_tables(pts, eu, ev, Duv, sigma),
                 schedule="greedy_color", name=f"pose_K{n}_L{L}_keep{keep:g}_s{seed}")


def pose_dense(n: int, L: int = 13, seed: int = 0, sigma: float = 0.05) -> Model:
    """The shape of the paper's pose dataset (Sec. 7: fully connected, a few
    hundred to a few thousand nodes, 13 labels): huge edge counts with tiny
    tables; round-robin schedule (n - 1 matchings of n / 2 edges)."""
    m = pose_sparse(1.0, n, L, seed, sigma)
    m.schedule = "round_robin"
    m.name = f"pose_dense_K{n}_L{L}_s{seed}"
    return m


def trunc_linear_tables(labels: np.ndarray, eu: np.ndarray, ev: np.ndarray, param: np.ndarray,
                        quad: bool = False) -> np.ndarray:
    """Dense tables of truncated-linear costs w min(|s - t|, tau) (or, with
    quad, w min((s - t)^2, tau)), in float32 arithmetic (the distance exact,
    its square and the product each rounded once)."""
    out = []
    for e in range(eu.shape[0]):
        Lu, Lv = int(labels[eu[e]]), int(labels[ev[e]])
        d = np.abs(np.arange(Lu, dtype=np.float32)[:, None] - np.arange(Lv, dtype=np.float32)[None, :])
        if quad:
            d = (d * d).astype(np.float32)
        out.append((np.float32(param[e, 0]) * np.minimum(d, np.float32(param[e, 1]))).astype(np.float32).ravel())
    return np.concatenate(out) if out else np.zeros(0, np.float32)


def grid_trunc_linear(rows: int, cols: int, L: int, weight: float, tau: float, seed: int = 0,
                      Lmin: int = 0, quad: bool = False) -> Model:
    """Stereo-like model: a 4-connected rows x cols grid, labels on a line
    (L per node, or U{Lmin..L} when Lmin > 0), unary U[0, 4), pairwise
    w_e min(|s - t|, tau) (tau = 1: Potts), or w_e min((s - t)^2, tau) with
    quad, w_e = weight * U[0.5, 1.5); greedy edge colouring.  Carries both the
    parameters and the dense tables."""
    rng = np.random.default_rng(seed)
    n = rows * cols
    labels = (rng.integers(Lmin, L + 1, size=n) if Lmin > 0 else np.full(n, L)).astype(np.int32)
    unary = (4.0 * rng.random(int(labels.sum()))).astype(np.float32)
    idx = np.arange(n).reshape(rows, cols)
    eu = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    ev = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    order = np.lexsort((ev, eu))
    eu, ev = eu[order].astype(np.int32), ev[order].astype(np.int32)
    param = np.stack([weight * rng.uniform(0.5, 1.5, size=eu.shape[0]), np.full(eu.shape[0], tau)], axis=1)
    param = param.astype(np.float32)
    return Model(labels, eu, ev, unary, trunc_linear_tables(labels, eu, ev, param, quad), schedule="greedy_color",
                 name=f"grid{rows}x{cols}_L{L}_{'tq' if quad else 'tl'}{tau:g}_s{seed}",
                 pair_kind="trunc_quad" if quad else "trunc_linear", pair_param=param)


def knn(n: int = 2000, k: int = 50, L: int = 64, seed: int = 0) -> Model:
    """Semi-dense model: n random points in [0,1]^3, each linked to its k
    nearest neighbours (symmetrised by union); pairwise N(0,1)."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    pairs = set()
    block = 256
    for s in range(0, n, block):
        d = np.linalg.norm(pts[s:s + block, None, :] - pts[None, :, :], axis=2)
        for i in range(d.shape[0]):
            d[i, s + i] = np.inf
        nn = np.argsort(d, axis=1, kind="stable")[:, :k]
        for i in range(d.shape[0]):
            u = s + i
            for v in nn[i].tolist():
                pairs.add((min(u, v), max(u, v)))
    pairs = sorted(pairs)
    eu = np.asarray([p[0] for p in pairs], np.int32)
    ev = np.asarray([p[1] for p in pairs], np.int32)
    labels = np.full(n, L, np.int32)
    unary = rng.random(n * L).astype(np.float32)
    pw = _draw_pairwise(rng, labels[eu].astype(np.int64) * labels[ev], "normal")
    return Model(labels, eu, ev, unary, pw, schedule="greedy_color",
                 name=f"knn_n{n}_k{k}_L{L}_s{seed}")


def uneven_complete(n: int, Lmin: int, Lmax: int, seed: int, pairwise: str = "normal") -> Model:
    """K_n with per-node label counts L_u ~ U{Lmin..Lmax}."""
    rng = np.random.default_rng(seed)
    eu, ev = _complete_edges(n)
    labels = rng.integers(Lmin, Lmax + 1, size=n).astype(np.int32)
    unary = rng.random(int(labels.sum())).astype(np.float32)
    pw = _draw_pairwise(rng, labels[eu].astype(np.int64) * labels[ev], pairwise)
    return Model(labels, eu, ev, unary, pw, schedule="round_robin",
                 name=f"K{n}_L{Lmin}-{Lmax}_s{seed}")


def batch(count: int = 256, nmin: int = 10, nmax: int = 80, Lmin: int = 16, Lmax: int = 128,
          seed: int = 0) -> list:
    """Independent complete-graph models with uneven n and per-node L."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [uneven_complete(int(ns[i]), Lmin, Lmax, int(seeds[i])) for i in range(count)]


def tiny(n: int, L: int, seed: int, density: float = 1.0, uneven: bool = False,
         pairwise: str = "uniform") -> Model:
    """Small random model (for brute force): each pair of nodes is an edge with
    probability `density`; label counts uniform in 1..L if `uneven`."""
    rng = np.random.default_rng(seed)
    labels = (rng.integers(1, L + 1, size=n) if uneven else np.full(n, L)).astype(np.int32)
    iu, iv = _complete_edges(n)
    keep = rng.random(iu.shape[0]) < density
    eu, ev = iu[keep], iv[keep]
    unary = rng.random(int(labels.sum())).astype(np.float32)
    pw = _draw_pairwise(rng, labels[eu].astype(np.int64) * labels[ev], pairwise)
    return Model(labels, eu, ev, unary, pw, schedule="greedy_color",
                 name=f"tiny_n{n}_L{L}_s{seed}")


def tree(n: int, L: int, seed: int, kind: str = "path") -> Model:
    """Path or star graph with random costs (the LP relaxation is tight on trees)."""
    rng = np.random.default_rng(seed)
    if kind == "path":
        eu = np.arange(n - 1, dtype=np.int32)
        ev = eu + 1
    else:
        eu = np.zeros(n - 1, np.int32)
        ev = np.arange(1, n, dtype=np.int32)
    labels = np.full(n, L, np.int32)
    unary = rng.random(n * L).astype(np.float32)
    pw = _draw_pairwise(rng, labels[eu].astype(np.int64) * labels[ev], "normal")
    return Model(labels, eu, ev, unary, pw, schedule="greedy_color",
                 name=f"{kind}_n{n}_L{L}_s{seed}")


# The five workload shapes (small one first).
def config(i: int, seed: int = 0):
    if i == 1:
        return complete(20, 8, seed=seed, pairwise="uniform"), 200
    if i == 2:
        return pose_like(60, 300, seed=seed), 500
    if i == 3:
        return knn(2000, 50, 64, seed=seed), 300
    if i == 4:
        return batch(256, seed=seed), 100
    if i == 5:
        return [complete(50, 64, seed=seed + j, pairwise="normal") for j in range(16)], 50
    raise ValueError(i)
