"""The oracle's own edge schedules (Sec. 6 Parallelization, Alg. 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Written independently of
the product's C++ schedule builder; the test suite checks that both produce
the same arrays.

A schedule is (matching_off [M+1], edge_order [E]): matching k is
edge_order[matching_off[k]:matching_off[k+1]], a list of edge ids no two of
which share a node (Sec. 6: a matching).  Matchings are visited in order and
the whole queue is repeated every iteration (Sec. 6, circular task queue).

Readings where the paper is silent:
  * complete graphs use the round-robin ("circle") 1-factorization: node n-1
    is fixed, round r pairs (r, n-1) and ((r+k) mod (n-1), (r-k) mod (n-1))
    for k = 1..n/2-1; odd n adds a dummy node whose pairs are dropped;
  * other graphs use greedy edge colouring: edges in (u, v)-lexicographic order
    get the smallest colour free at both ends; colour classes are the
    matchings, in colour order;
  * Alg. 1 ("repeat a matching on the remaining edges") is implemented with a
    greedy maximal matching scanning remaining edges in (u, v) order;
  * within a matching, edges are ordered by (u, v).
"""
from __future__ import annotations

import numpy as np


def _pack(matchings, edge_index):
    off = [0]
    order = []
    for m in matchings:
        m = sorted(m)
        order.extend(edge_index[p] for p in m)
        off.append(len(order))
    return np.asarray(off, np.int32), np.asarray(order, np.int32)


def _index(edge_u, edge_v):
    idx = {}
    for e, (u, v) in enumerate(zip(edge_u.tolist(), edge_v.tolist())):
        if (u, v) in idx:
            raise ValueError("duplicate edge")
        idx[(u, v)] = e
    return idx


def round_robin(n: int, edge_u, edge_v):
    """1-factorization of K_n by the circle method (readings above)."""
    idx = _index(np.asarray(edge_u), np.asarray(edge_v))
    if len(idx) != n * (n - 1) // 2:
        raise ValueError("round_robin needs the complete graph")
    m = n if n % 2 == 0 else n + 1  # m-1 rounds on m (even) vertices
    matchings = []
    for r in range(m - 1):
        pairs = [(r, m - 1)]
        for k in range(1, m // 2):
            pairs.append(((r + k) % (m - 1), (r - k) % (m - 1)))
        keep = []
        for a, b in pairs:
            if a >= n or b >= n:
                continue  # pair with the dummy vertex
            keep.append((min(a, b), max(a, b)))
        if keep:
            matchings.append(keep)
    return _pack(matchings, idx)


def greedy_color(n: int, edge_u, edge_v):
    """Greedy edge colouring in (u, v) order; classes = matchings."""
    edge_u, edge_v = np.asarray(edge_u), np.asarray(edge_v)
    idx = _index(edge_u, edge_v)
    used = [set() for _ in range(n)]
    classes = {}
    for (u, v) in sorted(idx):
        c = 0
        while c in used[u] or c in used[v]:
            c += 1
        used[u].add(c)
        used[v].add(c)
        classes.setdefault(c, []).append((u, v))
    return _pack([classes[c] for c in sorted(classes)], idx)


def alg1(n: int, edge_u, edge_v):
    """Alg. 1: repeatedly take a (greedy, maximal) matching of the remaining edges."""
    edge_u, edge_v = np.asarray(edge_u), np.asarray(edge_v)
    idx = _index(edge_u, edge_v)
    remaining = sorted(idx)
    matchings = []
    while remaining:
        busy = set()
        m, rest = [], []
        for (u, v) in remaining:
            if u in busy or v in busy:
                rest.append((u, v))
            else:
                busy.add(u)
                busy.add(v)
                m.append((u, v))
        matchings.append(m)
        remaining = rest
    return _pack(matchings, idx)


def build(kind: str, n: int, edge_u, edge_v):
    return {"round_robin": round_robin, "greedy_color": greedy_color, "alg1": alg1}[kind](n, edge_u, edge_v)


def flatten(matching_off, edge_order):
    """Visiting order of one iteration: the matchings concatenated."""
    return np.asarray(edge_order, np.int32)


def is_valid(n: int, E: int, edge_u, edge_v, matching_off, edge_order) -> bool:
    """Each matching shares no node; every edge appears exactly once."""
    edge_u, edge_v = np.asarray(edge_u), np.asarray(edge_v)
    seen = np.zeros(E, np.int64)
    for k in range(len(matching_off) - 1):
        nodes = set()
        for e in edge_order[matching_off[k]:matching_off[k + 1]]:
            if not (0 <= e < E):
                return False
            seen[e] += 1
            u, v = int(edge_u[e]), int(edge_v[e])
            if u in nodes or v in nodes:
                return False
            nodes.add(u)
            nodes.add(v)
    return bool(np.all(seen == 1))
