"""Brute-force MAP for tiny models (enumerates every labeling; n <= 6, L <= 4)."""
import itertools

import numpy as np


def map_energy(model):
    L = model.labels.tolist()
    uoff = np.concatenate([[0], np.cumsum(L)])
    sizes = [L[u] * L[v] for u, v in zip(model.edge_u.tolist(), model.edge_v.tolist())]
    poff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    un = model.unary.astype(np.float64)
    pw = model.pairwise.astype(np.float64)
    best, arg = np.inf, None
    for y in itertools.product(*[range(l) for l in L]):
        e = sum(un[uoff[u] + y[u]] for u in range(len(L)))
        for k, (u, v) in enumerate(zip(model.edge_u.tolist(), model.edge_v.tolist())):
            e += pw[poff[k] + y[u] * L[v] + y[v]]
        if e < best:
            best, arg = e, y
    return best, np.asarray(arg, np.int32)
