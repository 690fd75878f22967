"""FP64 CPU oracle for MPLP++ (Tourani et al., arXiv 2004.08227).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2004_08227_gb300``) never imports it, and
it never imports the product.

The arithmetic lives in ``mplpp_oracle.c`` (plain loops, FP64, table form: the
current reparametrized costs are stored and overwritten, Sec. 4 Def. 1).  This
module compiles it with gcc and wraps it with ctypes.  ``schedule.py`` holds the
oracle's own edge-schedule builders (Sec. 6, Alg. 1), written independently of
the product's C++ ones.

Parity status of each function (see the test files named):
  update_edge  H / M / U   pinned: worked example (appendix, Prop. 3 proof),
                           Def. 1 invariants, Prop. 2 dominance  [test_oracle_update]
  run, bound               pinned: Lemma B.4 monotone D, D <= brute-force MAP,
                           Prop. 1 single-edge exactness, Thm. 2, trees
                           [test_oracle_solver]
  run_parallel             pinned: equals run bit for bit (any thread count),
                           rejects a matching that repeats a node
                           [test_oracle_solver]
  round, energy            pinned: brute-force argmin definition, energy
                           invariance under reparametrization [test_oracle_solver]
  grad                     pinned: FP64 central finite differences
                           [test_oracle_grad]
  schedules                pinned: matching/partition validator, closed-form
                           counts (n-1 perfect matchings of K_n) [test_oracle_schedule]
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mplpp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

RULE_U, RULE_M, RULE_H = 0, 1, 2
_RULES = {"U": RULE_U, "M": RULE_M, "H": RULE_H}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, so x86 and Arm agree),
    with OpenMP where the compiler has it (orc_run_parallel; without it that
    function runs on one thread)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            I, D, P = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            lib.orc_update_edge.argtypes = [I, I, I, P, P, P, P, P, P]
            lib.orc_update_edge.restype = I
            lib.orc_bound.argtypes = [I, P, P, I, P, P, P, P, P]
            lib.orc_bound.restype = D
            lib.orc_run.argtypes = [I, I, P, P, I, P, P, P, I, P, I, P, P, P]
            lib.orc_run.restype = I
            lib.orc_energy.argtypes = [I, P, P, I, P, P, P, P, P, P]
            lib.orc_energy.restype = D
            lib.orc_round.argtypes = [I, P, P, I, P, P, P, P, P, P, P]
            lib.orc_round.restype = I
            lib.orc_run_parallel.argtypes = [I, I, P, P, I, P, P, P, I, P, P, I, P, P, I]
            lib.orc_run_parallel.restype = I
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = I
            lib.orc_grad.argtypes = [I, P, P, I, P, P, P, I, P, I, P, P, P, P, P]
            lib.orc_grad.restype = I
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Graph:
    """Index arrays of one model in the oracle's layout (see mplpp_oracle.c)."""

    def __init__(self, labels, edge_u, edge_v):
        self.L = np.ascontiguousarray(labels, dtype=np.int32)
        self.eu = np.ascontiguousarray(edge_u, dtype=np.int32)
        self.ev = np.ascontiguousarray(edge_v, dtype=np.int32)
        self.n = int(self.L.shape[0])
        self.E = int(self.eu.shape[0])
        if self.E and not np.all(self.eu < self.ev):
            raise ValueError("edges must satisfy u < v (Sec. 3 Notation)")
        self.uoff = np.zeros(self.n + 1, dtype=np.int64)
        np.cumsum(self.L, out=self.uoff[1:])
        sizes = self.L[self.eu].astype(np.int64) * self.L[self.ev].astype(np.int64)
        self.poff = np.zeros(self.E + 1, dtype=np.int64)
        np.cumsum(sizes, out=self.poff[1:])

    @classmethod
    def of(cls, model) -> "Graph":
        return cls(model.labels, model.edge_u, model.edge_v)

    def table(self, th_uv: np.ndarray, e: int) -> np.ndarray:
        Lu, Lv = int(self.L[self.eu[e]]), int(self.L[self.ev[e]])
        return th_uv[self.poff[e]:self.poff[e + 1]].reshape(Lu, Lv)

    def unary(self, th_u: np.ndarray, u: int) -> np.ndarray:
        return th_u[self.uoff[u]:self.uoff[u + 1]]


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def update_edge(rule: str, th_u, th_v, th_uv, record: bool = False):
    """One BCA update (eqs. U, M, H) on a single edge; returns new copies.

    th_uv is the L_u x L_v current pairwise table; returns (th_u', th_v',
    th_uv') and, with record=True and rule H, the argmins (t1, s2, t3)."""
    lib = _load()
    tu, tv = _f64(th_u).copy(), _f64(th_v).copy()
    tuv = _f64(th_uv).copy()
    Lu, Lv = tu.shape[0], tv.shape[0]
    assert tuv.shape == (Lu, Lv)
    rec = [np.zeros(Lu, np.int32), np.zeros(Lv, np.int32), np.zeros(Lu, np.int32)]
    rp = [_p(r) for r in rec] if record else [None, None, None]
    if lib.orc_update_edge(_RULES[rule], Lu, Lv, _p(tu), _p(tv), _p(tuv), *rp):
        raise MemoryError("oracle update failed")
    if record:
        return tu, tv, tuv, tuple(rec)
    return tu, tv, tuv


def initial_state(model):
    """phi = 0: the reparametrized costs start as the given costs (FP64 copies)."""
    return _f64(model.unary).copy(), _f64(model.pairwise).copy()


def run(model, order, iterations: int, rule: str = "H", state=None, history: bool = False):
    """`iterations` BCA iterations visiting edges in `order` (flattened schedule).

    Returns (th_u, th_uv[, D_hist]) -- the reparametrized costs after the run."""
    lib = _load()
    g = Graph.of(model)
    th_u, th_uv = initial_state(model) if state is None else (_f64(state[0]).copy(), _f64(state[1]).copy())
    order = np.ascontiguousarray(order, dtype=np.int32)
    hist = np.zeros(max(iterations, 1), np.float64)
    rc = lib.orc_run(_RULES[rule], g.n, _p(g.L), _p(g.uoff), g.E, _p(g.eu), _p(g.ev), _p(g.poff),
                     int(order.shape[0]), _p(order), int(iterations), _p(th_u), _p(th_uv),
                     _p(hist) if history else None)
    if rc:
        raise MemoryError("oracle run failed")
    if history:
        return th_u, th_uv, hist[:iterations]
    return th_u, th_uv


def run_parallel(model, matching_off, order, iterations: int, rule: str = "H", state=None,
                 threads: int = 0):
    """The iterations of ``run`` with the edges of each matching updated by
    host threads (OpenMP; Sec. 6: edges of a matching are independent).  The
    result equals ``run``'s bit for bit.  threads <= 0: the OpenMP default."""
    lib = _load()
    g = Graph.of(model)
    th_u, th_uv = initial_state(model) if state is None else (_f64(state[0]).copy(), _f64(state[1]).copy())
    off = np.ascontiguousarray(matching_off, dtype=np.int32)
    order = np.ascontiguousarray(order, dtype=np.int32)
    rc = lib.orc_run_parallel(_RULES[rule], g.n, _p(g.L), _p(g.uoff), g.E, _p(g.eu), _p(g.ev), _p(g.poff),
                              int(off.shape[0]) - 1, _p(off), _p(order), int(iterations), _p(th_u), _p(th_uv),
                              int(threads))
    if rc == -2:
        raise ValueError("a matching repeats a node")
    if rc:
        raise MemoryError("oracle run failed")
    return th_u, th_uv


def max_threads() -> int:
    """Host threads orc_run_parallel uses by default (1 without OpenMP)."""
    return int(_load().orc_max_threads())


def bound(model, th_u, th_uv) -> float:
    """Dual bound D (eq. LP-lower-bound) of reparametrized costs."""
    lib = _load()
    g = Graph.of(model)
    th_u, th_uv = _f64(th_u), _f64(th_uv)
    return float(lib.orc_bound(g.n, _p(g.L), _p(g.uoff), g.E, _p(g.eu), _p(g.ev), _p(g.poff),
                               _p(th_u), _p(th_uv)))


def energy(model, labels, th_u=None, th_uv=None) -> float:
    """E(y|theta) (eq. energy-min); default costs are the model's own."""
    lib = _load()
    g = Graph.of(model)
    th_u = _f64(model.unary if th_u is None else th_u)
    th_uv = _f64(model.pairwise if th_uv is None else th_uv)
    y = np.ascontiguousarray(labels, dtype=np.int32)
    return float(lib.orc_energy(g.n, _p(g.L), _p(g.uoff), g.E, _p(g.eu), _p(g.ev), _p(g.poff),
                                _p(th_u), _p(th_uv), _p(y)))


def round_labels(model, th_u, th_uv, margins: bool = False):
    """Sequential primal rounding (Sec. 4 Primal Rounding), FP64."""
    lib = _load()
    g = Graph.of(model)
    th_u, th_uv = _f64(th_u), _f64(th_uv)
    x = np.zeros(g.n, np.int32)
    m = np.zeros(g.n, np.float64)
    if lib.orc_round(g.n, _p(g.L), _p(g.uoff), g.E, _p(g.eu), _p(g.ev), _p(g.poff),
                     _p(th_u), _p(th_uv), _p(x), _p(m)):
        raise MemoryError("oracle rounding failed")
    return (x, m) if margins else x


def grad(model, order, iterations: int):
    """Gradient of D after `iterations` H-iterations w.r.t. the original unary
    and pairwise costs (reverse mode of the table-form iteration).

    Returns (D, grad_unary [sum L], grad_pairwise [sum Lu*Lv])."""
    lib = _load()
    g = Graph.of(model)
    th_u, th_uv = initial_state(model)
    order = np.ascontiguousarray(order, dtype=np.int32)
    gu = np.zeros_like(th_u)
    guv = np.zeros_like(th_uv)
    D = np.zeros(1, np.float64)
    if lib.orc_grad(g.n, _p(g.L), _p(g.uoff), g.E, _p(g.eu), _p(g.ev), _p(g.poff),
                    int(order.shape[0]), _p(order), int(iterations), _p(th_u), _p(th_uv),
                    _p(gu), _p(guv), _p(D)):
        raise MemoryError("oracle gradient failed")
    return float(D[0]), gu, guv


def solve(model, order, iterations: int):
    """Convenience: run H, then bound, rounding and energy of the rounding."""
    th_u, th_uv = run(model, order, iterations)
    D = bound(model, th_u, th_uv)
    x, margin = round_labels(model, th_u, th_uv, margins=True)
    return {"th_u": th_u, "th_uv": th_uv, "bound": D, "labels": x, "margins": margin,
            "energy": energy(model, x)}
