"""mplpp_create's argument checks on the host (include/mplpp.h: a bad argument
returns MPLPP_E_INVALID, an option the chosen update does not support
MPLPP_E_UNSUPPORTED, the message is read back with mplpp_last_error(NULL),
and *out stays NULL).  Every case changes one field of a valid K_4 model; the
checks run before any CUDA call, so no GPU is needed and none is touched."""
import ctypes

import numpy as np
import pytest

from paper_2004_08227_gb300 import _lib

E_INVALID, E_UNSUPPORTED = -1, -7
SCHED_ROUND_ROBIN, SCHED_GREEDY, SCHED_USER = 0, 1, 3
MODE_PERSISTENT = 2
PAIR_DENSE, PAIR_TRUNC_LINEAR = 0, 1


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class _Case:
    """A valid K_4 model with three labels per node; fields can be replaced
    before the call.  The arrays stay referenced while the call runs."""

    def __init__(self):
        self.n = 4
        self.labels = np.full(4, 3, np.int32)
        eu, ev = zip(*[(u, v) for u in range(4) for v in range(u + 1, 4)])
        self.eu, self.ev = np.array(eu, np.int32), np.array(ev, np.int32)
        self.E = len(eu)
        self.unary = np.zeros(12, np.float32)
        self.pairwise = np.zeros(9 * self.E, np.float32)
        self.pair_param = None
        self.pair_kind = PAIR_DENSE
        self.sched = SCHED_ROUND_ROBIN
        self.off = self.order = None
        self.n_matchings = 0
        self.n_models = 1
        self.opt = _lib.MplppOptions()
        _lib.load().mplpp_options_default(ctypes.byref(self.opt))

    def create(self, null_out=False):
        lib = _lib.load()
        m = (_lib.MplppModel * 1)()
        md = m[0]
        md.n_nodes, md.n_edges = self.n, self.E
        md.labels, md.edge_u, md.edge_v = _ptr(self.labels), _ptr(self.eu), _ptr(self.ev)
        md.unary, md.pairwise = _ptr(self.unary), _ptr(self.pairwise)
        md.schedule_kind, md.n_matchings = self.sched, self.n_matchings
        md.matching_off, md.edge_order = _ptr(self.off), _ptr(self.order)
        md.pair_kind, md.pair_param = self.pair_kind, _ptr(self.pair_param)
        h = ctypes.c_void_p(1234)  # must be reset to NULL
        out = None if null_out else ctypes.byref(h)
        st = lib.mplpp_create(m, self.n_models, ctypes.byref(self.opt), None, out)
        msg = lib.mplpp_last_error(None)
        return st, (msg.decode() if msg else ""), (h.value if not null_out else None)


def _structured(c):
    c.pair_kind = PAIR_TRUNC_LINEAR
    c.pairwise = None
    c.pair_param = np.tile(np.array([1.0, 2.0], np.float32), c.E)


def _user(c, off, order):
    c.sched = SCHED_USER
    c.off, c.order = np.array(off, np.int32), np.array(order, np.int32)
    c.n_matchings = len(off) - 1


CASES = {
    "no models": (lambda c: setattr(c, "n_models", 0), E_INVALID, "at least one model"),
    "unknown mode": (lambda c: setattr(c.opt, "mode", 99), E_INVALID, "unknown mode"),
    "cluster 9": (lambda c: setattr(c.opt, "cluster", 9), E_INVALID, "cluster"),
    "unknown rule": (lambda c: setattr(c.opt, "rule", 5), E_INVALID, "unknown rule"),
    "M with backward": (lambda c: (setattr(c.opt, "rule", 1), setattr(c.opt, "record_every", 10)), E_INVALID,
                        "Handshake update only"),
    "M persistent": (lambda c: (setattr(c.opt, "rule", 1), setattr(c.opt, "mode", MODE_PERSISTENT)),
                     E_UNSUPPORTED, "looped driver only"),
    "threads 48": (lambda c: setattr(c.opt, "threads", 48), E_INVALID, "threads"),
    "threads 32": (lambda c: setattr(c.opt, "threads", 32), E_INVALID, "threads"),
    "threads 544": (lambda c: setattr(c.opt, "threads", 544), E_INVALID, "threads"),
    "no nodes": (lambda c: setattr(c, "n", 0), E_INVALID, "bad sizes"),
    "unknown pair_kind": (lambda c: setattr(c, "pair_kind", 5), E_INVALID, "pair_kind"),
    "NULL labels": (lambda c: setattr(c, "labels", None), E_INVALID, "NULL array"),
    "NULL unary": (lambda c: setattr(c, "unary", None), E_INVALID, "NULL array"),
    "NULL tables": (lambda c: setattr(c, "pairwise", None), E_INVALID, "NULL array"),
    "NULL edges": (lambda c: setattr(c, "eu", None), E_INVALID, "NULL array"),
    "structured with tables": (lambda c: (_structured(c), setattr(c, "pairwise", np.zeros(9 * c.E, np.float32))),
                               E_INVALID, "pairwise must be NULL"),
    "structured NULL param": (lambda c: (_structured(c), setattr(c, "pair_param", None)), E_INVALID, "NULL array"),
    "structured backward": (lambda c: (_structured(c), setattr(c.opt, "record_every", 10)), E_INVALID,
                            "no backward"),
    "structured NaN weight": (lambda c: (_structured(c), c.pair_param.__setitem__(4, np.nan)), E_INVALID,
                              "finite"),
    "structured negative tau": (lambda c: (_structured(c), c.pair_param.__setitem__(5, -1.0)), E_INVALID,
                                ">= 0"),
    "label 0": (lambda c: c.labels.__setitem__(2, 0), E_INVALID, "labels must be in 1..65535"),
    "label 65536": (lambda c: c.labels.__setitem__(2, 65536), E_INVALID, "labels must be in 1..65535"),
    "edge u > v": (lambda c: (c.eu.__setitem__(0, 1), c.ev.__setitem__(0, 0)), E_INVALID, "0 <= u < v < n"),
    "edge v = n": (lambda c: c.ev.__setitem__(5, 4), E_INVALID, "0 <= u < v < n"),
    "edge u = v": (lambda c: c.ev.__setitem__(0, 0), E_INVALID, "0 <= u < v < n"),
    "duplicate edge": (lambda c: (setattr(c, "sched", SCHED_GREEDY), c.ev.__setitem__(1, 1)), E_INVALID,
                       "duplicate edge"),
    "round robin, incomplete": (lambda c: (setattr(c, "E", 5)), E_INVALID, "complete graph"),
    "user schedule missing": (lambda c: setattr(c, "sched", SCHED_USER), E_INVALID, "user schedule missing"),
    "user: offsets short": (lambda c: _user(c, [0, 2, 4], [0, 5, 1, 4]), E_INVALID, "offsets"),
    "user: edge twice": (lambda c: _user(c, [0, 2, 4, 6], [0, 5, 1, 4, 2, 2]), E_INVALID, "appears twice"),
    "user: shared node": (lambda c: _user(c, [0, 2, 4, 6], [0, 1, 5, 4, 2, 3]), E_INVALID, "sharing a node"),
    "user: id out of range": (lambda c: _user(c, [0, 2, 4, 6], [0, 5, 1, 4, 2, 6]), E_INVALID, "out of range"),
    "user: offsets decrease": (lambda c: _user(c, [0, 2, 1, 6], [0, 5, 1, 4, 2, 3]), E_INVALID, "non-decreasing"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_create_rejects_bad_arguments_before_any_device_work(name):
    change, status, words = CASES[name]
    c = _Case()
    change(c)
    st, msg, h = c.create()
    assert st == status, (name, st, msg)
    assert words in msg, (name, msg)
    assert h is None or h == 0  # *out is NULL after a failed create


def test_create_rejects_a_null_out_pointer():
    st, msg, _ = _Case().create(null_out=True)
    assert st == E_INVALID and "out is NULL" in msg

