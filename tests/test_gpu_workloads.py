"""GPU parity against the FP64 oracle on the workloads of the paper's density
study (the pose model with edges removed at random, Sec. 7) and of its pose
dataset's shape (fully connected, L = 13), in every driver; the drivers
agree bit for bit.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

import oracle
from oracle import schedule as osched
from paper_2004_08227_gb300 import workloads as W
from paper_2004_08227_gb300.solver import Solver

import _parity as P

pytestmark = pytest.mark.gpu

RTOL_D = 1e-5


def _order(m):
    return osched.build(m.schedule, m.n, m.edge_u, m.edge_v)[1]


def _check(m, T, kw):
    sol = oracle.solve(m, _order(m), T)
    s = Solver([m], **kw)
    s.run(T)
    D = s.bound(exact=True)[0]
    assert abs(D - sol["bound"]) <= RTOL_D * max(abs(sol["bound"]), 1.0), (D, sol["bound"])
    xs, _ = s.labels_per_model()
    agg, msg = P.model_state(s, [m], 0)
    P.check_state(m, agg, sol["th_u"], what=m.name)
    P.check_tables(m, msg, sol["th_uv"], agg, what=m.name)
    P.check_labels(m, sol["th_u"], sol["th_uv"], xs[0], sol["labels"], what=m.name)
    return s.state_arrays()


DRIVERS = [{"mode": "persistent"}, {"mode": "looped"}, {"mode": "warp"}, {"mode": "persistent", "cluster": 2}]


@pytest.mark.parametrize("keep", [0.4, 0.1])
def test_sparsified_pose_parity(keep):
    m = W.pose_sparse(keep, 24, 40, seed=5)
    states = [_check(m, 12, kw) for kw in DRIVERS]
    for st in states[1:]:
        assert np.array_equal(st[1], states[0][1]) and np.array_equal(st[2], states[0][2])


def test_dense_pose_L13_parity():
    m = W.pose_dense(40, 13, seed=3)
    states = [_check(m, 8, kw) for kw in DRIVERS]
    for st in states[1:]:
        assert np.array_equal(st[1], states[0][1]) and np.array_equal(st[2], states[0][2])
