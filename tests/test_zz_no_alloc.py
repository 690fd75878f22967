"""mplpp_bound_noalloc against mplpp_bound, through the C ABI.

The no-allocation entry point is meant for callers that cannot call cudaMalloc
(a fixed device arena, a real-time loop, a plugin whose host runtime accounts
for every device byte); its working memory is a fixed device array shared by
all calls.  Two calls in a row must both reproduce the bound the solver's own
entry point computes for the same state (the second call finds the first
call's leftovers in the shared array)."""
import numpy as np
import pytest

import oracle
from paper_2004_08227_gb300 import workloads as W
from paper_2004_08227_gb300._lib import MplppError
from paper_2004_08227_gb300.solver import Solver, bound_noalloc

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def _device_inputs(m, agg, msg):
    import torch
    dev = "cuda"
    return (torch.tensor(m.labels, dtype=torch.int32, device=dev),
            torch.tensor(m.edge_u, dtype=torch.int32, device=dev),
            torch.tensor(m.edge_v, dtype=torch.int32, device=dev),
            torch.tensor(m.pairwise, dtype=torch.float32, device=dev),
            torch.tensor(agg, dtype=torch.float32, device=dev),
            torch.tensor(msg, dtype=torch.float32, device=dev))


@pytest.mark.parametrize("make", [lambda: W.uneven_complete(9, 1, 70, seed=3),
                                  lambda: W.knn(300, 6, 13, seed=2),
                                  lambda: W.pose_like(10, 300, seed=4)])
def test_noalloc_bound_matches_solver_bound_twice(make):
    import torch
    m = make()
    s = Solver([m])
    s.run(7)
    ref = float(s.bound(exact=True)[0])
    _, agg, msg = s.state_arrays()
    args = _device_inputs(m, agg, msg)
    # the oracle's bound (Sec. 3, eq. LP-lower-bound) of the same state, given
    # in table form: theta^phi_u = agg, theta^phi_uv = theta_uv - phi_{v->u} - phi_{u->v}
    a32, m32 = agg.astype(np.float32).astype(np.float64), msg.astype(np.float32).astype(np.float64)
    L = m.labels.astype(np.int64)
    tabs, k, q = [], 0, 0
    for a, b in zip(m.edge_u, m.edge_v):
        Lu, Lv = int(L[a]), int(L[b])
        t = m.pairwise[k:k + Lu * Lv].astype(np.float64).reshape(Lu, Lv)
        tabs.append(((t - m32[q:q + Lu, None]) - m32[q + Lu:q + Lu + Lv][None, :]).ravel())
        k += Lu * Lv
        q += Lu + Lv
    D_oracle = oracle.bound(m, a32, np.concatenate(tabs))
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        bound_noalloc(*args, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= RTOL * max(1.0, abs(ref)), (got, ref)
        assert abs(got - D_oracle) <= RTOL * max(1.0, abs(D_oracle)), (got, D_oracle)


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    n = 65537
    labels = torch.ones(n, dtype=torch.int32, device="cuda")
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    f = torch.zeros(1, dtype=torch.float32, device="cuda")
    agg = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(MplppError) as ei:
        bound_noalloc(labels, e, e, f, agg, f, out)
    assert ei.value.status == -7


@pytest.mark.parametrize("what", ["zero_label", "edge_u_eq_v", "edge_v_out_of_range"])
def test_noalloc_device_check_rejects_bad_labels_and_edges(what):
    """The device-side check: MPLPP_E_INVALID, and out keeps its sentinel
    (no kernel after the check reads the other inputs or writes out)."""
    import torch
    m = W.uneven_complete(6, 2, 9, seed=1)
    s = Solver([m])
    s.run(2)
    _, agg, msg = s.state_arrays()
    labels, eu, ev, pw, ag, ms = _device_inputs(m, agg, msg)
    if what == "zero_label":
        labels[3] = 0
    elif what == "edge_u_eq_v":
        ev[2] = eu[2]
    else:
        ev[0] = m.n
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    with pytest.raises(MplppError) as ei:
        bound_noalloc(labels, eu, ev, pw, ag, ms, out)
    assert ei.value.status == -1
    torch.cuda.synchronize()
    assert np.isnan(float(out.item()))
    # a valid call right after still gives the solver's bound
    labels, eu, ev, pw, ag, ms = _device_inputs(m, agg, msg)
    bound_noalloc(labels, eu, ev, pw, ag, ms, out)
    ref = float(s.bound(exact=True)[0])
    assert abs(float(out.item()) - ref) <= RTOL * max(1.0, abs(ref))


def test_noalloc_wrapper_rejects_wrong_lengths_and_host_arrays():
    """The binding checks what the C entry point trusts: lengths, dtypes,
    devices (nothing reaches the GPU for these calls)."""
    import torch
    m = W.uneven_complete(5, 2, 6, seed=2)
    s = Solver([m])
    _, agg, msg = s.state_arrays()
    labels, eu, ev, pw, ag, ms = _device_inputs(m, agg, msg)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        bound_noalloc(labels, eu, ev, pw, ag[:-1], ms, out)
    with pytest.raises(ValueError):
        bound_noalloc(labels, eu, ev, pw[:-3], ag, ms, out)
    with pytest.raises(ValueError):
        bound_noalloc(labels, eu, ev, pw, ag, ms.double(), out)
    with pytest.raises(ValueError):
        bound_noalloc(labels.cpu(), eu, ev, pw, ag, ms, out)
