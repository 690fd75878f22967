"""mplpp_bound_noalloc against mplpp_bound, through the C ABI.

The no-allocation entry point is meant for callers that cannot call cudaMalloc
(a fixed device arena, a real-time loop, a plugin whose host runtime accounts
for every device byte); its working memory is a fixed device array shared by
all calls.  Two calls in a row must both reproduce the bound the solver's own
entry point computes for the same state (the second call finds the first
call's leftovers in the shared array)."""
import numpy as np
import pytest

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
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        bound_noalloc(*args, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= RTOL * max(1.0, abs(ref)), (got, ref)


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
