"""Host-side checks of the C-ABI library (no GPU needed).

The library loads, exports every entry point include/mplpp.h declares, and its
host schedule builder agrees bit for bit with the oracle's independent one.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import schedule as osched
from paper_2004_08227_gb300 import _lib, workloads as W
from paper_2004_08227_gb300.solver import schedule

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mplpp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mplpp_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    declared = _declared()
    assert set(declared) == set(_lib.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib._build, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError):
        _lib.load(build_if_needed=False)


@pytest.mark.parametrize("n", [2, 3, 4, 7, 20, 21, 60])
def test_round_robin_matches_oracle(n):
    m = W.complete(n, 1, seed=0)
    a = schedule("round_robin", n, m.edge_u, m.edge_v)
    b = osched.round_robin(n, m.edge_u, m.edge_v)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("kind", ["greedy_color", "alg1"])
@pytest.mark.parametrize("seed", range(4))
def test_greedy_schedules_match_oracle(kind, seed):
    m = W.tiny(40, 1, seed=seed, density=0.25)
    # a shuffled edge list: the schedule must not depend on the input order
    perm = np.random.default_rng(seed).permutation(m.E)
    eu, ev = m.edge_u[perm], m.edge_v[perm]
    a = schedule(kind, m.n, eu, ev)
    b = osched.build(kind, m.n, eu, ev)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert osched.is_valid(m.n, m.E, eu, ev, *a)


def test_knn_greedy_colouring_matches_oracle():
    m = W.knn(300, 8, 4, seed=1)
    a = schedule("greedy_color", m.n, m.edge_u, m.edge_v)
    b = osched.greedy_color(m.n, m.edge_u, m.edge_v)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("eu,ev", [([1], [0]), ([0, 0], [1, 1]), ([0], [5]), ([-1], [1])])
def test_schedule_rejects_malformed_graphs(eu, ev):
    with pytest.raises(_lib.MplppError) as ei:
        schedule("greedy_color", 3, np.asarray(eu), np.asarray(ev))
    assert ei.value.status == -1


def test_round_robin_rejects_incomplete_graph():
    with pytest.raises(_lib.MplppError):
        schedule("round_robin", 4, np.asarray([0, 1]), np.asarray([1, 2]))


def test_struct_sizes_match_header():
    # layout of the option / info structs as the C compiler sees them
    assert ctypes.sizeof(_lib.MplppOptions) == 48
    assert ctypes.sizeof(_lib.MplppInfo) == 64
    assert ctypes.sizeof(_lib.MplppStateHeader) == 40


def test_ctypes_layout_equals_the_c_header(tmp_path):
    """Sizes and field offsets of the ABI structs, from a C compiler reading
    include/mplpp.h, against the ctypes declarations."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    checks = {"mplpp_model": (_lib.MplppModel, ["n_edges", "labels", "pairwise", "schedule_kind", "edge_order",
                                                "pair_kind", "pair_param"]),
              "mplpp_options": (_lib.MplppOptions, ["record_every", "threads", "rule", "spin_limit"]),
              "mplpp_info_t": (_lib.MplppInfo, ["edges", "phases", "launches_per_iteration", "labeling_launches",
                                                 "poller_warp", "device_bytes"])}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mplpp.h"', "int main(void) {"]
    for st, (_, fields) in checks.items():
        lines.append(f'printf("%zu\\n", sizeof({st}));')
        lines += [f'printf("%zu\\n", offsetof({st}, {f}));' for f in fields]
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-x", "c", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for _, (cls, fields) in checks.items():
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f in fields]
    assert got == want
