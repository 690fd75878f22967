"""Python binding of the MPLP++ solver: argument marshalling over the C ABI.

Every step of the method (Handshake updates, dual bound, rounding, energy,
backward) runs in the CUDA library; this module only passes pointers, sizes and
the CUDA stream.  PyTorch supplies device memory and the current stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import MODE, MODE_NAME, SCHED, check

try:
    import torch
except ImportError:  # pragma: no cover - torch is a hard dependency of the GPU path
    torch = None


def _ptr(a) -> ctypes.c_void_p:
    if a is None:
        return ctypes.c_void_p(0)
    if torch is not None and isinstance(a, torch.Tensor):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def schedule(kind: str, n: int, edge_u, edge_v):
    """Edge schedule built by the library (Sec. 6): (matching_off, edge_order)."""
    lib = _lib.load()
    eu, ev = _i32(edge_u), _i32(edge_v)
    E = int(eu.shape[0])
    off = np.zeros(E + 1, np.int32)
    order = np.zeros(max(E, 1), np.int32)
    nm = ctypes.c_int32(0)
    check(lib.mplpp_schedule(SCHED[kind], int(n), E, _ptr(eu), _ptr(ev), _ptr(off), _ptr(order), ctypes.byref(nm)))
    return off[:nm.value + 1].copy(), order[:E].copy()


def bound_noalloc(labels, edge_u, edge_v, pairwise, agg, msg, out, stream=None):
    """mplpp_bound_noalloc: dual bound of one model from caller-owned CUDA
    tensors (int32 labels / edges, FP32 pairwise / agg / msg in the state
    layout, FP64 out[1]); allocates no device memory.

    The C entry point trusts the array lengths, so they are checked here:
    every argument a contiguous CUDA tensor of the right dtype on the current
    device, and (for valid labels and edges; invalid ones are left to the
    library's own check, MPLPP_E_INVALID) agg, msg and pairwise holding
    sum L_u, sum (L_u + L_v) and sum L_u L_v entries."""
    dev = torch.cuda.current_device()
    for name, t, dt in (("labels", labels, torch.int32), ("edge_u", edge_u, torch.int32),
                        ("edge_v", edge_v, torch.int32), ("pairwise", pairwise, torch.float32),
                        ("agg", agg, torch.float32), ("msg", msg, torch.float32), ("out", out, torch.float64)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{name} must be a CUDA tensor on the current device (cuda:{dev})")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    n, E = int(labels.numel()), int(edge_u.numel())
    if int(edge_v.numel()) != E:
        raise ValueError("edge_u and edge_v must have the same length")
    if out.numel() < 1:
        raise ValueError("out must hold one value")
    L = labels.to(torch.int64)
    valid = n >= 1 and bool(((L >= 1) & (L <= 65535)).all())
    if valid and E:
        eu, ev = edge_u.to(torch.int64), edge_v.to(torch.int64)
        valid = bool(((eu >= 0) & (eu < ev) & (ev < n)).all())
    if valid:
        need = {"agg": int(L.sum()), "msg": 0, "pairwise": 0}
        if E:
            Lu, Lv = L[edge_u.long()], L[edge_v.long()]
            need["msg"] = int((Lu + Lv).sum())
            need["pairwise"] = int((Lu * Lv).sum())
        for name, t in (("agg", agg), ("msg", msg), ("pairwise", pairwise)):
            if (E or name == "agg") and int(t.numel()) != need[name]:
                raise ValueError(f"{name} must hold {need[name]} entries for these labels and edges, "
                                 f"got {int(t.numel())}")
    lib = _lib.load()
    st = _current_stream() if stream is None else ctypes.c_void_p(stream)
    status = lib.mplpp_bound_noalloc(n, E, _ptr(labels), _ptr(edge_u), _ptr(edge_v), _ptr(pairwise), _ptr(agg),
                                     _ptr(msg), _ptr(out), st)
    if status != _lib.MPLPP_OK:
        msg_ = lib.mplpp_noalloc_last_error()
        raise _lib.MplppError(status, msg_.decode() if msg_ else "")
    return out


def _current_stream():
    if torch is None or not torch.cuda.is_available():
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Solver:
    """Batched MPLP++ solver over one or more independent models.

    models: objects with ``labels``, ``edge_u``, ``edge_v``, ``unary``,
    ``pairwise`` and ``schedule`` (see ``workloads.Model``).  With
    ``device_inputs=True`` the unary / pairwise attributes are float32 CUDA
    tensors; otherwise host arrays (numpy or pinned torch tensors).
    ``user_schedules`` optionally gives ``(matching_off, edge_order)`` per model.
    ``rule`` is the update applied to each edge (Sec. 4): "H" (Handshake, the
    default), or "M" / "U" (MPLP and uniform updates, for comparison; looped
    driver only, no backward).  A model with ``pair_kind == "trunc_linear"``
    passes its costs as ``pair_param`` ([E, 2]: w, tau per edge) unless
    ``structured=False``, which passes its dense ``pairwise`` tables instead.
    """

    def __init__(self, models, *, mode: str = "auto", use_graph: bool = True, record_every: int = 0,
                 cluster: int = 0, threads: int = 0, spin_limit: int = 1 << 22, device_inputs: bool = False,
                 user_schedules=None, stream=None, test_unreachable_wait: bool = False, rule: str = "H",
                 structured: bool = True, test_fp64_replay: bool = False, test_checkpoints: bool = False):
        self._lib = _lib.load()
        self._h = ctypes.c_void_p(0)
        models = list(models)
        self.n_models = len(models)
        self.node_counts = [int(np.asarray(m.labels).shape[0]) for m in models]
        keep = []
        arr = (_lib.MplppModel * self.n_models)()
        for i, m in enumerate(models):
            L, eu, ev = _i32(m.labels), _i32(m.edge_u), _i32(m.edge_v)
            keep += [L, eu, ev]
            # structured costs (w, tau per edge) go in pair_param instead of tables
            kind = getattr(m, "pair_kind", "dense") if structured else "dense"
            src = m.pair_param if kind != "dense" else m.pairwise
            if device_inputs:
                un, pw = m.unary, src
                assert un.is_cuda and un.dtype == torch.float32 and un.is_contiguous()
                assert pw.is_cuda and pw.dtype == torch.float32 and pw.is_contiguous()
            else:
                un = m.unary if (torch is not None and isinstance(m.unary, torch.Tensor)) else \
                    np.ascontiguousarray(m.unary, dtype=np.float32)
                pw = src if (torch is not None and isinstance(src, torch.Tensor)) else \
                    np.ascontiguousarray(src, dtype=np.float32)
            keep += [un, pw]
            md = arr[i]
            md.n_nodes, md.n_edges = int(L.shape[0]), int(eu.shape[0])
            md.labels, md.edge_u, md.edge_v = _ptr(L), _ptr(eu), _ptr(ev)
            md.unary = _ptr(un)
            md.pair_kind = _lib.PAIR[kind]
            if kind == "dense":
                md.pairwise = _ptr(pw)
            else:
                md.pair_param = _ptr(pw)
            if user_schedules is not None and user_schedules[i] is not None:
                off, order = _i32(user_schedules[i][0]), _i32(user_schedules[i][1])
                keep += [off, order]
                md.schedule_kind = SCHED["user"]
                md.n_matchings = int(off.shape[0]) - 1
                md.matching_off, md.edge_order = _ptr(off), _ptr(order)
            else:
                md.schedule_kind = SCHED[getattr(m, "schedule", "greedy_color")]
        opt = _lib.MplppOptions()
        self._lib.mplpp_options_default(ctypes.byref(opt))
        opt.mode = MODE[mode]
        opt.use_graph = int(bool(use_graph))
        opt.inputs_on_device = int(bool(device_inputs))
        opt.record_every = int(record_every)
        opt.cluster = int(cluster)
        opt.threads = int(threads)
        opt.spin_limit = int(spin_limit)
        opt.test_unreachable_wait = int(bool(test_unreachable_wait))
        opt.test_backward = (1 if test_fp64_replay else 0) | (2 if test_checkpoints else 0)
        opt.rule = _lib.RULE[rule]
        self.rule = rule
        self.device_inputs = bool(device_inputs)
        self._stream = _current_stream() if stream is None else ctypes.c_void_p(stream)
        st = self._lib.mplpp_create(arr, self.n_models, ctypes.byref(opt), self._stream, ctypes.byref(self._h))
        del keep
        check(st, None)
        self.unary_sizes = [int(np.asarray(m.labels, dtype=np.int64).sum()) for m in models]
        self.pair_sizes = [int((np.asarray(m.labels, np.int64)[_i32(m.edge_u)] *
                                np.asarray(m.labels, np.int64)[_i32(m.edge_v)]).sum()) for m in models]

    def update_costs(self, unaries, pairwises):
        """mplpp_update_costs: new costs of the same shapes for every model
        (host arrays / tensors, or device tensors if device_inputs), phi reset
        to 0; the mapping, work lists and captured graphs are kept."""
        keep = []
        if len(unaries) != self.n_models or len(pairwises) != self.n_models:
            raise ValueError("one unary and one pairwise array per model")
        for un, pw in zip(unaries, pairwises):
            if self.device_inputs or (torch is not None and isinstance(un, torch.Tensor)):
                assert un.dtype == torch.float32 and un.is_contiguous()
                assert pw.dtype == torch.float32 and pw.is_contiguous()
            else:
                un = np.ascontiguousarray(un, dtype=np.float32)
                pw = np.ascontiguousarray(pw, dtype=np.float32)
            keep += [un, pw]
        pu = (ctypes.c_void_p * self.n_models)(*[_ptr(a).value for a in keep[0::2]])
        pp = (ctypes.c_void_p * self.n_models)(*[_ptr(a).value for a in keep[1::2]])
        self._check(self._lib.mplpp_update_costs(self._h, pu, pp))
        del keep

    # ---- lifecycle -------------------------------------------------------------------
    def close(self):
        if self._h and self._h.value:
            self._lib.mplpp_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st):
        check(st, self._h)

    # ---- the C ABI ---------------------------------------------------------------------
    def run(self, iterations: int):
        self._check(self._lib.mplpp_run(self._h, int(iterations)))
        return self

    def sync(self):
        self._check(self._lib.mplpp_sync(self._h))

    def bound(self, exact: bool = True) -> np.ndarray:
        out = np.zeros(self.n_models, np.float64)
        self._check(self._lib.mplpp_bound(self._h, _ptr(out), int(bool(exact))))
        return out

    def labeling(self):
        """(labels [sum n] int32, energies [n_models] float64)."""
        x = np.zeros(sum(self.node_counts), np.int32)
        en = np.zeros(self.n_models, np.float64)
        self._check(self._lib.mplpp_labeling(self._h, _ptr(x), _ptr(en)))
        return x, en

    def labels_per_model(self):
        x, en = self.labeling()
        out, k = [], 0
        for n in self.node_counts:
            out.append(x[k:k + n])
            k += n
        return out, en

    def backward(self, dD=None, grad_unary=None, grad_pairwise=None):
        """Gradient of sum_m dD[m] * D_m w.r.t. the original costs (concatenated
        over models).  Host arrays are returned unless device inputs are used,
        in which case the given (or new) CUDA tensors are filled."""
        dD = np.ones(self.n_models, np.float32) if dD is None else np.ascontiguousarray(dD, np.float32)
        if self.device_inputs:
            if grad_unary is None:
                grad_unary = torch.empty(sum(self.unary_sizes), dtype=torch.float32, device="cuda")
            if grad_pairwise is None:
                grad_pairwise = torch.empty(max(1, sum(self.pair_sizes)), dtype=torch.float32, device="cuda")
        else:
            if grad_unary is None:
                grad_unary = np.zeros(sum(self.unary_sizes), np.float32)
            if grad_pairwise is None:
                grad_pairwise = np.zeros(max(1, sum(self.pair_sizes)), np.float32)
        self._check(self._lib.mplpp_backward(self._h, _ptr(dD), _ptr(grad_unary), _ptr(grad_pairwise)))
        return grad_unary, grad_pairwise

    def reset(self):
        self._check(self._lib.mplpp_reset(self._h))

    def state_size(self) -> int:
        n = ctypes.c_size_t(0)
        self._check(self._lib.mplpp_state_size(self._h, ctypes.byref(n)))
        return n.value

    def save_state(self) -> bytes:
        buf = ctypes.create_string_buffer(self.state_size())
        self._check(self._lib.mplpp_save_state(self._h, buf, len(buf)))
        return buf.raw

    def load_state(self, data: bytes):
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        self._check(self._lib.mplpp_load_state(self._h, buf, len(data)))

    def state_arrays(self):
        """(iterations, agg [sum L] float64, msg [sum (L_u + L_v)] float64)."""
        raw = self.save_state()
        h = _lib.MplppStateHeader.from_buffer_copy(raw[:ctypes.sizeof(_lib.MplppStateHeader)])
        f = np.frombuffer(raw[ctypes.sizeof(_lib.MplppStateHeader):], dtype=np.float64)
        return int(h.iterations), f[:h.n_unary].copy(), f[h.n_unary:h.n_unary + h.n_msg].copy()

    def set_state(self, agg, msg, iterations: int = 0):
        raw = bytearray(self.save_state())
        h = _lib.MplppStateHeader.from_buffer_copy(bytes(raw[:ctypes.sizeof(_lib.MplppStateHeader)]))
        h.iterations = int(iterations)
        body = np.concatenate([np.asarray(agg, np.float64), np.asarray(msg, np.float64)]).tobytes()
        self.load_state(bytes(h) + body)

    def autotune(self, iterations: int = 3) -> dict:
        """Measured mapping choice (mplpp_autotune); returns its JSON report."""
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self._lib.mplpp_autotune(self._h, int(iterations), buf, len(buf)))
        return json.loads(buf.value.decode()) if buf.value else {}

    def info(self) -> dict:
        inf = _lib.MplppInfo()
        self._check(self._lib.mplpp_info(self._h, ctypes.byref(inf)))
        return {"iterations": inf.iterations, "bytes_per_iteration": inf.bytes_per_iteration, "edges": inf.edges,
                "phases": inf.phases, "mode": MODE_NAME.get(inf.mode, inf.mode), "cluster": inf.cluster,
                "threads": inf.threads, "grid": inf.grid, "launches_per_iteration": inf.launches_per_iteration,
                "labeling_launches": inf.labeling_launches, "poller_warp": inf.poller_warp,
                "device_bytes": inf.device_bytes}


if torch is not None:
    class MPLPPBound(torch.autograd.Function):
        """D after `iterations` H-iterations as a differentiable function of the
        (concatenated, FP32, CUDA) unary and pairwise costs of the models whose
        structure `graphs` gives (objects with labels, edge_u, edge_v, schedule)."""

        @staticmethod
        def forward(ctx, unary, pairwise, graphs, iterations, record_every=10):
            class _M:
                pass
            models, uo, po = [], 0, 0
            for g in graphs:
                L = np.asarray(g.labels, np.int64)
                nu = int(L.sum())
                npw = int((L[np.asarray(g.edge_u)] * L[np.asarray(g.edge_v)]).sum())
                m = _M()
                m.labels, m.edge_u, m.edge_v = g.labels, g.edge_u, g.edge_v
                m.schedule = getattr(g, "schedule", "greedy_color")
                m.unary = unary[uo:uo + nu]
                m.pairwise = pairwise[po:po + npw]
                uo += nu
                po += npw
                models.append(m)
            solver = Solver(models, device_inputs=True, record_every=max(1, int(record_every)))
            solver.run(int(iterations))
            D = solver.bound(exact=True)
            ctx.solver = solver
            ctx.shapes = (unary.shape, pairwise.shape)
            return torch.as_tensor(D, dtype=torch.float64, device=unary.device)

        @staticmethod
        def backward(ctx, gD):
            gu = torch.empty(ctx.shapes[0], dtype=torch.float32, device=gD.device)
            gp = torch.empty(ctx.shapes[1], dtype=torch.float32, device=gD.device)
            ctx.solver.backward(gD.detach().float().cpu().numpy(), gu, gp)
            return gu, gp, None, None, None
