"""Python API over the C ABI (torch device memory and streams).

    potential(X, eps=0.0, alpha=0.0, mode="fp32")   -> Phi, shape (N,), float64
    forces(X, mode="fp32")                          -> F, shape (N, 3)
    potential_vjp(X, g, mode="fp32")                -> d(g . Phi)/dX
    Potential.apply(X)                              -> Phi with autograd

``X`` is a CUDA float64 tensor of shape (N, 3). Modes: "fp64" (exhaustive,
FP64 everywhere), "fp32" (exhaustive, FP32 triple arithmetic with FP64
accumulation), "tree" (multi-tree approximation with relative ``eps``),
"tree_abs" (multi-tree with absolute bound ``eps`` = tau). All work runs on
the current torch CUDA stream.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np
import torch

from . import _lib

MODES = {"fp64": _lib.MBM_EXH_FP64, "fp32": _lib.MBM_EXH_FP32, "tree": _lib.MBM_TREE,
         "tree_abs": _lib.MBM_TREE | _lib.MBM_ABS}

_ctx_lock = threading.Lock()
_contexts = {}


class Context:
    """Owns an ``mbm_ctx`` (scratch arena, status word) on one device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        L = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(L.mbm_ctx_create(int(device), int(hbm_budget_bytes), ctypes.byref(h)))
        self.handle = h
        self.device = device

    def set_timing(self, enable: bool = True):
        """Record CUDA events around each solve's dominant kernel."""
        _lib.check(_lib.load().mbm_ctx_set_timing(self.handle, int(bool(enable))))

    def last_kernel_ms(self) -> float:
        """Dominant-kernel time of the last timed solve (waits for it)."""
        return float(_lib.load().mbm_ctx_last_kernel_ms(self.handle))

    def bytes_in_use(self) -> int:
        return int(_lib.load().mbm_ctx_bytes_in_use(self.handle))

    def close(self):
        if self.handle:
            _lib.load().mbm_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover - interpreter shutdown order varies
        try:
            self.close()
        except Exception:
            pass


def default_context(device=None) -> Context:
    if device is None:
        device = torch.cuda.current_device()
    with _ctx_lock:
        ctx = _contexts.get(device)
        if ctx is None:
            ctx = Context(device)
            _contexts[device] = ctx
    return ctx


def _mode(mode) -> int:
    if isinstance(mode, int):
        return mode
    try:
        return MODES[mode]
    except KeyError:
        raise ValueError(f"unknown mode {mode!r}; expected one of {sorted(MODES)}") from None


def _check_points(X: torch.Tensor) -> torch.Tensor:
    if not isinstance(X, torch.Tensor) or not X.is_cuda:
        raise TypeError("X must be a CUDA tensor")
    if X.dim() != 2 or X.shape[1] != 3:
        raise ValueError("X must have shape (N, 3)")
    if X.dtype != torch.float64:
        X = X.to(torch.float64)
    return X.contiguous()


def _stream_handle() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Tree:
    """A built spatial tree (mbm_tree) for one point set; reusable across solves."""

    def __init__(self, X: torch.Tensor, config: _lib.Config | None = None,
                 ctx: Context | None = None):
        X = _check_points(X)
        self.ctx = ctx or default_context(X.device.index)
        cfg = config if config is not None else _lib.default_config()
        h = ctypes.c_void_p()
        _lib.check(_lib.load().mbm_tree_build(self.ctx.handle, ctypes.c_void_p(X.data_ptr()),
                                              X.shape[0], ctypes.byref(cfg), _stream_handle(),
                                              ctypes.byref(h)))
        self.handle = h
        self.n = X.shape[0]
        self.device = X.device

    def info(self):
        nn, nl, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _lib.check(_lib.load().mbm_tree_info(self.handle, ctypes.byref(nn), ctypes.byref(nl),
                                             ctypes.byref(d)))
        return {"n_nodes": nn.value, "n_leaves": nl.value, "depth": d.value}

    def export(self):
        """perm, node boxes, centres and Phi^l as CPU numpy arrays."""
        m = self.info()["n_nodes"]
        perm = torch.empty(self.n, dtype=torch.int64, device=self.device)
        lo = torch.empty((m, 3), dtype=torch.float64, device=self.device)
        hi = torch.empty_like(lo)
        cen = torch.empty_like(lo)
        phil = torch.empty(m, dtype=torch.float64, device=self.device)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr())
        _lib.check(_lib.load().mbm_tree_export(self.handle, ptr(perm), ptr(lo), ptr(hi), ptr(cen),
                                               ptr(phil), _stream_handle()))
        torch.cuda.synchronize(self.device)
        return {k: v.cpu().numpy() for k, v in
                dict(perm=perm, lo=lo, hi=hi, cen=cen, phil=phil).items()}

    def close(self):
        if self.handle:
            _lib.load().mbm_tree_free(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def tree_config(**kw) -> _lib.Config:
    """Default mbm_config with fields overridden (tau, leaf_size, m_limit, zeta,
    seed, mc_rule, validate, seed_levels)."""
    return _lib.default_config(**kw)


def potential(X: torch.Tensor, eps: float = 0.0, alpha: float = 0.0, mode="fp32",
              config: _lib.Config | None = None, tree=None, stats: bool = False,
              ctx: Context | None = None, out: torch.Tensor | None = None,
              tuple_counts: torch.Tensor | None = None):
    """Phi(x_i) for every particle (Eq. 1 with the Axilrod-Teller phi).

    tuple_counts: optional int64 CUDA tensor (N,) that receives, in tree
    modes, the number of point triples credited to each particle."""
    X = _check_points(X)
    n = X.shape[0]
    ctx = ctx or default_context(X.device.index)
    phi = out if out is not None else torch.empty(n, dtype=torch.float64, device=X.device)
    cfg = config if config is not None else _lib.default_config()
    if tuple_counts is not None:
        cfg = _lib.Config.from_buffer_copy(cfg)
        cfg.tuple_counts = tuple_counts.data_ptr()
    st = _lib.Stats()
    L = _lib.load()
    _lib.check(L.mbm_potential_ex(ctx.handle, ctypes.c_void_p(X.data_ptr()), n, float(eps),
                                  float(alpha), _mode(mode), ctypes.byref(cfg),
                                  tree.handle if tree is not None else None,
                                  ctypes.c_void_p(phi.data_ptr()),
                                  ctypes.byref(st) if stats else None, _stream_handle()))
    return (phi, st.as_dict()) if stats else phi


def potential_host(X: np.ndarray, eps: float = 0.0, alpha: float = 0.0, mode="fp32",
                   config: _lib.Config | None = None, ctx: Context | None = None,
                   out: np.ndarray | None = None) -> np.ndarray:
    """Host-buffer entry point: X and the result live in host memory."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim != 2 or X.shape[1] != 3:
        raise ValueError("X must have shape (N, 3)")
    n = X.shape[0]
    ctx = ctx or default_context()
    phi = out if out is not None else np.empty(n, dtype=np.float64)
    cfg = config if config is not None else _lib.default_config()
    _lib.check(_lib.load().mbm_potential_host(
        ctx.handle, X.ctypes.data_as(ctypes.c_void_p), n, float(eps), float(alpha), _mode(mode),
        ctypes.byref(cfg), phi.ctypes.data_as(ctypes.c_void_p), _stream_handle()))
    return phi


def potential_sampled(X: torch.Tensor, idx, ctx: Context | None = None) -> torch.Tensor:
    """Exact Phi (FP32 bulk, FP64 accumulation) of the particles idx only."""
    X = _check_points(X)
    n = X.shape[0]
    idx_t = torch.as_tensor(np.asarray(idx, dtype=np.int64), device=X.device)
    if idx_t.numel() and (int(idx_t.min()) < 0 or int(idx_t.max()) >= n):
        raise IndexError("particle index out of range")
    ctx = ctx or default_context(X.device.index)
    out = torch.empty(idx_t.numel(), dtype=torch.float64, device=X.device)
    _lib.check(_lib.load().mbm_potential_sampled(ctx.handle, ctypes.c_void_p(X.data_ptr()), n,
                                                 ctypes.c_void_p(idx_t.data_ptr()), idx_t.numel(),
                                                 ctypes.c_void_p(out.data_ptr()), _stream_handle()))
    return out


def farfield3(Xq: torch.Tensor, Y2: torch.Tensor, Y3: torch.Tensor, p: int,
              ctx: Context | None = None, validate: bool = True) -> torch.Tensor:
    """p-th order three-body far-field expansion (Sec. 3.2) at each query point
    of sum_{y2 in Y2} sum_{y3 in Y3} phi(x, y2, y3), about the centres of mass."""
    Xq, Y2, Y3 = (_check_points(t) for t in (Xq, Y2, Y3))
    if not (Xq.device == Y2.device == Y3.device):
        raise ValueError("query and source points must be on one device")
    ctx = ctx or default_context(Xq.device.index)
    out = torch.empty(Xq.shape[0], dtype=torch.float64, device=Xq.device)
    _lib.check(_lib.load().mbm_farfield3(ctx.handle, ctypes.c_void_p(Xq.data_ptr()), Xq.shape[0],
                                         ctypes.c_void_p(Y2.data_ptr()), Y2.shape[0],
                                         ctypes.c_void_p(Y3.data_ptr()), Y3.shape[0], int(p),
                                         int(bool(validate)), ctypes.c_void_p(out.data_ptr()),
                                         _stream_handle()))
    return out


def forces(X: torch.Tensor, mode="fp32", eps: float = 0.0, alpha: float = 0.0,
           ctx: Context | None = None, config: _lib.Config | None = None, tree=None,
           stats: bool = False, tuple_counts: torch.Tensor | None = None):
    """F_i = -dE/dx_i, E = sum over unordered triples of phi: exhaustive
    ("fp32", "fp64") or tree-approximated ("tree", "tree_abs": every component
    within eps S_i + tau, S_i the sum of |grad_i phi| over the tuples)."""
    X = _check_points(X)
    ctx = ctx or default_context(X.device.index)
    F = torch.empty_like(X)
    cfg = config if config is not None else _lib.default_config()
    if tuple_counts is not None:
        cfg = _lib.Config.from_buffer_copy(cfg)
        cfg.tuple_counts = tuple_counts.data_ptr()
    st = _lib.Stats()
    _lib.check(_lib.load().mbm_forces_ex(ctx.handle, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                         float(eps), float(alpha), _mode(mode), ctypes.byref(cfg),
                                         tree.handle if tree is not None else None,
                                         ctypes.c_void_p(F.data_ptr()),
                                         ctypes.byref(st) if stats else None, _stream_handle()))
    return (F, st.as_dict()) if stats else F


def potential_vjp(X: torch.Tensor, g: torch.Tensor, mode="fp32",
                  ctx: Context | None = None) -> torch.Tensor:
    """d/dX of sum_l g_l Phi_l."""
    X = _check_points(X)
    g = g.detach().to(device=X.device, dtype=torch.float64).contiguous()
    if g.shape != (X.shape[0],):
        raise ValueError("g must have shape (N,)")
    ctx = ctx or default_context(X.device.index)
    G = torch.empty_like(X)
    _lib.check(_lib.load().mbm_potential_vjp(ctx.handle, ctypes.c_void_p(X.data_ptr()),
                                             X.shape[0], ctypes.c_void_p(g.data_ptr()),
                                             _mode(mode), ctypes.c_void_p(G.data_ptr()),
                                             _stream_handle()))
    return G


class Potential(torch.autograd.Function):
    """Phi(X) with a backward pass through the adjoint kernel."""

    @staticmethod
    def forward(ctx, X, mode="fp32"):
        ctx.save_for_backward(X)
        ctx.mode = mode
        return potential(X.detach(), mode=mode)

    @staticmethod
    def backward(ctx, grad_phi):
        (X,) = ctx.saved_tensors
        return potential_vjp(X.detach(), grad_phi, mode=ctx.mode).to(X.dtype), None


class Server:
    """Continuous-batching request server (mbm_server) on one GPU.

    submit() takes host numpy arrays and returns a ticket; poll() waits for
    it. Results land in the numpy output the request was given."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, slots: int = 4):
        h = ctypes.c_void_p()
        _lib.check(_lib.load().mbm_server_create(int(device), int(hbm_budget_bytes), int(slots),
                                                 ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, X: np.ndarray, kind: str = "potential", mode="fp32", eps: float = 0.0,
               alpha: float = 0.0, system_id: int = 0, config: _lib.Config | None = None,
               out: np.ndarray | None = None) -> int:
        X = np.ascontiguousarray(X, dtype=np.float64)
        n = X.shape[0]
        k = _lib.MBM_REQ_FORCES if kind == "forces" else _lib.MBM_REQ_POTENTIAL
        if out is None:
            out = np.empty((n, 3) if k == _lib.MBM_REQ_FORCES else n, dtype=np.float64)
        cfg = config if config is not None else _lib.default_config()
        req = _lib.Request(k, _mode(mode), n, X.ctypes.data, out.ctypes.data, float(eps),
                           float(alpha), int(system_id), ctypes.pointer(cfg))
        t = ctypes.c_uint64()
        _lib.check(_lib.load().mbm_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = (X, out, cfg)
        return t.value

    def poll(self, ticket: int, timeout_us: int = -1):
        """(status, result dict, output array); status MBM_PENDING / MBM_ETIMEDOUT when not done."""
        r = _lib.Result()
        st = _lib.load().mbm_poll(self.handle, int(ticket), ctypes.byref(r), int(timeout_us))
        if st in (_lib.MBM_PENDING, -5):
            return st, None, None
        _lib.check(st)
        X, out, _ = self._keep.pop(ticket)
        return r.status, r.as_dict(), out

    def stats(self):
        a, p, r, c = (ctypes.c_int64() for _ in range(4))
        b = ctypes.c_size_t()
        _lib.check(_lib.load().mbm_server_stats(self.handle, ctypes.byref(a), ctypes.byref(p),
                                                ctypes.byref(r), ctypes.byref(c), ctypes.byref(b)))
        return {"admitted": a.value, "pending": p.value, "rejected": r.value,
                "completed": c.value, "reserved_bytes": b.value}

    def close(self):
        if self.handle:
            _lib.load().mbm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
