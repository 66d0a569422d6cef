"""FP64 CPU oracle for the Axilrod-Teller three-body sum.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The GPU library never
imports, links or runs anything from here, and nothing here comes from the
GPU library.

The C sources in this directory are plain, slow, obviously correct loops in
FP64 with compensated sums; ``build()`` compiles them with gcc (OpenMP, no
fast-math, no FMA contraction) into ``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SOURCES = ["at_oracle.c", "tree_oracle.c", "farfield_oracle.c"]
_LIB = None
_LOCK = threading.Lock()


def _lib_path() -> str:
    return os.path.join(_BUILD, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc; returns the path of the shared library."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _lib_path()
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(out):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(out) >= newest:
            return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = build()
            L = ctypes.CDLL(path)
            i64, dp, ip = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
            L.oracle_at_phi.restype = ctypes.c_double
            L.oracle_at_phi.argtypes = [dp, dp, dp]
            L.oracle_phi.argtypes = [dp, i64, ip, i64, dp, dp, ctypes.c_int]
            L.oracle_phi_parts.argtypes = [dp, i64, ip, i64, dp, ctypes.c_int]
            L.oracle_energy.argtypes = [dp, i64, dp, ctypes.c_int]
            L.oracle_grad.argtypes = [dp, i64, ip, i64, dp, dp, ctypes.c_int]
            L.oracle_vjp.argtypes = [dp, i64, dp, ip, i64, dp, dp, ctypes.c_int]
            L.oracle_max_threads.restype = ctypes.c_int
            if hasattr(L, "oracle_tree_potential"):
                _bind_tree(L)
            _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _points(X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim != 2 or X.shape[1] != 3:
        raise ValueError("X must be (N, 3)")
    return X


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def at_phi(xi, xj, xk) -> float:
    """phi(x_i, x_j, x_k), Axilrod-Teller (Sec. 1)."""
    a, b, c = (np.ascontiguousarray(v, dtype=np.float64) for v in (xi, xj, xk))
    return float(lib().oracle_at_phi(_dp(a), _dp(b), _dp(c)))


def phi(X, idx=None, with_abs=False, nthreads=0):
    """Phi(x_i) for the given particle indices (all if None), Eq. 1."""
    X = _points(X)
    n = len(X)
    idx = np.arange(n, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
    if idx.size and (idx.min() < 0 or idx.max() >= n):
        raise IndexError("particle index out of range")
    out = np.zeros(len(idx))
    ab = np.zeros(len(idx)) if with_abs else None
    rc = lib().oracle_phi(_dp(X), n, _ip(idx), len(idx), _dp(out),
                          _dp(ab) if with_abs else None, int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_phi failed ({rc})")
    return (out, ab) if with_abs else out


def phi_parts(X, idx=None, nthreads=0):
    """Sum over the terms of Phi(x_i) of (1 + 3|cos cos cos|)/(r r r)^3: the
    magnitudes of each term's two parts, the scale of its rounding error."""
    X = _points(X)
    n = len(X)
    idx = np.arange(n, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(len(idx))
    rc = lib().oracle_phi_parts(_dp(X), n, _ip(idx), len(idx), _dp(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_phi_parts failed ({rc})")
    return out


def energy(X, nthreads=0) -> float:
    """E = sum over unordered triples a<b<c of phi."""
    X = _points(X)
    out = np.zeros(1)
    rc = lib().oracle_energy(_dp(X), len(X), _dp(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_energy failed ({rc})")
    return float(out[0])


def grad(X, idx=None, nthreads=0, with_norm=False):
    """dE/dx_i for the given indices (forces are the negative). with_norm also
    returns sum over the triples of |grad_i phi| (scale for rounding errors)."""
    X = _points(X)
    n = len(X)
    idx = np.arange(n, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((len(idx), 3))
    nrm = np.zeros(len(idx)) if with_norm else None
    rc = lib().oracle_grad(_dp(X), n, _ip(idx), len(idx), _dp(out),
                           _dp(nrm) if with_norm else None, int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_grad failed ({rc})")
    return (out, nrm) if with_norm else out


def forces(X, idx=None, nthreads=0, with_norm=False):
    r = grad(X, idx, nthreads, with_norm)
    return (-r[0], r[1]) if with_norm else -r


def vjp(X, g, idx=None, nthreads=0, with_norm=False):
    """d/dx_m of sum_l g_l Phi_l for the given indices m."""
    X = _points(X)
    n = len(X)
    g = np.ascontiguousarray(g, dtype=np.float64)
    if g.shape != (n,):
        raise ValueError("g must have shape (N,)")
    idx = np.arange(n, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((len(idx), 3))
    nrm = np.zeros(len(idx)) if with_norm else None
    rc = lib().oracle_vjp(_dp(X), n, _dp(g), _ip(idx), len(idx), _dp(out),
                          _dp(nrm) if with_norm else None, int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_vjp failed ({rc})")
    return (out, nrm) if with_norm else out


def _bind_tree(L):  # filled in by the tree oracle bindings
    from . import tree as _tree
    _tree.bind(L)
