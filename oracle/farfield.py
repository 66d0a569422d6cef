"""ctypes bindings of the far-field expansion oracle (farfield_oracle.c).
Test infrastructure only.

farfield3 is the p-th order three-body far-field expansion of §3.2 (Eq.
truncated_three_body_farfield_expansion); pairset_sum is the exact double sum
it approximates. Product terms are (s12, s13, s23, w): the potential
sum_m w_m |x - y2|^(2 s12_m) |x - y3|^(2 s13_m) |y2 - y3|^(2 s23_m); None
selects the Axilrod-Teller terms (law of cosines)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib as _oracle_lib

_BOUND = None


def _lib(L=None):
    global _BOUND
    if L is None:
        L = _oracle_lib()
    if L is _BOUND or getattr(L, "_ff_bound", False):
        return L
    i64, dbl, vp, ci = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
    L.oracle_at_product_terms.argtypes = [vp, vp, vp, vp]
    L.oracle_ff_index.argtypes = [ci, vp]
    L.oracle_ff_derivs.argtypes = [vp, dbl, ci, vp]
    L.oracle_ff_moments.argtypes = [vp, i64, vp, ci, vp]
    L.oracle_farfield3.argtypes = [vp, i64, vp, i64, vp, i64, vp, vp, ci, ci, vp, vp, vp, vp, vp, ci]
    L.oracle_pairset_sum.argtypes = [vp, i64, vp, i64, vp, i64, ci, vp, vp, vp, vp, vp, ci]
    L._ff_bound = True
    if L is _oracle_lib():
        _BOUND = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data


def _pts(X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim != 2 or X.shape[1] != 3:
        raise ValueError("points must be (n, 3)")
    return X


def at_product_terms(L=None):
    """The Axilrod-Teller potential as product terms: arrays s12, s13, s23, w."""
    L = _lib(L)
    s = [np.zeros(16) for _ in range(4)]
    n = L.oracle_at_product_terms(*[_p(a) for a in s])
    return tuple(a[:n].copy() for a in s)


def multi_indices(p, L=None):
    """The multi-indices a with |a| <= p in the oracle's order, shape (n(p), 3)."""
    L = _lib(L)
    n = L.oracle_ff_index(int(p), None)
    if n < 0:
        raise ValueError("order out of range")
    a = np.zeros((n, 3), dtype=np.int32)
    L.oracle_ff_index(int(p), _p(a))
    return a


def derivs(v0, s, p, L=None):
    """D^a g(v0) for g(v) = (v.v)^s and every |a| <= p (multi_indices order)."""
    L = _lib(L)
    v0 = np.ascontiguousarray(v0, dtype=np.float64)
    out = np.zeros(200)
    n = L.oracle_ff_derivs(_p(v0), float(s), int(p), _p(out))
    if n < 0:
        raise ValueError("order out of range")
    return out[:n].copy()


def moments(Y, p, c=None, L=None):
    """M_a(P, c) = sum_y (-1)^|a| (y - c)^a / a!, c = centre of mass if None."""
    L = _lib(L)
    Y = _pts(Y)
    c = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
    out = np.zeros(200)
    n = L.oracle_ff_moments(_p(Y), len(Y), _p(c), int(p), _p(out))
    if n < 0:
        raise ValueError("order out of range")
    return out[:n].copy()


def _terms(terms):
    if terms is None:
        return 0, None, None, None, None
    s12, s13, s23, w = (np.ascontiguousarray(t, dtype=np.float64) for t in terms)
    return len(w), s12, s13, s23, w


def farfield3(Xq, Y2, Y3, p, terms=None, c2=None, c3=None, nthreads=0, L=None):
    """p-th order far-field expansion at each query point of the P2 x P3 sum."""
    L = _lib(L)
    Xq, Y2, Y3 = _pts(Xq), _pts(Y2), _pts(Y3)
    nt, s12, s13, s23, w = _terms(terms)
    c2 = None if c2 is None else np.ascontiguousarray(c2, dtype=np.float64)
    c3 = None if c3 is None else np.ascontiguousarray(c3, dtype=np.float64)
    out = np.zeros(len(Xq))
    rc = L.oracle_farfield3(_p(Xq), len(Xq), _p(Y2), len(Y2), _p(Y3), len(Y3), _p(c2), _p(c3),
                            int(p), nt, _p(s12), _p(s13), _p(s23), _p(w), _p(out), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_farfield3 failed ({rc})")
    return out


def pairset_sum(Xq, Y2, Y3, terms=None, nthreads=0, L=None):
    """Exact sum over y2 in P2, y3 in P3 of the potential at each query point."""
    L = _lib(L)
    Xq, Y2, Y3 = _pts(Xq), _pts(Y2), _pts(Y3)
    nt, s12, s13, s23, w = _terms(terms)
    out = np.zeros(len(Xq))
    rc = L.oracle_pairset_sum(_p(Xq), len(Xq), _p(Y2), len(Y2), _p(Y3), len(Y3), nt, _p(s12),
                              _p(s13), _p(s23), _p(w), _p(out), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_pairset_sum failed ({rc})")
    return out
