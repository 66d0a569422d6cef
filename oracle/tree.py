"""ctypes bindings of the tree-path oracle (tree_oracle.c). Test infrastructure only."""
from __future__ import annotations

import ctypes

import numpy as np

_L = None


def bind(L):
    global _L
    i64, dbl, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    L.oracle_tree_potential.argtypes = [vp, i64, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int, dbl,
                                        ctypes.c_uint64, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    bind_trace(L)
    L.oracle_tree_layout.argtypes = [vp, i64, ctypes.c_int, vp, vp, vp, vp, vp, vp]
    L.oracle_tree_depth.argtypes = [i64, ctypes.c_int]
    L.oracle_philox4x32_10.argtypes = [vp, vp, vp]
    L.oracle_z_two_sided.argtypes = [dbl]
    L.oracle_z_two_sided.restype = dbl
    L.oracle_phi_interval.argtypes = [vp, vp, vp, vp]
    _L = L


def bind_trace(L):
    """Argument types of the trace and partner-draw entry points on library L."""
    i64, dbl, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    L.oracle_mc_draw.argtypes = [vp, vp, vp, ctypes.c_int, i64, vp, i64, vp]
    L.oracle_tree_potential_trace.argtypes = [vp, i64, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int,
                                              dbl, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, vp, vp, vp, i64, vp, vp, vp, vp, vp,
                                              i64, vp]
    if hasattr(L, "oracle_tree_forces"):
        L.oracle_tree_forces.argtypes = [vp, i64, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int, dbl,
                                         ctypes.c_uint64, ctypes.c_int, vp, vp, vp]


def _lib():
    if _L is None:
        import oracle
        oracle.lib()
    return _L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def tree_potential(X, eps=0.0, tau=0.0, alpha=0.0, leaf_size=32, m_limit=256, zeta=32.0,
                   seed=0x5eed5eed, mc_rule=0, seed_up=3, with_counts=False):
    """Serial restatement of the multi-tree algorithm; returns (Phi, counts, stats)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = len(X)
    out = np.zeros(n)
    counts = np.zeros(n, dtype=np.int64) if with_counts else None
    stats = np.zeros(6, dtype=np.int64)
    rc = _lib().oracle_tree_potential(_p(X), n, float(eps), float(tau), float(alpha),
                                      int(leaf_size), int(m_limit), float(zeta), int(seed),
                                      int(mc_rule), int(seed_up), _p(out),
                                      _p(counts) if with_counts else None, _p(stats))
    if rc != 0:
        raise RuntimeError("oracle_tree_potential failed")
    keys = ["visited", "det_prunes", "mc_prunes", "mc_attempts", "base_cases", "mc_samples"]
    return out, counts, dict(zip(keys, stats.tolist()))


def tree_potential_trace(X, eps=0.0, tau=0.0, alpha=0.0, leaf_size=32, m_limit=256, zeta=32.0,
                         seed=0x5eed5eed, mc_rule=0, seed_up=3, cap_tri=1 << 16, cap_mc=1 << 18,
                         lib=None, forces=False):
    """tree_potential (or, with forces=True, tree_forces) plus the record of every
    prune: returns (result, stats, trace) with trace = {"kind", "P" (node triples),
    "mc_tri", "mc_pt", "mc_mean", "mc_sig", "mc_m"} (mean and sigma: 3 per point
    for forces). `lib` may name another compiled copy of the oracle (planted-mistake
    tests)."""
    L = lib if lib is not None else _lib()
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = len(X)
    dim = 3 if forces else 1
    out = np.zeros(n * dim)
    stats = np.zeros(6, dtype=np.int64)
    tri = np.zeros((cap_tri, 4), dtype=np.int64)
    mc_tri = np.zeros(cap_mc, dtype=np.int64)
    mc_pt = np.zeros(cap_mc, dtype=np.int64)
    mc_m = np.zeros(cap_mc, dtype=np.int64)
    mc_mean = np.zeros(cap_mc * dim)
    mc_sig = np.zeros(cap_mc * dim)
    n_out = np.zeros(2, dtype=np.int64)
    rc = L.oracle_tree_potential_trace(_p(X), n, float(eps), float(tau), float(alpha),
                                       int(leaf_size), int(m_limit), float(zeta), int(seed),
                                       int(mc_rule), int(seed_up), int(dim == 3), _p(out),
                                       _p(stats), _p(tri),
                                       cap_tri, _p(mc_tri), _p(mc_pt), _p(mc_mean), _p(mc_sig),
                                       _p(mc_m), cap_mc, _p(n_out))
    if rc != 0:
        raise RuntimeError("oracle_tree_potential_trace failed")
    nt, nm = int(n_out[0]), int(n_out[1])
    if nt > cap_tri or nm > cap_mc:
        raise RuntimeError(f"trace capacity exceeded ({nt} prunes, {nm} Monte Carlo points)")
    keys = ["visited", "det_prunes", "mc_prunes", "mc_attempts", "base_cases", "mc_samples"]
    trace = {"kind": tri[:nt, 0].copy(), "P": tri[:nt, 1:].copy(), "mc_tri": mc_tri[:nm],
             "mc_pt": mc_pt[:nm], "mc_mean": mc_mean[:nm * dim].reshape(nm, dim).squeeze(),
             "mc_sig": mc_sig[:nm * dim].reshape(nm, dim).squeeze(), "mc_m": mc_m[:nm]}
    if dim == 3:
        out = out.reshape(n, 3)
        trace["mc_mean"] = trace["mc_mean"].reshape(-1, 3)
        trace["mc_sig"] = trace["mc_sig"].reshape(-1, 3)
    return out, dict(zip(keys, stats.tolist())), trace


def tree_forces(X, eps=0.0, tau=0.0, alpha=0.0, leaf_size=32, m_limit=256, zeta=32.0,
                seed=0x5eed5eed, seed_up=3, with_counts=False):
    """Serial restatement of the tree forces (force criterion of tree_oracle.c);
    returns (F (N x 3), counts, stats)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = len(X)
    out = np.zeros((n, 3))
    counts = np.zeros(n, dtype=np.int64) if with_counts else None
    stats = np.zeros(6, dtype=np.int64)
    rc = _lib().oracle_tree_forces(_p(X), n, float(eps), float(tau), float(alpha), int(leaf_size),
                                   int(m_limit), float(zeta), int(seed), int(seed_up), _p(out),
                                   _p(counts) if with_counts else None, _p(stats))
    if rc != 0:
        raise RuntimeError("oracle_tree_forces failed")
    keys = ["visited", "det_prunes", "mc_prunes", "mc_attempts", "base_cases", "mc_samples"]
    return out, counts, dict(zip(keys, stats.tolist()))


def mc_draw(P, begin, end, slot, x, r, lib=None):
    """Partner pairs (y, z) the Monte Carlo sampler draws for point x of `slot`
    in node triple P (slot point ranges [begin, end)), from 32-bit words r (2 per draw)."""
    L = lib if lib is not None else _lib()
    P = np.ascontiguousarray(P, dtype=np.int64)
    b = np.ascontiguousarray(begin, dtype=np.int64)
    e = np.ascontiguousarray(end, dtype=np.int64)
    r = np.ascontiguousarray(r, dtype=np.uint32).ravel()
    n = len(r) // 2
    yz = np.zeros((n, 2), dtype=np.int64)
    L.oracle_mc_draw(_p(P), _p(b), _p(e), int(slot), int(x), _p(r), n, _p(yz))
    return yz


def tree_layout(X, leaf_size=32):
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = len(X)
    depth = _lib().oracle_tree_depth(n, leaf_size)
    m = (2 << depth) - 1
    perm = np.zeros(n, dtype=np.int64)
    begin = np.zeros(m, dtype=np.int64)
    end = np.zeros(m, dtype=np.int64)
    lo = np.zeros((m, 3)); hi = np.zeros((m, 3)); cen = np.zeros((m, 3))
    _lib().oracle_tree_layout(_p(X), n, int(leaf_size), _p(perm), _p(begin), _p(end), _p(lo),
                              _p(hi), _p(cen))
    return {"depth": depth, "perm": perm, "begin": begin, "end": end, "lo": lo, "hi": hi,
            "cen": cen}


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _lib().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def z_two_sided(alpha):
    return float(_lib().oracle_z_two_sided(float(alpha)))


def phi_interval(sq_lo, sq_hi):
    """[phi_lo, phi_hi] for squared side intervals (c: slots 1-2, b: 1-3, a: 2-3)."""
    lo = np.ascontiguousarray(sq_lo, dtype=np.float64)
    hi = np.ascontiguousarray(sq_hi, dtype=np.float64)
    a = np.zeros(1); b = np.zeros(1)
    _lib().oracle_phi_interval(_p(lo), _p(hi), _p(a), _p(b))
    return float(a[0]), float(b[0])
