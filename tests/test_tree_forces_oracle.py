"""Pins of the tree-forces restatement (oracle/tree_oracle.c, oracle_tree_forces).

The paper approximates potentials only; the forces F = -grad E follow the
same recursion (Algorithm 2) under a force criterion stated in the oracle:
each component within eps S(x) + tau, S(x) = sum over the tuples containing x
of |grad_x phi|_2. Pins:
  * eps = tau = 0 admits no prune: the exact forces (the FP64 gradient of the
    exhaustive oracle, itself pinned by central differences and identities);
  * the tuple counts of all prunes and base cases are C(N-1, 2) per particle;
  * alpha = 0: every component of every particle within eps S + tau (the
    deterministic rule's bound is a theorem, not a heuristic: S's seed is a
    true lower bound and |grad| is bounded over the boxes);
  * alpha > 0: at least 1 - alpha of the particles within (binomial slack);
  * the result rebuilt from the record of prunes: exact forces minus the exact
    contribution of each pruned node triple plus what it credits
    (-T_x grad_x phi(c1, c2, c3) for a deterministic prune, -T_x mu(x) for a
    Monte Carlo prune), with the gradient in this file taken from the
    pair-vector form (the oracle differentiates the cosines instead);
  * planted mistakes in the credits, the push and the base case fail a pin.
"""
import ctypes
import os
import subprocess
from math import comb

import numpy as np
import pytest

import oracle
from oracle import tree
from paper_1105_2769_gb300 import inputs

LEAF = 8


def grad_first(xa, xb, xc):
    """d phi(a, b, c) / d a for arrays of triples (pair-vector form):
    with u = b - a, v = c - a, w = c - b, unit vectors e, p1 = e_u.e_v,
    p2 = e_u.e_w, p3 = e_v.e_w, t = p1 p2 p3, R = (r_u r_v r_w)^-3:
    grad = -g_u - g_v, g_u = 3R/r_u (q e_u - p2 p3 e_v - p1 p3 e_w),
    g_v = 3R/r_v (q e_v - p2 p3 e_u - p1 p2 e_w), q = 5t - 1."""
    u, v, w = xb - xa, xc - xa, xc - xb
    ru, rv, rw = (np.linalg.norm(z, axis=-1, keepdims=True) for z in (u, v, w))
    eu, ev, ew = u / ru, v / rv, w / rw
    p1 = (eu * ev).sum(-1, keepdims=True)
    p2 = (eu * ew).sum(-1, keepdims=True)
    p3 = (ev * ew).sum(-1, keepdims=True)
    t = p1 * p2 * p3
    R = 1.0 / (ru * rv * rw) ** 3
    q = 5.0 * t - 1.0
    gu = 3.0 * R / ru * (q * eu - p2 * p3 * ev - p1 * p3 * ew)
    gv = 3.0 * R / rv * (q * ev - p2 * p3 * eu - p1 * p2 * ew)
    return -gu - gv


def test_pair_vector_gradient_matches_oracle():
    rng = np.random.default_rng(4)
    for _ in range(20):
        a, b, c = rng.normal(size=(3, 3)) * 2.0
        g = np.zeros(3)
        lib = oracle.lib()
        lib.oracle_at_grad.argtypes = [ctypes.POINTER(ctypes.c_double)] * 4
        p = lambda z: np.ascontiguousarray(z).ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa
        lib.oracle_at_grad(p(a), p(b), p(c), p(g))
        np.testing.assert_allclose(grad_first(a, b, c), g, rtol=1e-11, atol=1e-14 * np.abs(g).max())


def _point_triples(r0, r1, r2):
    A, B, C = (np.arange(b, e) for b, e in (r0, r1, r2))
    I, J, K = (g.ravel() for g in np.meshgrid(A, B, C, indexing="ij"))
    m = np.ones(len(I), bool)
    if tuple(r0) == tuple(r1):
        m &= I < J
    if tuple(r1) == tuple(r2):
        m &= J < K
    return I[m], J[m], K[m]


_EXACT = {}


def _exact_sorted(X, leaf_size):
    key = (X.tobytes(), leaf_size)
    if key not in _EXACT:
        L = tree.tree_layout(X, leaf_size)
        Xs = X[L["perm"]]
        _EXACT[key] = (L, Xs) + tuple(oracle.forces(Xs, with_norm=True))
    return _EXACT[key]


def rebuild(X, F, trace, leaf_size=LEAF):
    """max over particles of |F - expected|_inf / S, from the record of prunes."""
    L, Xs, ex, S = _exact_sorted(X, leaf_size)
    perm, beg, end = L["perm"], L["begin"], L["end"]
    n = len(X)
    cen = np.array([Xs[b:e].mean(0) if e > b else np.zeros(3) for b, e in zip(beg, end)])
    expected = ex.copy()
    rows = {}
    for e, k in enumerate(trace["mc_tri"]):
        rows.setdefault(int(k), []).append(e)
    for k, (kind, P) in enumerate(zip(trace["kind"], trace["P"])):
        I, J, K = _point_triples(*[(beg[v], end[v]) for v in P])
        gi = grad_first(Xs[I], Xs[J], Xs[K])
        gj = grad_first(Xs[J], Xs[I], Xs[K])
        gk = grad_first(Xs[K], Xs[I], Xs[J])
        for idx, g in ((I, gi), (J, gj), (K, gk)):
            for d in range(3):
                expected[:, d] += np.bincount(idx, g[:, d], n)   # remove -(-grad)
        Tx = sum(np.bincount(a, None, n) for a in (I, J, K))
        if kind == 0:
            c = [cen[v] for v in P]
            slots = []
            for s in range(3):
                if s > 0 and P[s] == P[s - 1]:
                    continue
                others = [c[o] for o in range(3) if o != s]
                g = grad_first(c[s], others[0], others[1])
                pts = np.arange(beg[P[s]], end[P[s]])
                expected[pts] += -Tx[pts, None] * g[None, :]
                slots.append(s)
        else:
            for e in rows.get(k, []):
                p = trace["mc_pt"][e]
                expected[p] += -Tx[p] * trace["mc_mean"][e]
    err = np.abs(F[perm] - expected).max(axis=1) / S
    return float(err.max())


@pytest.fixture(scope="module")
def gmm():
    X = np.ascontiguousarray(inputs.gaussian_mixture(400, 4, 7.0, 0.5, 1.5, 0.05, 5))
    F, S = oracle.forces(X, with_norm=True)
    return X, F, S


def _cases(S):
    med = float(np.median(S))
    return [("relative", dict(eps=0.1)), ("absolute", dict(eps=0.0, tau=1e-3 * med)),
            ("absolute, large", dict(eps=0.0, tau=1e3 * med)),
            ("Monte Carlo", dict(eps=0.1, alpha=0.05, zeta=4.0))]


def test_eps_zero_is_exact_and_counts_partition(gmm):
    X, F, S = gmm
    Ft, cnt, st = tree.tree_forces(X, eps=0.0, leaf_size=LEAF, with_counts=True)
    assert st["det_prunes"] == 0 and st["mc_prunes"] == 0
    assert np.all(np.abs(Ft - F).max(axis=1) <= 1e-12 * S)
    assert np.all(cnt == comb(len(X) - 1, 2))


@pytest.mark.parametrize("case", range(4))
def test_guarantees_partition_and_rebuild(gmm, case):
    X, F, S = gmm
    name, kw = _cases(S)[case]
    Ft, cnt, st = tree.tree_forces(X, leaf_size=LEAF, with_counts=True, **kw)
    assert np.all(cnt == comb(len(X) - 1, 2))
    assert st["det_prunes"] > 0
    eps, tau, alpha = kw.get("eps", 0.0), kw.get("tau", 0.0), kw.get("alpha", 0.0)
    within = (np.abs(Ft - F) <= eps * S[:, None] + tau + 1e-12 * S[:, None]).all(axis=1)
    if alpha == 0.0:
        assert within.all()
    else:
        assert st["mc_prunes"] > 0
        assert within.mean() >= 1 - alpha - 3.0 * np.sqrt(alpha * (1 - alpha) / len(X))
    Fr, st2, tr = tree.tree_potential_trace(X, leaf_size=LEAF, forces=True, **kw)
    assert np.array_equal(Fr, Ft) and st2 == st
    err = rebuild(X, Fr, tr)
    print(name, st, f"rebuild err {err:.2e}")
    assert err <= 1e-12


FORCE_MUTANTS = {
    "control": None,
    "prune credit with the wrong sign": ("S->node_acc3[3 * P[s] + d] += -T[s] * g[d];",
                                         "S->node_acc3[3 * P[s] + d] += T[s] * g[d];"),
    "prune gradient of the wrong slot": ("grad_slot(c0, c1, c2, s, g);",
                                         "grad_slot(c0, c1, c2, 0, g);"),
    "Monte Carlo credit with the wrong sign": ("pt_add3(S, x, est + 3 * q, 1.0);",
                                               "pt_add3(S, x, est + 3 * q, -1.0);"),
    "no push of force accumulators": (
        "for (int d = 0; d < 3; ++d) S.node_acc3[3 * v + d] += S.node_acc3[3 * par + d];",
        "for (int d = 0; d < 3; ++d) S.node_acc3[3 * v + d] += 0.0 * S.node_acc3[3 * par + d];"),
    "base case misses the third member": ("grad_slot(a, b, c, 2, g); pt_add3(S, k, g, -1.0);",
                                          "grad_slot(a, b, c, 2, g);"),
}


def _mutant(tmp_path, name, edit):
    here = os.path.dirname(oracle.__file__)
    src = open(os.path.join(here, "tree_oracle.c")).read()
    if edit is not None:
        assert src.count(edit[0]) == 1, name
        src = src.replace(edit[0], edit[1])
    tag = "f" + "".join(ch if ch.isalnum() else "_" for ch in name)
    c, so = tmp_path / f"{tag}.c", tmp_path / f"{tag}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(so), str(c), os.path.join(here, "at_oracle.c"), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    tree.bind_trace(L)
    return L


@pytest.fixture(scope="module")
def small():
    X = np.ascontiguousarray(inputs.gaussian_mixture(240, 3, 6.0, 0.5, 1.5, 0.05, 6))
    F, S = oracle.forces(X, with_norm=True)
    return X, F, S


@pytest.mark.parametrize("name", list(FORCE_MUTANTS))
def test_force_pins_reject_planted_mistakes(tmp_path, small, name):
    X, F, S = small
    L = _mutant(tmp_path, name, FORCE_MUTANTS[name])
    holds = []
    # prunes of internal nodes (push), Monte Carlo credits, and the exact case
    for case_name, kw in (_cases(S)[2], ("Monte Carlo", dict(eps=0.1, alpha=0.05, zeta=2.0))):
        Ft, st, tr = tree.tree_potential_trace(X, leaf_size=LEAF, forces=True, lib=L, **kw)
        eps, tau, alpha = kw.get("eps", 0.0), kw.get("tau", 0.0), kw.get("alpha", 0.0)
        within = (np.abs(Ft - F) <= eps * S[:, None] + tau + 1e-12 * S[:, None]).all(axis=1)
        ok = within.all() if alpha == 0.0 else within.mean() >= 0.9
        holds += [bool(ok), rebuild(X, Ft, tr) <= 1e-12]
    Ft, _, _ = tree.tree_potential_trace(X, leaf_size=LEAF, forces=True, lib=L, eps=0.0)
    holds.append(bool(np.all(np.abs(Ft - F).max(axis=1) <= 1e-12 * S)))
    print(name, holds)
    if name == "control":
        assert all(holds)
    else:
        assert not all(holds), f"the force pins did not catch: {name}"
