"""The far-field expansion (§3.2) as the credit of deterministic prunes, at
identical decisions: an oracle-level measurement of what a p > 0 summarize
would give the tree (§4 Summarize credits the monopole T_x phi(c1, c2, c3)).

The tree oracle records every prune it makes. For each deterministic prune
of three distinct nodes (case (d) of Fig. 4) this test replaces, for every
point x of each slot, the monopole credit by the far-field oracle's p-th
order expansion of the other two nodes' double sum at x, and compares the
rebuilt result with the exact sum. On the 4-component mixture (N = 400,
leaf size 8) with the prunes of tau = 1e-3 median|Phi| and of eps = 0.5, a
second-order credit cuts the largest error at least tenfold. (With a tau
large enough to prune adjacent nodes, p = 4 diverges where p = 2 still
helps, and neither the p = 0 interval nor a size/distance guard separates
those cases: a p > 0 rule needs its own error bound, which the paper does
not give for this potential.)
"""
import numpy as np
import pytest

import oracle
from oracle import farfield as off
from oracle import tree
from paper_1105_2769_gb300 import inputs

LEAF = 8


@pytest.fixture(scope="module")
def gmm():
    X = np.ascontiguousarray(inputs.gaussian_mixture(400, 4, 7.0, 0.5, 1.5, 0.05, 5))
    ex, ab = oracle.phi(X, with_abs=True)
    return X, ex, ab


def _recredit(X, phi, trace, p):
    """Result with every distinct-node deterministic credit replaced by the
    order-p expansion at each point (sorted order of the tree layout)."""
    L = tree.tree_layout(X, LEAF)
    perm, beg, end = L["perm"], L["begin"], L["end"]
    Xs = X[perm]
    out = phi[perm].copy()
    n_done = 0
    for kind, P in zip(trace["kind"], trace["P"]):
        if kind != 0 or len(set(P.tolist())) != 3:
            continue
        pts = [Xs[beg[v]:end[v]] for v in P]
        cen = [q.mean(0) for q in pts]
        for s in range(3):
            a, b = [t for t in range(3) if t != s]
            mono = len(pts[a]) * len(pts[b]) * oracle.at_phi(cen[0], cen[1], cen[2])
            out[beg[P[s]]:end[P[s]]] += off.farfield3(pts[s], pts[a], pts[b], p) - mono
        n_done += 1
    return out, perm, n_done


@pytest.mark.parametrize("case", ["tau", "eps"])
def test_second_order_credit_is_tighter(gmm, case):
    X, ex, ab = gmm
    med = float(np.median(np.abs(ex)))
    kw = dict(eps=0.0, tau=1e-3 * med) if case == "tau" else dict(eps=0.5)
    phi, st, tr = tree.tree_potential_trace(X, leaf_size=LEAF, **kw)
    assert st["det_prunes"] > 100
    got2, perm, n_done = _recredit(X, phi, tr, 2)
    assert n_done == st["det_prunes"]  # every prune on this set joins three distinct nodes
    exs = ex[perm]
    e0 = np.max(np.abs(phi[perm] - exs) / np.abs(exs))
    e2 = np.max(np.abs(got2 - exs) / np.abs(exs))
    print(f"{case}: {n_done} prunes, max |error| / |Phi|: monopole {e0:.2e}, p = 2 {e2:.2e}")
    assert e0 > 1e-5  # the prunes carry a visible error
    assert e2 <= 0.1 * e0
