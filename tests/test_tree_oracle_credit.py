"""Pins of the values the tree oracle credits (Summarize, Algorithm 5, top-down).

The oracle records every prune it makes (node triple, and for a Monte Carlo
prune each point's sample mean and sigma). From that record alone, this test
rebuilds what the result must be, by its own bookkeeping:

  * the tree's node membership comes from the layout (pinned separately), and
    centres of mass are recomputed here as the mean of each node's points;
  * each pruned node triple's point triples are enumerated here (the
    canonical cases of Fig. 4 as set conditions, not as counts), giving for
    each of its points x the exact contribution E_x and the tuple count T_x;
  * a deterministic prune (Sec. 4, Summarize) gives x exactly
    T_x phi(c_1, c_2, c_3), a Monte Carlo prune (Algorithm 5) T_x mu(x);
  * the credits of internal nodes reach every point below them (Sec. 3,
    top-down phase).

So  Phi~(x) = Phi(x) - sum_t E_x(t) + sum_t credit_x(t)  must hold to FP64
rounding (1e-12 sum|phi|), while the credits themselves are ~1e-7..0.5 of
sum|phi| on these sets: dropping a credit, giving it to the wrong node,
using another centre, scaling by another count or skipping a level of the
push moves Phi~ by orders of magnitude more than the tolerance.

The Monte Carlo sampler (Algorithm 4, read as uniform with replacement over
the T_x tuples that contain x) is pinned on its own: every drawn partner pair
must make a valid tuple of the node triple (distinct points, one per slot,
none of them x), and over many draws every valid tuple must come up with
equal frequency (chi-square). The sample means are then checked against the
exact tuple means: (mu - E_x/T_x)/sigma_mu stays in a near-normal spread
(skewed phi and m >= 30 make it a little wider than N(0, 1)).

Planted mistakes: copies of the oracle source with one slip each in these
steps are compiled separately; each must fail a pin here, and an unmodified
copy must pass.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import tree
from paper_1105_2769_gb300 import inputs

LEAF = 8


def _phi_lc(xa, xb, xc):
    """phi of many triples at once, by the law of cosines on squared sides
    (a second form of Sec. 1's phi; the oracle forms cosines by dot products)."""
    c = ((xa - xb) ** 2).sum(-1)
    b = ((xa - xc) ** 2).sum(-1)
    a = ((xb - xc) ** 2).sum(-1)
    num = (b + c - a) * (a + c - b) * (a + b - c)
    return (1.0 + 3.0 * num / (8.0 * a * b * c)) / (a * b * c) ** 1.5


def _point_triples(r0, r1, r2):
    """All unordered point triples of a node triple given by sorted index
    ranges: the product of the three ranges, with an ordering condition
    between slots that hold the same node (so each triple appears once)."""
    A, B, C = (np.arange(b, e) for b, e in (r0, r1, r2))
    I, J, K = (g.ravel() for g in np.meshgrid(A, B, C, indexing="ij"))
    m = np.ones(len(I), bool)
    if tuple(r0) == tuple(r1):
        m &= I < J
    if tuple(r1) == tuple(r2):
        m &= J < K
    return I[m], J[m], K[m]


def rebuild(X, phi, trace, leaf_size=LEAF):
    """Expected result from the trace; returns (max |phi - expected| / sum|phi|,
    credit magnitude / sum|phi| per particle, Monte Carlo z values)."""
    L = tree.tree_layout(X, leaf_size)
    perm, beg, end = L["perm"], L["begin"], L["end"]
    n = len(X)
    Xs = X[perm]
    ex, ab = oracle.phi(Xs, with_abs=True)
    cen = np.array([Xs[b:e].mean(0) if e > b else np.zeros(3) for b, e in zip(beg, end)])
    expected = ex.copy()
    cabs = np.zeros(n)
    rows = {}
    for e, k in enumerate(trace["mc_tri"]):
        rows.setdefault(int(k), []).append(e)
    z = []
    for k, (kind, P) in enumerate(zip(trace["kind"], trace["P"])):
        I, J, K = _point_triples(*[(beg[v], end[v]) for v in P])
        f = _phi_lc(Xs[I], Xs[J], Xs[K])
        Ex = sum(np.bincount(a, f, n) for a in (I, J, K))
        Tx = sum(np.bincount(a, None, n) for a in (I, J, K))
        expected -= Ex
        if kind == 0:
            credit = Tx * oracle.at_phi(cen[P[0]], cen[P[1]], cen[P[2]])
        else:
            credit = np.zeros(n)
            for e in rows.get(k, []):
                p = trace["mc_pt"][e]
                credit[p] = Tx[p] * trace["mc_mean"][e]
                z.append((trace["mc_mean"][e] - Ex[p] / Tx[p]) / trace["mc_sig"][e])
        expected += credit
        cabs += np.abs(credit)
    err = np.abs(phi[perm] - expected) / ab
    return float(err.max()), cabs / ab, np.abs(np.array(z))


@pytest.fixture(scope="module")
def gmm():
    X = np.ascontiguousarray(inputs.gaussian_mixture(400, 4, 7.0, 0.5, 1.5, 0.05, 5))
    return X, oracle.phi(X)


def _cases(ex):
    med = float(np.median(np.abs(ex)))
    return [  # (name, solve arguments)
        ("absolute tau", dict(eps=0.0, tau=1e-3 * med)),
        ("absolute tau, large", dict(eps=0.0, tau=1e3 * med)),
        ("Monte Carlo", dict(eps=0.1, alpha=0.05, zeta=4.0)),
    ]


def _sampler_ok(lib=None, seed=11):
    """Partner draws of every canonical case (Fig. 4) and slot: valid tuples,
    uniform over the T_x tuples containing x."""
    from scipy.stats import chi2
    rng = np.random.default_rng(seed)
    # node triples as (node ids, point ranges per slot): cases (a)-(d)
    cases = [((5, 5, 5), [(0, 7)] * 3),
             ((5, 5, 9), [(0, 6), (0, 6), (6, 11)]),
             ((5, 9, 9), [(0, 5), (5, 11), (5, 11)]),
             ((5, 7, 9), [(0, 4), (4, 9), (9, 15)])]
    for P, rngs in cases:
        for slot in range(3):
            if slot > 0 and P[slot] == P[slot - 1]:
                continue
            b, e = rngs[slot]
            for x in (b, e - 1):
                I, J, K = _point_triples(*rngs)
                keep = (I == x) | (J == x) | (K == x)
                valid = {tuple(sorted(t)) for t in zip(I[keep], J[keep], K[keep])}
                n = 400 * len(valid)
                r = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
                yz = tree.mc_draw(P, [q[0] for q in rngs], [q[1] for q in rngs], slot, x, r,
                                  lib=lib)
                got = [tuple(sorted((x, y, z))) for y, z in yz]
                if any(len(set(t)) < 3 or t not in valid for t in got):
                    return False
                counts = np.array([sum(1 for t in got if t == v) for v in sorted(valid)])
                if len(valid) > 1:
                    stat = ((counts - n / len(valid)) ** 2 / (n / len(valid))).sum()
                    if chi2.sf(stat, len(valid) - 1) < 1e-6:
                        return False
    return True


def test_sampler_draws_valid_uniform_tuples():
    assert _sampler_ok()


def _pins(X, ex, solve, lib=None):
    """Every pin of this file on one build of the oracle; returns {pin: holds}."""
    out = {"sampler": _sampler_ok(lib)}
    for name, kw in _cases(ex):
        phi, st, tr = solve(X, **kw)
        if not np.all(np.isfinite(phi)):
            out[name] = False
            continue
        err, rel, z = rebuild(X, phi, tr)
        out[name] = err <= 1e-12
        if kw.get("alpha", 0.0) > 0.0:
            out[name + ": prunes"] = st["mc_prunes"] > 0 and st["det_prunes"] > 0
            out[name + ": estimates"] = len(z) > 0 and (z <= 3.0).mean() >= 0.85
        else:
            out[name + ": prunes"] = st["det_prunes"] > 0
    return out


def _solve_with(lib):
    def solve(X, **kw):
        return tree.tree_potential_trace(X, leaf_size=LEAF, lib=lib, **kw)
    return solve


def test_credits_rebuild_exactly(gmm):
    X, ex = gmm
    for name, kw in _cases(ex):
        phi, st, tr = tree.tree_potential_trace(X, leaf_size=LEAF, **kw)
        err, rel, z = rebuild(X, phi, tr)
        print(f"{name}: {st}; max err/sum|phi| {err:.2e}; credit/sum|phi| median "
              f"{np.median(rel):.2e} max {rel.max():.2e}")
        assert err <= 1e-12
        # the credits are far above the tolerance for most particles, so the
        # identity resolves every one of them
        assert (rel > 1e-9).mean() >= 0.5
        if kw.get("alpha", 0.0) > 0.0:
            assert st["mc_prunes"] > 0 and len(z) > 100
            print(f"  Monte Carlo |z| <= 1.96: {(z <= 1.96).mean():.3f}, <= 3: "
                  f"{(z <= 3).mean():.3f}, max {z.max():.1f}")
            assert (z <= 3.0).mean() >= 0.85


def test_internal_node_credits_are_pushed(gmm):
    """Prunes of internal nodes happen on these sets, so the push is exercised."""
    X, ex = gmm
    L = tree.tree_layout(X, LEAF)
    first_leaf = (1 << L["depth"]) - 1
    _, _, tr = tree.tree_potential_trace(X, leaf_size=LEAF, eps=0.0,
                                         tau=1e3 * float(np.median(np.abs(ex))))
    assert (tr["P"] < first_leaf).any()


# one slip per mutant, as (text in tree_oracle.c, replacement)
CREDIT_MUTANTS = {
    "control": None,
    "prune credit dropped": ("S->node_acc[P[s]] += T[s] * f;",
                             "S->node_acc[P[s]] += 0.0 * T[s] * f;"),
    "prune credit given to the first node": ("S->node_acc[P[s]] += T[s] * f;",
                                             "S->node_acc[P[0]] += T[s] * f;"),
    "box centre instead of centre of mass": (
        "t->cen[3 * v + k] = cnt > 0 ? s[k] / (double)cnt : 0.0;",
        "t->cen[3 * v + k] = cnt > 0 ? 0.5 * (l[k] + h[k]) : 0.0;"),
    "Monte Carlo credit scaled by T^root": ("*est = Ti * mean;", "*est = S->troot * mean;"),
    "Monte Carlo credit dropped": ("pt_add(S, x, est[q++]);", "q++;"),
    "Monte Carlo partner from the wrong node": (
        "*y = bb[o1] + draw_below(r0, nn[o1]);", "*y = bb[o2] + draw_below(r0, nn[o2]);"),
    "push of one level only": ("for (int64_t v = 0; v < t.n_nodes; ++v) {",
                               "for (int64_t v = t.n_nodes - 1; v >= 0; --v) {"),
    "no push": ("S.node_acc[v] += S.node_acc[par];", "S.node_acc[v] += 0.0 * S.node_acc[par];"),
}


def _mutant_lib(tmp_path, name, edit):
    here = os.path.dirname(oracle.__file__)
    src = open(os.path.join(here, "tree_oracle.c")).read()
    if edit is not None:
        assert src.count(edit[0]) == 1, name
        src = src.replace(edit[0], edit[1])
    tag = "m" + "".join(ch if ch.isalnum() else "_" for ch in name)
    c, so = tmp_path / f"{tag}.c", tmp_path / f"{tag}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(so), str(c), os.path.join(here, "at_oracle.c"), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    tree.bind_trace(L)
    return L


@pytest.mark.parametrize("name", list(CREDIT_MUTANTS))
def test_credit_pins_reject_planted_mistakes(tmp_path, gmm, name):
    X, ex = gmm
    lib = _mutant_lib(tmp_path, name, CREDIT_MUTANTS[name])
    pins = _pins(X, ex, _solve_with(lib), lib)
    print(name, pins)
    if name == "control":
        assert all(pins.values())
    else:
        assert not all(pins.values()), f"the credit pins did not catch: {name}"
