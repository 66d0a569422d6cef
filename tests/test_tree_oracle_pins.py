"""Pins of the tree-path oracle (serial restatement of Algorithms 1-5).

  * eps = tau = 0 admits no prune, so the result is the exact sum (Eq. 1);
  * the per-particle tuple counts of all prunes and base cases add up to
    T^root = C(N-1, 2) exactly (Fig. 4 cases, proof of the Sec. 5 theorem);
  * the deterministic guarantee of Sec. 5 (alpha = 0: every particle within
    eps |Phi| + tau) and the probabilistic one (alpha > 0: at least a
    1 - alpha fraction, checked with binomial slack);
  * the p = 0 interval bound contains phi of every point triple of random
    boxes (brute force);
  * Philox-4x32-10 against the known-answer vectors published with the
    generator (Salmon et al., SC'11, Random123);
  * the two-sided normal quantile against textbook values.
"""
from math import comb

import numpy as np
import pytest

import oracle
from oracle import tree
from paper_1105_2769_gb300 import inputs


@pytest.fixture(scope="module")
def gmm():
    X = inputs.gaussian_mixture(1200, 6, 10.0, 0.5, 1.5, 0.05, 5)
    return X, oracle.phi(X)


def test_philox_known_answers():
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in kat:
        assert tree.philox4x32_10(ctr, key).tolist() == want


def test_normal_quantile():
    assert tree.z_two_sided(0.05) == pytest.approx(1.959963984540054, abs=1e-12)
    assert tree.z_two_sided(0.1) == pytest.approx(1.6448536269514722, abs=1e-12)
    assert tree.z_two_sided(0.5) == pytest.approx(0.6744897501960817, abs=1e-12)


def test_interval_bound_contains_brute_force():
    rng = np.random.default_rng(3)
    for trial in range(40):
        boxes = []
        for _ in range(3):
            c = rng.uniform(-4, 4, size=3)
            h = rng.uniform(0.05, 1.0, size=3)
            boxes.append((c - h, c + h))
        pts = [rng.uniform(lo, hi, size=(12, 3)) for lo, hi in boxes]
        # include the corners so extremes of distances are attained
        def d2(b1, b2):
            (l1, h1), (l2, h2) = b1, b2
            gap = np.maximum(0, np.maximum(l2 - h1, l1 - h2))
            far = np.maximum(h2 - l1, h1 - l2)
            return (gap ** 2).sum(), (far ** 2).sum()
        pairs = [d2(boxes[0], boxes[1]), d2(boxes[0], boxes[2]), d2(boxes[1], boxes[2])]
        lo_b, hi_b = tree.phi_interval([p[0] for p in pairs], [p[1] for p in pairs])
        vals = [oracle.at_phi(a, b, c) for a in pts[0] for b in pts[1] for c in pts[2]]
        if np.isfinite(lo_b):
            assert min(vals) >= lo_b
        if np.isfinite(hi_b):
            assert max(vals) <= hi_b


def test_layout_is_a_valid_tree():
    X = inputs.uniform_cube(777, 5.0, 0.05, 8)
    L = tree.tree_layout(X, 32)
    n, d = len(X), L["depth"]
    assert sorted(L["perm"].tolist()) == list(range(n))
    assert L["begin"][0] == 0 and L["end"][0] == n
    for v in range((1 << d) - 1):  # children partition the parent
        assert L["begin"][2 * v + 1] == L["begin"][v]
        assert L["end"][2 * v + 1] == L["begin"][2 * v + 2]
        assert L["end"][2 * v + 2] == L["end"][v]
    leaves = range((1 << d) - 1, (2 << d) - 1)
    assert max(L["end"][v] - L["begin"][v] for v in leaves) <= 32
    Xs = X[L["perm"]]
    for v in range((2 << d) - 1):
        P = Xs[L["begin"][v]:L["end"][v]]
        assert np.all(P >= L["lo"][v]) and np.all(P <= L["hi"][v])
        np.testing.assert_allclose(L["cen"][v], P.mean(axis=0), rtol=1e-12, atol=1e-12)


def test_eps_zero_is_exact_and_counts_partition(gmm):
    X, ex = gmm
    phi, cnt, st = tree.tree_potential(X, eps=0.0, with_counts=True)
    assert st["det_prunes"] == 0 and st["mc_prunes"] == 0
    np.testing.assert_allclose(phi, ex, rtol=1e-12)
    assert np.all(cnt == comb(len(X) - 1, 2))


@pytest.mark.parametrize("eps,alpha", [(0.1, 0.0), (0.01, 0.0), (0.1, 0.05), (0.01, 0.05)])
def test_guarantees_and_partition(gmm, eps, alpha):
    X, ex = gmm
    phi, cnt, st = tree.tree_potential(X, eps=eps, alpha=alpha, zeta=4.0, with_counts=True)
    assert np.all(cnt == comb(len(X) - 1, 2))
    assert st["det_prunes"] + st["mc_prunes"] > 0
    within = np.abs(phi - ex) <= eps * np.abs(ex)
    if alpha == 0.0:
        assert within.all()
    else:
        n = len(X)
        slack = 3.0 * np.sqrt(alpha * (1 - alpha) / n)
        assert within.mean() >= 1 - alpha - slack


def test_absolute_rule(gmm):
    X, ex = gmm
    tau = 1e-3 * np.median(np.abs(ex))
    phi, cnt, st = tree.tree_potential(X, eps=0.0, tau=tau, with_counts=True)
    assert np.all(cnt == comb(len(X) - 1, 2))
    assert st["det_prunes"] > 0
    assert np.all(np.abs(phi - ex) <= tau)


def test_mc_is_deterministic_in_seed(gmm):
    X, _ = gmm
    a, _, sa = tree.tree_potential(X, eps=0.1, alpha=0.05, seed=7, zeta=4.0)
    b, _, sb = tree.tree_potential(X, eps=0.1, alpha=0.05, seed=7, zeta=4.0)
    c, _, sc = tree.tree_potential(X, eps=0.1, alpha=0.05, seed=8, zeta=4.0)
    assert np.array_equal(a, b) and sa == sb
    assert sc["mc_samples"] != sa["mc_samples"] or not np.array_equal(a, c)


# ---------------------------------------------------------------------------
# Planted mistakes in the tree restatement: each mutant is a copy of the
# oracle with one plausible slip (a Fig. 4 count, the budget's T^root),
# compiled on its own; the pins (exact at eps = 0, tuple counts = C(N-1, 2),
# the deterministic, absolute and Monte Carlo guarantees) must reject every
# one of them and accept the unmodified copy. Slips in the values a prune
# credits, in the Monte Carlo sampler and in the top-down push pass these
# pins (with T^root in the budget a pruned contribution is far below the
# allowed error); test_tree_oracle_credit.py pins those steps.
# ---------------------------------------------------------------------------
_TREE_MUTANTS = {
    "control": None,
    "Fig. 4 case (b) count": ("(n[0] - 1.0) * n[2];     /* (b) */", "n[0] * n[2];     /* (b) */"),
    "Fig. 4 case (c) count": ("n[0] * (n[1] - 1.0);     /* (c) */", "n[0] * n[1];     /* (c) */"),
    "Fig. 4 case (d) slot": ("if (slot == 0) return n[1] * n[2];", "if (slot == 0) return n[0] * n[2];"),
    "budget without T^root": ("(lb > 0.0 ? lb : 0.0) + S->tau) / S->troot;",
                              "(lb > 0.0 ? lb : 0.0) + S->tau);"),
}


def _tree_mutant(tmp_path, name, edit):
    import ctypes
    import os
    import subprocess
    here = os.path.dirname(oracle.__file__)
    src = open(os.path.join(here, "tree_oracle.c")).read()
    if edit is not None:
        assert src.count(edit[0]) == 1, name
        src = src.replace(edit[0], edit[1])
    tag = f"t{abs(hash(name))}"
    c = tmp_path / f"{tag}.c"
    so = tmp_path / f"{tag}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(so), str(c), os.path.join(here, "at_oracle.c"), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    i64, dbl, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    L.oracle_tree_potential.argtypes = [vp, i64, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int, dbl,
                                        ctypes.c_uint64, ctypes.c_int, ctypes.c_int, vp, vp, vp]

    def solve(X, eps, tau=0.0, alpha=0.0, zeta=32.0):
        out = np.zeros(len(X))
        cnt = np.zeros(len(X), dtype=np.int64)
        st = np.zeros(6, dtype=np.int64)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        assert L.oracle_tree_potential(p(X), len(X), eps, tau, alpha, 8, 256, zeta, 1, 0, 3,
                                       p(out), p(cnt), p(st)) == 0
        return out, cnt, st
    return solve


@pytest.mark.parametrize("name", list(_TREE_MUTANTS))
def test_tree_pins_reject_planted_mistakes(tmp_path, name):
    X = np.ascontiguousarray(inputs.gaussian_mixture(600, 4, 8.0, 0.5, 1.5, 0.05, 5))
    ex = oracle.phi(X)
    solve = _tree_mutant(tmp_path, name, _TREE_MUTANTS[name])
    T = comb(len(X) - 1, 2)
    checks = []
    phi, cnt, _ = solve(X, 0.0)                              # exact, partition
    checks += [np.allclose(phi, ex, rtol=1e-12, atol=0), np.all(cnt == T)]
    phi, cnt, st = solve(X, 0.1)                             # deterministic guarantee
    checks += [np.all(cnt == T), np.all(np.abs(phi - ex) <= 0.1 * np.abs(ex))]
    tau = 1e-3 * float(np.median(np.abs(ex)))                # absolute rule
    phi, cnt, st = solve(X, 0.0, tau=tau)
    checks += [st[1] > 0, np.all(cnt == T), np.all(np.abs(phi - ex) <= tau)]
    phi, cnt, st = solve(X, 0.1, alpha=0.05, zeta=4.0)       # Monte Carlo, partition
    within = np.abs(phi - ex) <= 0.1 * np.abs(ex)
    checks += [st[2] > 0, np.all(cnt == T),
               within.mean() >= 0.95 - 3.0 * np.sqrt(0.05 * 0.95 / len(X))]
    holds = all(bool(c) for c in checks)
    if name == "control":
        assert holds
    else:
        assert not holds, f"the pins did not catch: {name}"
