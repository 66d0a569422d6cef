"""Tree-approximated forces on the GPU against the tree-forces oracle.

Bars (written here): FP32-bulk gradient terms carry rounding relative to
their own size, so agreement is measured against S_i = sum over the tuples of
|grad_i phi|_2, as for the exhaustive adjoint: 3e-5 S_i.
  * eps = 0 admits no prune: the exact forces (oracle gradient), and the
    tuple counts partition C(N-1, 2);
  * deterministic rule: the same prunes as the restatement (the budget uses
    the seed A^l in FP32 on the GPU and FP64 in the oracle; on these sets no
    decision sits within that rounding), every particle equal to the
    restatement within the bar and within eps S_i + tau of the exact forces;
  * Monte Carlo: prune counts within 2 %, >= 99 % of particles equal to the
    restatement within the bar, >= 1 - alpha within eps S_i.
"""
from math import comb

import numpy as np
import pytest
import torch

import oracle
from oracle import tree as otree
from paper_1105_2769_gb300 import api, inputs

pytestmark = pytest.mark.gpu

BAR = 3e-5


def _gpu(X, eps, alpha, mode="tree", **cfg):
    cfg.setdefault("seed_levels", 3)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    counts = torch.zeros(len(X), dtype=torch.int64, device="cuda")
    F, st = api.forces(Xd, eps=eps, alpha=alpha, mode=mode, config=api.tree_config(**cfg),
                       stats=True, tuple_counts=counts)
    return F.cpu().numpy(), counts.cpu().numpy(), st


@pytest.fixture(scope="module")
def small():
    X = np.ascontiguousarray(inputs.gaussian_mixture(400, 4, 7.0, 0.5, 1.5, 0.05, 5))
    F, S = oracle.forces(X, with_norm=True)
    return X, F, S


@pytest.fixture(scope="module")
def gmm():
    X = np.ascontiguousarray(inputs.gaussian_mixture(1200, 6, 10.0, 0.5, 1.5, 0.05, 5))
    F, S = oracle.forces(X, with_norm=True)
    return X, F, S


def _dev(a, b, S):
    return np.abs(a - b).max(axis=1) / S


def test_eps_zero_is_exact(small):
    X, F, S = small
    G, cnt, st = _gpu(X, 0.0, 0.0, leaf_size=8)
    assert st["det_prunes"] == 0 and st["mc_prunes"] == 0
    print("eps=0: max dev / S", _dev(G, F, S).max())
    assert np.all(_dev(G, F, S) <= BAR)
    assert np.all(cnt == comb(len(X) - 1, 2))


@pytest.mark.parametrize("case", ["eps", "tau", "tau_large"])
def test_deterministic_parity_and_guarantee(small, case):
    X, F, S = small
    med = float(np.median(S))
    if case == "eps":
        kw, mode, arg = dict(eps=0.1), "tree", 0.1
    elif case == "tau":
        kw, mode, arg = dict(tau=1e-3 * med), "tree_abs", 1e-3 * med
    else:
        kw, mode, arg = dict(tau=1e3 * med), "tree_abs", 1e3 * med
    G, cnt, st = _gpu(X, arg, 0.0, mode=mode, leaf_size=8)
    ref, _, rst = otree.tree_forces(X, leaf_size=8, with_counts=True, **kw)
    print(case, "gpu det", st["det_prunes"], "oracle det", rst["det_prunes"],
          "max dev / S", _dev(G, ref, S).max())
    assert np.all(cnt == comb(len(X) - 1, 2))
    assert st["det_prunes"] == rst["det_prunes"] > 0
    assert np.all(_dev(G, ref, S) <= BAR)
    eps, tau = kw.get("eps", 0.0), kw.get("tau", 0.0)
    assert np.all(np.abs(G - F) <= (eps + BAR) * S[:, None] + tau)


@pytest.mark.parametrize("eps", [0.1, 0.01])
def test_monte_carlo_parity_and_guarantee(gmm, eps):
    X, F, S = gmm
    alpha = 0.05
    G, cnt, st = _gpu(X, eps, alpha, zeta=4.0)
    ref, _, rst = otree.tree_forces(X, eps=eps, alpha=alpha, zeta=4.0, with_counts=True)
    print(f"eps={eps}: gpu mc {st['mc_prunes']}/{st['mc_attempts']} det {st['det_prunes']}, "
          f"oracle mc {rst['mc_prunes']}/{rst['mc_attempts']} det {rst['det_prunes']}")
    assert np.all(cnt == comb(len(X) - 1, 2))
    assert st["mc_prunes"] > 0
    assert abs(st["mc_prunes"] - rst["mc_prunes"]) <= max(2, 0.02 * rst["mc_prunes"])
    assert (_dev(G, ref, S) <= BAR).mean() >= 0.99
    within = (np.abs(G - F) <= eps * S[:, None]).all(axis=1)
    slack = 3.0 * np.sqrt(alpha * (1 - alpha) / len(X))
    assert within.mean() >= 1 - alpha - slack


def test_tree_reuse_and_small_inputs(gmm):
    X, F, S = gmm
    Xd = torch.from_numpy(X).cuda()
    t = api.Tree(Xd, config=api.tree_config(seed_levels=3))
    a = api.forces(Xd, eps=0.1, alpha=0.05, mode="tree", tree=t,
                   config=api.tree_config(seed_levels=3, zeta=4.0)).cpu().numpy()
    b = api.forces(Xd, eps=0.1, alpha=0.05, mode="tree",
                   config=api.tree_config(seed_levels=3, zeta=4.0)).cpu().numpy()
    assert np.all(np.abs(a - b).max(axis=1) <= 1e-9 * S)
    t.close()
    for n in (3, 5, 40):
        Xs = inputs.uniform_cube(n, 1.0, 0.05, 200 + n)
        r, s = oracle.forces(Xs, with_norm=True)
        g = api.forces(torch.from_numpy(Xs).cuda(), eps=0.05, mode="tree").cpu().numpy()
        assert np.all(np.abs(g - r) <= (0.05 + BAR) * s[:, None])
