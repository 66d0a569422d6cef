"""Forces and VJP of the exhaustive sum (step a10) against the oracle.

Bars (written here): each gradient term carries rounding relative to its own
size and terms cancel in the sum, so the error is measured against
S_i = sum over triples of |grad_i phi|:
  FP64: |F_gpu - F_oracle|_inf <= 1e-12 S_i;  FP32 bulk: <= 3e-5 S_i
(a gradient term has about twice the FP32 operations of phi).
Central differences use FP64 energies from the GPU's FP64 mode, which is
itself pinned to the oracle in test_gpu_exhaustive.py."""
import numpy as np
import pytest
import torch

import oracle
from paper_1105_2769_gb300 import api, inputs

pytestmark = pytest.mark.gpu

BAR = {"fp64": 1e-12, "fp32": 3e-5}


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_forces_match_oracle_config1(mode):
    X = inputs.workload("exh64_n512")
    F = api.forces(_dev(X), mode=mode).cpu().numpy()
    ref, nrm = oracle.forces(X, with_norm=True)
    err = np.abs(F - ref).max(axis=1) / nrm
    print(f"{mode}: max |dF| / sum|grad phi| = {err.max():.3e}")
    assert err.max() <= BAR[mode]


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [3, 33, 100])
def test_forces_small_and_ragged(mode, n):
    X = inputs.uniform_cube(n, 1.5, 0.05, 300 + n)
    F = api.forces(_dev(X), mode=mode).cpu().numpy()
    ref, nrm = oracle.forces(X, with_norm=True)
    assert np.all(np.abs(F - ref).max(axis=1) <= BAR[mode] * nrm)


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_vjp_matches_oracle(mode):
    X = inputs.uniform_cube(300, 2.5, 0.05, 77)
    g = inputs.random_weights(len(X), 78)
    G = api.potential_vjp(_dev(X), torch.from_numpy(g), mode=mode).cpu().numpy()
    ref, nrm = oracle.vjp(X, g, with_norm=True)
    assert np.all(np.abs(G - ref).max(axis=1) <= BAR[mode] * nrm)


def test_force_identities_fp64():
    X = inputs.uniform_cube(400, 3.0, 0.1, 81)
    F = api.forces(_dev(X), mode="fp64").cpu().numpy()
    E = api.potential(_dev(X), mode="fp64").cpu().numpy().sum() / 3.0
    scale = np.abs(F).sum()
    assert np.abs(F.sum(axis=0)).max() <= 1e-11 * scale                   # momentum
    assert np.abs(np.cross(X, F).sum(axis=0)).max() <= 1e-10 * np.abs(np.cross(X, F)).sum()
    assert (X * F).sum() == pytest.approx(9.0 * E, rel=1e-10)               # virial


def test_central_differences():
    """64 particles of a 2 048-point set at the density of the 65 536-point
    force workload (cube side 10, d_min 0.5); h = 1e-4; FP64 energies."""
    X = inputs.uniform_cube(2048, 10.0, 0.5, 4)
    idx = inputs.sample_indices(len(X), 64, 9)
    F32 = api.forces(_dev(X), mode="fp32").cpu().numpy()[idx]
    F64 = api.forces(_dev(X), mode="fp64").cpu().numpy()[idx]
    h = 1e-4
    fd = np.zeros((len(idx), 3))
    for q, i in enumerate(idx):
        for d in range(3):
            Xp = X.copy(); Xp[i, d] += h
            Xm = X.copy(); Xm[i, d] -= h
            Ep = api.potential(_dev(Xp), mode="fp64").sum().item() / 3.0
            Em = api.potential(_dev(Xm), mode="fp64").sum().item() / 3.0
            fd[q, d] = -(Ep - Em) / (2 * h)
    scale = np.abs(fd).max(axis=1, keepdims=True)
    e64 = (np.abs(F64 - fd) / scale).max()
    e32 = (np.abs(F32 - fd) / scale).max()
    print(f"central differences: fp64 {e64:.2e}, fp32 {e32:.2e} (relative to max |F_i|)")
    assert e64 <= 1e-5 and e32 <= 1e-3


def test_autograd_backward():
    X = inputs.uniform_cube(200, 2.0, 0.05, 91)
    g = inputs.random_weights(len(X), 92)
    Xt = _dev(X).requires_grad_(True)
    phi = api.Potential.apply(Xt, "fp64")
    phi.backward(torch.from_numpy(g).cuda())
    ref = oracle.vjp(X, g)
    np.testing.assert_allclose(Xt.grad.cpu().numpy(), ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
