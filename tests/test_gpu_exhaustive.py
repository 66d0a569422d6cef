"""Parity of the exhaustive CUDA path (steps a1-a3) with the FP64 oracle.

Bars (written here, from the target accuracy of each mode):
  FP64 mode : max |Phi_gpu - Phi_oracle| / |Phi_oracle| <= 1e-12
  FP32 bulk : every term carries a few FP32 roundings relative to its own
              size (about 30 operations at eps32 = 6e-8), and terms of both
              signs cancel in Phi, so the bar is on the error relative to the
              sum of absolute terms: |Phi_gpu - Phi_oracle| <= 3e-6 sum_t|phi_t|.
              On the N = 32 768 workload (cube side 32, d_min 0.5) particles
              without strong cancellation (|Phi| >= 0.3 sum_t|phi_t|) must
              also meet |Phi_gpu - Phi_oracle| <= 1e-6 |Phi_oracle|.
All calls go through the C ABI (ctypes binding)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1105_2769_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 3e-6}


def _rel(a, b):
    return np.max(np.abs(a - b) / np.abs(b))


def _check(got, X, mode, idx=None):
    """Apply the bar of `mode` (see module docstring)."""
    ref, ref_abs = oracle.phi(X, idx, with_abs=True)
    if idx is not None:
        got = got[idx]
    rel = _rel(got, ref)
    rel_abs = np.max(np.abs(got - ref) / ref_abs)
    print(f"{mode}: max rel err {rel:.3e}, max err / sum|phi| {rel_abs:.3e}")
    if mode == "fp64":
        assert rel <= TOL["fp64"]
    else:
        assert rel_abs <= TOL["fp32"]


def _gpu(X, mode, **kw):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    out = api.potential(Xd, mode=mode, **kw)
    return out.cpu().numpy()


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_config1_full_parity(mode):
    """N = 512 uniform in the unit cube (d_min 0.01): every particle."""
    X = inputs.workload("exh64_n512")
    _check(_gpu(X, mode), X, mode)


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [3, 4, 31, 32, 33, 63, 65, 100, 257, 1000])
def test_ragged_sizes(mode, n):
    """Sizes that hit partial tiles, single tiles, and several tiles."""
    X = inputs.uniform_cube(n, max(1.0, (n / 200.0) ** (1 / 3) * 2), 0.05, 100 + n)
    _check(_gpu(X, mode), X, mode)


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_small_n_is_zero(mode):
    for n in (0, 1, 2):
        X = np.random.default_rng(n).uniform(size=(n, 3))
        got = _gpu(X, mode) if n else np.zeros(0)
        assert got.shape == (n,) and np.all(got == 0)


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_closed_forms_on_gpu(mode):
    d = 1.7
    tri = np.array([[0, 0, 0], [d, 0, 0], [d / 2, d * np.sqrt(3) / 2, 0]])
    rt = 1e-12 if mode == "fp64" else 1e-6
    np.testing.assert_allclose(_gpu(tri, mode), 1.375 / d ** 9, rtol=rt)
    col = np.array([[0, 0, 0], [2 * d, 0, 0], [d, 0, 0]])
    np.testing.assert_allclose(_gpu(col, mode), -0.25 / d ** 9, rtol=rt)
    tet = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    np.testing.assert_allclose(_gpu(tet, mode), 4.125 / 2 ** 13.5, rtol=rt)


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_invalid_inputs_rejected(mode):
    X = inputs.uniform_cube(50, 1.0, 0.05, 3)
    Xn = X.copy()
    Xn[7, 1] = np.nan
    with pytest.raises(_lib.MbmError) as e:
        _gpu(Xn, mode)
    assert e.value.status == -1
    Xc = X.copy()
    Xc[40] = Xc[9]
    with pytest.raises(_lib.MbmError) as e:
        _gpu(Xc, mode)
    assert e.value.status == -1
    # the context stays usable afterwards
    _check(_gpu(X, mode), X, mode)


def test_sum_identity_and_permutation_gpu():
    X = inputs.uniform_cube(700, 4.0, 0.1, 17)
    phi = _gpu(X, "fp64")
    E = oracle.energy(X)
    assert phi.sum() == pytest.approx(3 * E, rel=1e-12)
    perm = np.random.default_rng(1).permutation(len(X))
    np.testing.assert_allclose(_gpu(X[perm], "fp64"), phi[perm], rtol=1e-12)


def test_host_entry_point_matches_device():
    X = inputs.uniform_cube(300, 2.0, 0.05, 23)
    dev = _gpu(X, "fp32")
    host = api.potential_host(X, mode="fp32")
    assert _rel(host, dev) <= 1e-13


def test_full_size_fp32_sampled():
    """N = 32 768 in [0,32]^3 (d_min 0.5), the launch the benchmark times;
    16 seeded particles against the oracle."""
    X = inputs.workload("exh32_n32768")
    idx = inputs.sample_indices(len(X), 16, 2024)
    ref, ref_abs = oracle.phi(X, idx, with_abs=True)
    got = _gpu(X, "fp32")[idx]
    rel = np.abs(got - ref) / np.abs(ref)
    rel_abs = np.abs(got - ref) / ref_abs
    plain = np.abs(ref) >= 0.3 * ref_abs
    print(f"N=32768 fp32: max rel err {rel.max():.3e} (non-cancelling: {rel[plain].max():.3e}, "
          f"{plain.sum()} of {len(idx)}), max err / sum|phi| {rel_abs.max():.3e}")
    assert rel_abs.max() <= TOL["fp32"]
    assert rel[plain].max() <= 1e-6


def test_midsize_sampled_both_modes():
    """N = 4096 uniform in [0,16]^3: 64 seeded particles against the oracle."""
    X = inputs.uniform_cube(4096, 16.0, 0.5, 31)
    idx = inputs.sample_indices(len(X), 64, 5)
    _check(_gpu(X, "fp32"), X, "fp32", idx)
    _check(_gpu(X, "fp64"), X, "fp64", idx)


def test_repeat_calls_stable():
    X = inputs.uniform_cube(2000, 10.0, 0.5, 41)
    a = _gpu(X, "fp32")
    b = _gpu(X, "fp32")
    assert _rel(a, b) <= 1e-12


def test_sampled_exact_matches_oracle():
    """The sampled exact kernel (reference for tree accuracy at large N)."""
    X = inputs.uniform_cube(3000, 14.4, 0.5, 57)
    idx = inputs.sample_indices(len(X), 40, 3)
    got = api.potential_sampled(torch.from_numpy(X).cuda(), idx).cpu().numpy()
    ref, ref_abs = oracle.phi(X, idx, with_abs=True)
    assert np.all(np.abs(got - ref) <= TOL["fp32"] * ref_abs)
    # agrees with the full exhaustive FP32 solve on the same particles
    full = _gpu(X, "fp32")[idx]
    assert np.all(np.abs(got - full) <= TOL["fp32"] * ref_abs)


def test_sampled_rejects_out_of_range_index_on_device():
    """Indices are checked on the device too (the C entry point cannot trust
    its caller): an index outside [0, N) is skipped and reported."""
    import ctypes
    X = torch.from_numpy(inputs.uniform_cube(200, 4.0, 0.5, 61)).cuda()
    idx = torch.tensor([0, 5, 200, -1, 7], dtype=torch.int64, device="cuda")
    out = torch.full((5,), 7.0, dtype=torch.float64, device="cuda")
    ctx = api.default_context()
    st = _lib.load().mbm_potential_sampled(ctx.handle, ctypes.c_void_p(X.data_ptr()), 200,
                                           ctypes.c_void_p(idx.data_ptr()), 5,
                                           ctypes.c_void_p(out.data_ptr()), None)
    assert st == -1  # MBM_EINVAL
    o = out.cpu().numpy()
    assert o[2] == 0.0 and o[3] == 0.0
    ref, ref_abs = oracle.phi(X.cpu().numpy(), np.array([0, 5, 7]), with_abs=True)
    assert np.all(np.abs(o[[0, 1, 4]] - ref) <= TOL["fp32"] * ref_abs)
    # the context stays usable
    good = api.potential_sampled(X, [0, 5, 7]).cpu().numpy()
    assert np.all(np.abs(good - o[[0, 1, 4]]) <= 1e-12 * ref_abs)
