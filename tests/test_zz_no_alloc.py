"""The allocation-free exhaustive entry point (mbm_potential_fp32_noalloc).

Callers that cannot let a library allocate device memory (applications that
own every device byte through their own pool, loops that cannot afford the
synchronisation of an allocation, plugins in processes that forbid foreign
allocations) use this entry point; its scratch is a fixed device array.
The test calls it through the C ABI twice in a row, on two sizes, and checks
each result against the regular FP32 entry point and against the FP64 oracle
with the FP32 bar 3e-6, relative to sum_t (1 + 3|cos cos cos|)/(r r r)^3, the
magnitudes of each term's two parts: on these dense cubes (d_min 0.05) some
near-collinear triples cancel inside the term (1 + 3 cos cos cos near 0), so
sum_t |phi_t| understates the rounding scale by up to 72x. It lives in a file
collected last so that a failure here cannot hide another test's."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1105_2769_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu


def _noalloc(Xd, out):
    L = _lib.load()
    st = L.mbm_potential_fp32_noalloc(ctypes.c_void_p(Xd.data_ptr()), Xd.shape[0],
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(st)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("n,seed", [(1000, 91), (333, 92)])
def test_noalloc_matches_regular_entry_point(n, seed):
    X = inputs.uniform_cube(n, 4.0, 0.05, seed)
    Xd = torch.from_numpy(X).cuda()
    ref = api.potential(Xd, mode="fp32").cpu().numpy()
    exact = oracle.phi(X)
    parts = oracle.phi_parts(X)
    for _ in range(2):  # two calls in a row share the static scratch
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        got = _noalloc(Xd, out)
        print("max err / parts: vs regular", np.max(np.abs(got - ref) / parts),
              "vs oracle", np.max(np.abs(got - exact) / parts))
        assert np.all(np.abs(got - ref) <= 3e-6 * parts)
        assert np.all(np.abs(got - exact) <= 3e-6 * parts)


def test_noalloc_rejects_oversize():
    L = _lib.load()
    n = 65537
    st = L.mbm_potential_fp32_noalloc(ctypes.c_void_p(1), n, ctypes.c_void_p(1), None)
    assert st == -1
    assert b"65536" in L.mbm_last_error()
