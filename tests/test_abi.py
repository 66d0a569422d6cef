"""Host-side checks of the C-ABI library: it builds, loads, and exports every
symbol that include/*.h declares. No compute call is made (no GPU needed)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mbm_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1105_2769_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_entry_points():
    names = _declared_symbols()
    for required in ["mbm_ctx_create", "mbm_potential", "mbm_forces", "mbm_potential_vjp",
                     "mbm_last_error", "mbm_potential_host"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared_symbols()) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_declared_symbol():
    from paper_1105_2769_gb300 import _lib
    bound = set(_lib.SIGNATURES) | set(_lib.OPTIONAL)
    missing = sorted(_declared_symbols() - bound)
    assert not missing, f"declared but not bound in Python: {missing}"


def test_version_and_defaults(lib):
    from paper_1105_2769_gb300 import _lib
    assert b"sm_103a" in lib.mbm_version()
    c = _lib.default_config()
    assert c.leaf_size == 32 and c.m_limit == 256 and c.zeta == 32.0 and c.validate == 1
    assert c.seed_levels == 8 and not c.tuple_counts


def test_ctx_create_without_gpu_fails_cleanly(lib):
    """With no GPU the context call must return an error status, not crash."""
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.mbm_ctx_create(0, 0, ctypes.byref(h))
    assert st != 0
    assert lib.mbm_last_error()


def test_null_and_bad_arguments_rejected_on_host(lib):
    import ctypes
    from paper_1105_2769_gb300 import _lib
    # NULL context is rejected before any CUDA call
    st = lib.mbm_potential(None, None, 10, 0.0, 0.0, 1, None, None)
    assert st == -1
    st = lib.mbm_forces(None, None, 10, 0.0, 0.0, 1, None, None)
    assert st in (-1, -7)
    assert lib.mbm_ctx_destroy(None) == 0
    assert _lib.STATUS_NAMES[-1] == "MBM_EINVAL"
    # far-field expansion: NULL context, then order checks, before any CUDA call
    assert lib.mbm_farfield3(None, None, 4, None, 3, None, 3, 2, 1, None, None) == -1
    assert b"ctx" in lib.mbm_last_error()
