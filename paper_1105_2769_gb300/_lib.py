"""ctypes binding of ``libmbm.so`` (argument marshalling only).

Every function here forwards plain pointers, sizes and a stream handle to
the C ABI declared in ``include/mbm.h``; all computation happens in the
library's CUDA kernels. Loading fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmbm.so")

MBM_OK, MBM_PENDING = 0, 1
STATUS_NAMES = {0: "MBM_OK", 1: "MBM_PENDING", -1: "MBM_EINVAL", -2: "MBM_ENOMEM",
                -3: "MBM_EBUDGET", -4: "MBM_EOVERFLOW", -5: "MBM_ETIMEDOUT",
                -6: "MBM_ECUDA", -7: "MBM_ENOTSUP"}
MBM_EXH_FP64, MBM_EXH_FP32, MBM_TREE, MBM_ABS = 0, 1, 2, 0x100


class MbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("leaf_size", ctypes.c_int32),
                ("m_limit", ctypes.c_int32), ("zeta", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("mc_rule", ctypes.c_int32),
                ("validate", ctypes.c_int32), ("seed_levels", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("tuple_counts", ctypes.c_void_p),
                ("trav_chunk", ctypes.c_int32), ("base_cap", ctypes.c_int32),
                ("est_cap", ctypes.c_int32), ("reserved1", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("node_triples_visited", ctypes.c_int64), ("det_prunes", ctypes.c_int64),
                ("mc_prunes", ctypes.c_int64), ("mc_attempts", ctypes.c_int64),
                ("base_cases", ctypes.c_int64), ("base_triples", ctypes.c_int64),
                ("mc_samples", ctypes.c_int64), ("levels", ctypes.c_int64),
                ("ms_build", ctypes.c_double), ("ms_seed", ctypes.c_double),
                ("ms_traverse", ctypes.c_double), ("ms_base", ctypes.c_double),
                ("ms_finalize", ctypes.c_double), ("chunks", ctypes.c_int64),
                ("base_flushes", ctypes.c_int64), ("mc_batches", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_lock = threading.Lock()

_vp, _i64, _dbl, _int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int

class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("mode", ctypes.c_int32), ("N", ctypes.c_int64),
                ("X_host", ctypes.c_void_p), ("out_host", ctypes.c_void_p),
                ("eps", ctypes.c_double), ("alpha", ctypes.c_double),
                ("system_id", ctypes.c_uint64), ("cfg", ctypes.POINTER(Config))]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("queue_ms", ctypes.c_double), ("compute_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("bytes_reserved", ctypes.c_int64),
                ("dev_start_ns", ctypes.c_int64), ("dev_end_ns", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


MBM_REQ_POTENTIAL, MBM_REQ_FORCES = 0, 1

# name -> (restype, argtypes); mirrors include/mbm.h
SIGNATURES = {
    "mbm_version": (ctypes.c_char_p, []),
    "mbm_last_error": (ctypes.c_char_p, []),
    "mbm_config_default": (None, [ctypes.POINTER(Config)]),
    "mbm_ctx_create": (_int, [_int, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "mbm_ctx_destroy": (_int, [_vp]),
    "mbm_ctx_bytes_in_use": (ctypes.c_size_t, [_vp]),
    "mbm_ctx_set_timing": (_int, [_vp, _int]),
    "mbm_ctx_last_kernel_ms": (ctypes.c_double, [_vp]),
    "mbm_potential": (_int, [_vp, _vp, _i64, _dbl, _dbl, _int, _vp, _vp]),
    "mbm_potential_ex": (_int, [_vp, _vp, _i64, _dbl, _dbl, _int, ctypes.POINTER(Config), _vp,
                                _vp, ctypes.POINTER(Stats), _vp]),
    "mbm_potential_host": (_int, [_vp, _vp, _i64, _dbl, _dbl, _int, ctypes.POINTER(Config),
                                  _vp, _vp]),
    "mbm_forces": (_int, [_vp, _vp, _i64, _dbl, _dbl, _int, _vp, _vp]),
    "mbm_forces_ex": (_int, [_vp, _vp, _i64, _dbl, _dbl, _int, ctypes.POINTER(Config), _vp, _vp,
                             ctypes.POINTER(Stats), _vp]),
    "mbm_potential_vjp": (_int, [_vp, _vp, _i64, _vp, _int, _vp, _vp]),
    "mbm_potential_fp32_noalloc": (_int, [_vp, _i64, _vp, _vp]),
    "mbm_tree_build": (_int, [_vp, _vp, _i64, ctypes.POINTER(Config), _vp, ctypes.POINTER(_vp)]),
    "mbm_tree_free": (_int, [_vp]),
    "mbm_tree_info": (_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                             ctypes.POINTER(ctypes.c_int32)]),
    "mbm_tree_export": (_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mbm_potential_sampled": (_int, [_vp, _vp, _i64, _vp, _i64, _vp, _vp]),
    "mbm_farfield3": (_int, [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _int, _int, _vp, _vp]),
    "mbm_server_create": (_int, [_int, ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(_vp)]),
    "mbm_server_destroy": (_int, [_vp]),
    "mbm_submit": (_int, [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "mbm_poll": (_int, [_vp, ctypes.c_uint64, ctypes.POINTER(Result), _i64]),
    "mbm_server_stats": (_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                ctypes.POINTER(ctypes.c_size_t)]),
}
OPTIONAL = {}


def load():
    """Load the library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in {**SIGNATURES, **OPTIONAL}.items():
                if not hasattr(L, name):
                    if name in OPTIONAL:
                        continue
                    raise ImportError(f"libmbm.so does not export {name}")
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status):
    if status != MBM_OK:
        msg = load().mbm_last_error()
        raise MbmError(status, msg.decode() if msg else "")
    return status


def default_config(**overrides) -> Config:
    c = Config()
    load().mbm_config_default(ctypes.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c
