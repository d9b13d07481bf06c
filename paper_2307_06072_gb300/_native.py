"""ctypes binding of ``libmpcgemm.so`` (argument marshalling only).

Every function here forwards to the C ABI declared in ``include/mpcgemm.h``;
no step of the computation runs in Python.  Device memory and streams come
from PyTorch.  If the library is missing the import fails loudly: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpcgemm.so")

MPC_OK, MPC_EINVAL, MPC_ENOSPC, MPC_ERANGE, MPC_ENOTSUP, MPC_ECUDA = 0, -22, -28, -34, -95, -1000
METHODS = {"4m": 0, "3m": 1}
ALGOS = {"plain": 0, "ozaki": 1}
KERNELS = {"auto": 0, "tcgen05": 1, "mma_sync": 2, "tcgen05_2sm": 4, "tcgen05_n128": 5, "tcgen05_2sm_n128": 6}

EXPORTED = ("mpcgemm", "mpcgemm_ex", "mpcgemm_profiled", "mpcgemm_workspace_size", "mpcgemm_plan",
            "mpcgemm_read_status", "mpcgemm_noalloc", "mpcgemm_noalloc_read_status", "mpcgemm_batched", "mpcgemm_batched_workspace",
            "mpcgesv", "mpcgesv_workspace_size", "mpcgemm_strerror", "mpcgemm_version")
NOALLOC_SCRATCH_BYTES = 64 << 20


class MpcMat(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("sign", ctypes.c_void_p * 2), ("exp", ctypes.c_void_p * 2), ("limb", ctypes.c_void_p * 2)]


class OzParams(ctypes.Structure):
    _fields_ = [("guard_bits", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("cut_level", ctypes.c_int32), ("kernel", ctypes.c_int32), ("max_group", ctypes.c_int32),
                ("digit_bits", ctypes.c_int32), ("wait_limit_cycles", ctypes.c_int32), ("dump_accumulators", ctypes.c_int32),
                ("split", ctypes.c_int32), ("pair_planes", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class MpcProblem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64), ("p_bits", ctypes.c_int32),
                ("method", ctypes.c_int32), ("algo", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p)]


class Plan(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("method", ctypes.c_int32), ("p_bits", ctypes.c_int32),
                ("limbs", ctypes.c_int32), ("s", ctypes.c_int32), ("Q", ctypes.c_int32),
                ("kpad", ctypes.c_int32), ("gmax", ctypes.c_int32), ("n_products", ctypes.c_int32),
                ("n_groups_total", ctypes.c_int32), ("n_groups", ctypes.c_int32 * 4),
                ("planes_A", ctypes.c_int32), ("planes_B", ctypes.c_int32), ("acc_slots", ctypes.c_int32),
                ("bound_shift", ctypes.c_int32), ("bound_drop", ctypes.c_uint64 * 2),
                ("bound_lossy_a", ctypes.c_uint64 * 2), ("bound_lossy_b", ctypes.c_uint64 * 2),
                ("off_status", ctypes.c_uint64), ("off_rowexp", ctypes.c_uint64), ("off_colexp", ctypes.c_uint64),
                ("off_rowlossy", ctypes.c_uint64), ("off_collossy", ctypes.c_uint64),
                ("off_digits_a", ctypes.c_uint64), ("off_digits_b", ctypes.c_uint64),
                ("off_groups", ctypes.c_uint64), ("off_group_table", ctypes.c_uint64),
                ("off_fallback", ctypes.c_uint64), ("fallback_capacity", ctypes.c_uint64),
                ("off_fb_scratch", ctypes.c_uint64), ("fb_scratch_limbs", ctypes.c_uint64),
                ("fb_threads", ctypes.c_uint64), ("off_acc_dump", ctypes.c_uint64), ("off_units", ctypes.c_uint64),
                ("ws_bytes", ctypes.c_uint64), ("launches", ctypes.c_int32), ("digit_bits", ctypes.c_int32),
                ("off_group_order", ctypes.c_uint64), ("split", ctypes.c_int32), ("pair_batch", ctypes.c_int32)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else int(v)
        return out


class StageEvents(ctypes.Structure):
    _fields_ = [("ev", ctypes.c_void_p * 8)]


class Status(ctypes.Structure):
    _fields_ = [("erange", ctypes.c_int32), ("fallback_entries", ctypes.c_int32),
                ("fallback_overflow", ctypes.c_int32), ("uncertified", ctypes.c_int32),
                ("device_timeout", ctypes.c_int32)]


_lib = None


def lib():
    """The loaded C library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2307_06072_gb300.build.build() "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.mpcgemm.argtypes = [I64, I64, I64, I32, P, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P]
        L.mpcgemm.restype = ctypes.c_int
        L.mpcgemm_ex.argtypes = [I64, I64, I64, I32, P, P, P, ctypes.c_int, ctypes.c_int, P, P,
                                 ctypes.c_size_t, P]
        L.mpcgemm_ex.restype = ctypes.c_int
        L.mpcgemm_profiled.argtypes = [I64, I64, I64, I32, P, P, P, ctypes.c_int, ctypes.c_int, P, P, P,
                                       ctypes.c_size_t, P]
        L.mpcgemm_profiled.restype = ctypes.c_int
        L.mpcgemm_workspace_size.argtypes = [I64, I64, I64, I32, ctypes.c_int, ctypes.c_int]
        L.mpcgemm_workspace_size.restype = ctypes.c_size_t
        L.mpcgemm_plan.argtypes = [I64, I64, I64, I32, ctypes.c_int, ctypes.c_int, P, P]
        L.mpcgemm_plan.restype = ctypes.c_int
        L.mpcgemm_read_status.argtypes = [P, ctypes.c_size_t, P, P]
        L.mpcgemm_read_status.restype = ctypes.c_int
        L.mpcgemm_batched.argtypes = [ctypes.c_int, P, P, P, ctypes.c_size_t, P]
        L.mpcgemm_batched.restype = ctypes.c_int
        L.mpcgemm_batched_workspace.argtypes = [ctypes.c_int, P, P, P, P]
        L.mpcgemm_batched_workspace.restype = ctypes.c_int
        L.mpcgesv.argtypes = [I64, I32, P, P, P, I32, ctypes.c_int, P, ctypes.c_size_t, P]
        L.mpcgesv.restype = ctypes.c_int
        L.mpcgesv_workspace_size.argtypes = [I64, I32, I32, ctypes.c_int]
        L.mpcgesv_workspace_size.restype = ctypes.c_size_t
        L.mpcgemm_noalloc.argtypes = [I64, I64, I64, I32, P, P, P, ctypes.c_int, ctypes.c_int, P]
        L.mpcgemm_noalloc.restype = ctypes.c_int
        L.mpcgemm_noalloc_read_status.argtypes = [P, P]
        L.mpcgemm_noalloc_read_status.restype = ctypes.c_int
        L.mpcgemm_strerror.argtypes = [ctypes.c_int]
        L.mpcgemm_strerror.restype = ctypes.c_char_p
        L.mpcgemm_version.argtypes = []
        L.mpcgemm_version.restype = ctypes.c_int
        _lib = L
    return _lib


class MPCError(RuntimeError):
    def __init__(self, code: int):
        self.code = code
        super().__init__(f"mpcgemm error {code}: {strerror(code)}")


def strerror(code: int) -> str:
    return lib().mpcgemm_strerror(int(code)).decode()


def check(code: int) -> int:
    if code != MPC_OK:
        raise MPCError(code)
    return code


SPLITS = {"common": 0, "per_part": 1, "residual": 2}


def oz_params(guard_bits=0, slices=0, cut_level=0, kernel="auto", max_group=0, digit_bits=0,
              wait_limit_cycles=0, dump_accumulators=0, split="common", pair_planes=0) -> OzParams:
    return OzParams(int(guard_bits), int(slices), int(cut_level), KERNELS[kernel] if isinstance(kernel, str)
                    else int(kernel), int(max_group), int(digit_bits), int(wait_limit_cycles),
                    int(dump_accumulators), SPLITS[split] if isinstance(split, str) else int(split),
                    int(pair_planes))


def exported_symbols():
    """Names the header declares; all must resolve in the loaded library."""
    L = lib()
    return {name: getattr(L, name) for name in EXPORTED}


def np_ptr(a: np.ndarray) -> int:
    return a.ctypes.data
