"""ctypes loader for libcountgauss.so (the C ABI of include/countgauss.h).

The library is built in-tree by ``paper_1606_05732_gb300.build``.  Loading fails
loudly when it is missing: there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

CG_OK = 0
STATUS_NAMES = {
    0: "CG_OK", 1: "CG_ERR_INVALID_ARG", 2: "CG_ERR_UNSUPPORTED", 3: "CG_ERR_WORKSPACE",
    4: "CG_ERR_CUDA", 5: "CG_ERR_TIMEOUT", 6: "CG_ERR_DEVICE_BOUNDS", 7: "CG_ERR_NO_DEVICE",
}

PREC = {"fp32": 0, "bf16": 1, "bf16x3": 2, "fp8": 3, "fp8x3": 4}
OPT_PRECISION, OPT_DETERMINISTIC, OPT_ROW_OFFSET, OPT_KSPLIT, OPT_SKETCH_CTAS, OPT_TIMING = 1, 2, 3, 4, 5, 6
OPT_SCATTER, OPT_SCATTER_PASSES, OPT_SCATTER_ROWS = 7, 8, 9
SCATTER = {"auto": 0, "atomic": 1, "partition": 2, "deferred": 3, "binned": 4}
KERNEL_SKETCH, KERNEL_CONTRACT, KERNEL_PLAIN, KERNEL_ADJOINT_W, KERNEL_GATHER = range(5)
OP_APPLY_CSR, OP_APPLY_DENSE, OP_ADJOINT_DENSE, OP_ADJOINT_CSR, OP_PLAIN_CSR, OP_SKETCH, OP_CONTRACT = range(7)
OP_APPLY_CSR_HOST = 7
OP_APPLY_RIGHT_CSR = 8
OP_APPLY_CSR_I64 = 9
OP_SKETCH_I64 = 10
OPT_HOST_CHUNK = 10
OPT_HOST_READ = 11
OPT_ACCUMULATE = 12
HOST_READ = {"auto": 0, "copied": 1, "direct": 2}

P = ctypes.c_void_p
I32, I64, U32, U64, SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t

# name -> argtypes (every entry point returns cg_status as int)
SIGNATURES = {
    "cg_plan_create": [I64, I32, I32, I64, U64, ctypes.POINTER(P)],
    "cg_plan_destroy": [P],
    "cg_plan_set_option": [P, I32, I64],
    "cg_plan_get_option": [P, I32, ctypes.POINTER(I64)],
    "cg_workspace_size": [P, I32, I64, ctypes.POINTER(SZ)],
    "cg_plan_check": [P, P, P],
    "cg_plan_timing": [P, I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)],
    "cg_apply_csr": [P, P, P, P, I64, P, P, SZ, P],
    "cg_apply_right_csr": [P, P, P, P, I64, P, P, SZ, P],
    "cg_apply_csr_i64": [P, P, P, P, I64, P, P, SZ, P],
    "cg_sketch_csr_i64": [P, P, P, P, I64, P, P, SZ, P],
    "cg_apply_csr_host": [P, P, P, P, I64, P, P, SZ, P],
    "cg_apply_csr_noalloc": [P, P, P, P, I64, P, P],
    "cg_apply_dense": [P, P, I64, P, P, SZ, P],
    "cg_apply_adjoint": [P, P, P, P, I64, P, P, SZ, P],
    "cg_apply_adjoint_i64": [P, P, P, P, I64, P, P, SZ, P],
    "cg_plain_gaussian_apply": [P, P, P, P, I64, P, P, SZ, P],
    "cg_sketch_csr": [P, P, P, P, I64, P, P, SZ, P],
    "cg_sketch_dense": [P, P, I64, P, P, SZ, P],
    "cg_contract": [P, P, P, P, SZ, P],
    "cg_row_argmax_argmin": [P, I32, I32, P, P, P],
    "cg_nmf_anchors_csr": [P, P, P, P, I64, P, P, P, P, SZ, P],
    "cg_nmf_anchors_csr_i64": [P, P, P, P, I64, P, P, P, P, SZ, P],
    "cg_moments_f64": [P, I64, I32, P, P, P],
    "cg_batch_plan_create": [P, I32, ctypes.POINTER(P)],
    "cg_batch_plan_destroy": [P],
    "cg_batch_set_option": [P, I32, I64],
    "cg_batch_plan_get_option": [P, I32, ctypes.POINTER(I64)],
    "cg_batch_workspace_size": [P, ctypes.POINTER(SZ)],
    "cg_batch_apply": [P, P, SZ, P],
    "cg_batch_check": [P, P, P],
    "cg_batch_autotune": [P, P, SZ, P, I32, ctypes.POINTER(ctypes.c_double)],
    "cg_generate_words": [U64, U32, U64, I64, P, P],
    "cg_generate_hash_sign": [U64, I64, I64, I64, P, P, P],
    "cg_generate_gaussian": [U64, U32, I64, I64, I64, I64, I64, P, P],
    "cg_diag_random_reductions": [P, I64, I64, P],
}


BATCH_OPT_GRAPH, BATCH_OPT_SCATTER_NNZ, BATCH_OPT_CONTRACT_FMA, BATCH_OPT_CTAS_PER_SM = 1, 2, 3, 4
BATCH_OPT_WAIT_US, BATCH_OPT_TEST_DROP_SCATTER_ITEM = 5, 6


class BatchDesc(ctypes.Structure):
    """cg_batch_desc."""
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("m", ctypes.c_int32), ("B", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("vals", ctypes.c_void_p), ("nnz", ctypes.c_int64), ("Y", ctypes.c_void_p)]


class CountGaussError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} returned {STATUS_NAMES.get(status, status)}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcountgauss.so (building it first if it is absent and allowed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libcountgauss.so is not built ({path}); run paper_1606_05732_gb300.build")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, args in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.cg_status_string.argtypes = [ctypes.c_int]
        lib.cg_status_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def check(fn: str, status: int) -> None:
    if status != CG_OK:
        raise CountGaussError(fn, status)


def call(name: str, *args) -> None:
    """Call an entry point and raise CountGaussError on a non-OK status."""
    check(name, getattr(load(), name)(*args))
