"""FP64 CPU oracle for the CountGauss transform T.X = G.(S.X).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only code that may import this package.  The CUDA library
never links, loads or calls it, and it shares no code with the CUDA library (its
Philox, hash, Box-Muller and scatter are its own, in ``cg_oracle.c``).

The arithmetic lives in ``cg_oracle.c`` (plain C, double precision, naive loops);
this module compiles it with gcc on first use and marshals numpy arrays.  Each
wrapper names the passage of the paper it follows; the stream layout (which Philox
counter feeds which hash bucket, sign or Gaussian entry) is documented at the top of
``cg_oracle.c``.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(independent Philox from a library, closed forms, invariants, brute force and
exact moment identities).  Nothing is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libcg_oracle.so")

TAG_HASH = 0
TAG_G = 1
TAG_GTILDE = 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile cg_oracle.c into a shared library (gcc, -O2, IEEE arithmetic)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, u64, u32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32
            sigs = {
                "orc_philox4x32_10": [P, P, P],
                "orc_philox_words": [u64, u32, u64, i64, P],
                "orc_hash_sign": [u64, i64, i64, i64, P, P],
                "orc_box_muller_words": [P, i64, P],
                "orc_gaussian_block": [u64, u32, i64, i64, i64, i64, i64, P],
                "orc_sketch_csr": [u64, i64, i64, i64, i64, P, P, P, P],
                "orc_sketch_dense": [u64, i64, i64, i64, i64, P, P],
                "orc_contract": [u64, i64, i64, i64, P, P],
                "orc_contract_range": [u64, i64, i64, i64, i64, i64, P, P],
                "orc_apply_csr": [u64, i64, i64, i64, i64, i64, P, P, P, P, P],
                "orc_apply_dense": [u64, i64, i64, i64, i64, i64, P, P, P],
                "orc_plain_csr": [u64, i64, i64, i64, i64, P, P, P, i64, P, P],
                "orc_plain_dense": [u64, i64, i64, i64, i64, P, P],
                "orc_adjoint_w": [u64, i64, i64, i64, P, P],
                "orc_adjoint_dense": [u64, i64, i64, i64, i64, i64, P, P, P],
                "orc_adjoint_csr": [u64, i64, i64, i64, i64, i64, P, P, P, P, P],
                "orc_row_argmax_argmin": [i64, i64, P, P, P],
                "orc_apply_right_csr": [u64, i64, i64, i64, i64, i64, P, P, P, P],
            }
            for name, args in sigs.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = None
            lib.orc_uniform24.argtypes = [u32]
            lib.orc_uniform24.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------------
# Generator layer: Philox4x32-10 (SC'11), hash/sign (Section 1.1, Section 7),
# uniforms and Box-Muller normals for the unit-variance Gaussians of Theorem 1.
# --------------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: ctr (4 uint32), key (2 uint32) -> 4 uint32 words."""
    lib = _load()
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_words(seed: int, tag: int, idx0: int, count: int) -> np.ndarray:
    """Words of the stream layout for idx0..idx0+count-1: shape (count, 4) uint32."""
    lib = _load()
    out = np.zeros((count, 4), np.uint32)
    lib.orc_philox_words(seed, tag, idx0, count, _ptr(out))
    return out


def hash_sign(seed: int, B: int, row0: int, count: int):
    """CountSketch bucket h(i) in [0,B) and sign sigma(i) in {-1,+1} for global rows
    row0..row0+count-1 (Section 1.1; Section 7): word i mod 4 of the tag-0 call at
    floor(i/4), its multiply-high by B and its lowest bit."""
    lib = _load()
    h = np.zeros(count, np.int64)
    s = np.zeros(count, np.int32)
    lib.orc_hash_sign(seed, B, row0, count, _ptr(h), _ptr(s))
    return h, s


def uniform24(w: int) -> float:
    """u(w) = (2*(w>>9)+1) * 2^-24."""
    return _load().orc_uniform24(int(w))


def box_muller_words(words) -> np.ndarray:
    """Four normals per row of a (count, 4) uint32 word array."""
    lib = _load()
    w = _c(words, np.uint32).reshape(-1, 4)
    z = np.zeros(w.shape, np.float64)
    lib.orc_box_muller_words(_ptr(w), w.shape[0], _ptr(z))
    return z


def gaussian_block(seed: int, tag: int, R: int, r0: int, r1: int, c0: int, c1: int) -> np.ndarray:
    """Rows [r0,r1) x cols [c0,c1) of the R x C unit-variance Gaussian with `tag`
    (G: tag 1, R = m; G~: tag 2, R = m)."""
    lib = _load()
    out = np.zeros((r1 - r0, c1 - c0), np.float64)
    lib.orc_gaussian_block(seed, tag, R, r0, r1, c0, c1, _ptr(out))
    return out


def gaussian_G(seed: int, m: int, B: int) -> np.ndarray:
    """The full m x B matrix G of Theorem 1 (tiny sizes only)."""
    return gaussian_block(seed, TAG_G, m, 0, m, 0, B)


# --------------------------------------------------------------------------------
# The transform (Section 1.1; Algorithm 1 steps 1-2), the plain product (Abstract;
# Section 4) and the adjoint.
# --------------------------------------------------------------------------------
def _csr(row_ptr, col_idx, vals):
    return _c(row_ptr, np.int64), _c(col_idx, np.int64), _c(vals, np.float64)


def sketch_csr(seed, n, d, B, row_ptr, col_idx, vals, row_offset=0) -> np.ndarray:
    lib = _load()
    rp, ci, v = _csr(row_ptr, col_idx, vals)
    SX = np.zeros((B, d), np.float64)
    lib.orc_sketch_csr(seed, n, d, B, row_offset, _ptr(rp), _ptr(ci), _ptr(v), _ptr(SX))
    return SX


def sketch_dense(seed, B, X, row_offset=0) -> np.ndarray:
    lib = _load()
    X = _c(X, np.float64)
    n, d = X.shape
    SX = np.zeros((B, d), np.float64)
    lib.orc_sketch_dense(seed, n, d, B, row_offset, _ptr(X), _ptr(SX))
    return SX


def contract(seed, m, SX) -> np.ndarray:
    lib = _load()
    SX = _c(SX, np.float64)
    B, d = SX.shape
    Y = np.zeros((m, d), np.float64)
    lib.orc_contract(seed, m, B, d, _ptr(SX), _ptr(Y))
    return Y


def contract_range(seed, m, SX, b0, b1) -> np.ndarray:
    """The part of G.SX that columns b0 <= b < b1 of G contribute (m x d float64)."""
    lib = _load()
    SX = _c(SX, np.float64)
    B, d = SX.shape
    Y = np.zeros((m, d), np.float64)
    lib.orc_contract_range(seed, m, B, d, b0, b1, _ptr(SX), _ptr(Y))
    return Y


def _row_cuts(n, parts):
    return [n * k // parts for k in range(parts + 1)]


def apply_csr_parallel(seed, n, d, m, B, row_ptr, col_idx, vals, threads, row_offset=0, b_range=None):
    """Y = G.(S.X) for CSR X with the work spread over `threads` host threads: the
    sketch of each of `threads` row shards (global row offsets, the sharding remark of
    Section 4) and the contraction of each of `threads` ranges of the columns of G, each
    by the single-threaded functions above (the C calls release the interpreter lock),
    the shards' m x d or B x d results summed in FP64.  With b_range = (b0, b1) only
    columns b0 <= b < b1 of G are contracted (a part of the whole contraction)."""
    from concurrent.futures import ThreadPoolExecutor
    lib = _load()
    rp, ci, v = _csr(row_ptr, col_idx, vals)
    threads = max(1, int(threads))
    cuts = _row_cuts(n, threads)

    def sketch_part(k):
        a, b = cuts[k], cuts[k + 1]
        SXk = np.zeros((B, d), np.float64)
        rpk = np.ascontiguousarray(rp[a:b + 1])
        lib.orc_sketch_csr(seed, b - a, d, B, row_offset + a, _ptr(rpk), _ptr(ci), _ptr(v), _ptr(SXk))
        return SXk

    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(sketch_part, range(threads)))
    SX = parts[0]
    for P_ in parts[1:]:
        SX += P_
    del parts
    b0, b1 = (0, B) if b_range is None else b_range
    bcuts = [b0 + (b1 - b0) * k // threads for k in range(threads + 1)]

    def contract_part(k):
        Yk = np.zeros((m, d), np.float64)
        lib.orc_contract_range(seed, m, B, d, bcuts[k], bcuts[k + 1], _ptr(SX), _ptr(Yk))
        return Yk

    with ThreadPoolExecutor(threads) as ex:
        Ys = list(ex.map(contract_part, range(threads)))
    return sum(Ys[1:], Ys[0])


def apply_csr(seed, n, d, m, B, row_ptr, col_idx, vals, row_offset=0, return_sx=False):
    """Y = G.(S.X) for CSR X, m x d float64."""
    lib = _load()
    rp, ci, v = _csr(row_ptr, col_idx, vals)
    SX = np.zeros((B, d), np.float64)
    Y = np.zeros((m, d), np.float64)
    lib.orc_apply_csr(seed, n, d, m, B, row_offset, _ptr(rp), _ptr(ci), _ptr(v), _ptr(SX), _ptr(Y))
    return (Y, SX) if return_sx else Y


def apply_dense(seed, m, B, X, row_offset=0, return_sx=False):
    lib = _load()
    X = _c(X, np.float64)
    n, d = X.shape
    SX = np.zeros((B, d), np.float64)
    Y = np.zeros((m, d), np.float64)
    lib.orc_apply_dense(seed, n, d, m, B, row_offset, _ptr(X), _ptr(SX), _ptr(Y))
    return (Y, SX) if return_sx else Y


def apply_right_csr(seed, n, d, m, B, row_ptr, col_idx, vals, col_offset=0) -> np.ndarray:
    """Z = A.T^T, d x m float64, for a d x n CSR matrix A with one row per sample (the
    projection X.R, R = T^T, of Section 9 and Table 1).  Column c of A is the global
    index col_offset + c of T's columns."""
    lib = _load()
    rp, ci, v = _csr(row_ptr, col_idx, vals)
    Z = np.zeros((d, m), np.float64)
    lib.orc_apply_right_csr(seed, n, d, m, B, col_offset, _ptr(rp), _ptr(ci), _ptr(v), _ptr(Z))
    return Z


def plain_csr(seed, n, d, m, row_ptr, col_idx, vals, rows=None, row_offset=0) -> np.ndarray:
    """Rows `rows` (default: all m) of G~.X for CSR X; G~ is m x n_global, tag 2."""
    lib = _load()
    rp, ci, v = _csr(row_ptr, col_idx, vals)
    rows = np.arange(m, dtype=np.int64) if rows is None else _c(rows, np.int64)
    Y = np.zeros((rows.size, d), np.float64)
    lib.orc_plain_csr(seed, n, d, m, row_offset, _ptr(rp), _ptr(ci), _ptr(v), rows.size,
                      _ptr(rows), _ptr(Y))
    return Y


def plain_dense(seed, m, X, row_offset=0) -> np.ndarray:
    lib = _load()
    X = _c(X, np.float64)
    n, d = X.shape
    Y = np.zeros((m, d), np.float64)
    lib.orc_plain_dense(seed, n, d, m, row_offset, _ptr(X), _ptr(Y))
    return Y


def adjoint_w(seed, m, B, dY) -> np.ndarray:
    """W = G^T dY, B x d."""
    lib = _load()
    dY = _c(dY, np.float64)
    d = dY.shape[1]
    W = np.zeros((B, d), np.float64)
    lib.orc_adjoint_w(seed, m, B, d, _ptr(dY), _ptr(W))
    return W


def adjoint_dense(seed, n, m, B, dY, row_offset=0) -> np.ndarray:
    """dX = S^T G^T dY, n x d."""
    lib = _load()
    dY = _c(dY, np.float64)
    d = dY.shape[1]
    W = np.zeros((B, d), np.float64)
    dX = np.zeros((n, d), np.float64)
    lib.orc_adjoint_dense(seed, n, d, m, B, row_offset, _ptr(dY), _ptr(W), _ptr(dX))
    return dX


def adjoint_csr(seed, n, m, B, row_ptr, col_idx, dY, row_offset=0) -> np.ndarray:
    """dX = S^T G^T dY read at the nonzeros of a CSR pattern: nnz values."""
    lib = _load()
    rp = _c(row_ptr, np.int64)
    ci = _c(col_idx, np.int64)
    dY = _c(dY, np.float64)
    d = dY.shape[1]
    W = np.zeros((B, d), np.float64)
    dXv = np.zeros(ci.size, np.float64)
    lib.orc_adjoint_csr(seed, n, d, m, B, row_offset, _ptr(rp), _ptr(ci), _ptr(dY), _ptr(W),
                        _ptr(dXv))
    return dXv


def row_argmax_argmin(Z):
    """Algorithm 1 step 3: per row of Z, the column of its max and of its min
    (lowest index on ties)."""
    lib = _load()
    Z = _c(Z, np.float64)
    m, d = Z.shape
    imax = np.zeros(m, np.int64)
    imin = np.zeros(m, np.int64)
    lib.orc_row_argmax_argmin(m, d, _ptr(Z), _ptr(imax), _ptr(imin))
    return imax, imin
