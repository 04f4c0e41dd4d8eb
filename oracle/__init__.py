"""CPU oracle for score-only affine-gap (Gotoh) alignment -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never does: it
shares no code, header, table or helper with it.

The numerical work lives in ``gotoh_oracle.c`` (plain C, int64, the
recurrence of Sec. 2.1 of the AnySeq/GPU paper: Eqs. H, E, F and the printed
initialisation tables).  This module compiles it with gcc on first use and
wraps it with ctypes.  ``oracle.brute`` is an independent brute-force
enumerator of all alignments used to pin the DP on tiny inputs.
``oracle.band_features`` and ``oracle.mlp`` define the band predictor's pair
features and its network (float64) and are pinned by tests/test_band_oracle.py.

Every function here is parity-pinned by tests/test_oracle.py (brute force,
closed forms, invariants, hand-worked tables); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

LOCAL, GLOBAL, SEMIGLOBAL = 0, 1, 2
MODES = {"local": LOCAL, "global": GLOBAL, "semiglobal": SEMIGLOBAL, "semi": SEMIGLOBAL}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gotoh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain gcc -O2, no SIMD intrinsics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.oracle_score.restype = i64
        lib.oracle_score.argtypes = [u8p, i64, u8p, i64, i32p, i32, i64, i64, i32, i32p]
        lib.oracle_score_ex.restype = i64
        lib.oracle_score_ex.argtypes = [u8p, i64, u8p, i64, i32p, i32, i64, i64, i32, i32, i32p]
        lib.oracle_matrix.restype = i64
        lib.oracle_matrix.argtypes = [u8p, i64, u8p, i64, i32p, i32, i64, i64, i32, i64p, i32p]
        lib.oracle_score_banded.restype = i64
        lib.oracle_score_banded.argtypes = [u8p, i64, u8p, i64, i32p, i32, i64, i64, i64, i64, i32p]
        lib.oracle_score_blockband.restype = i64
        lib.oracle_score_blockband.argtypes = [u8p, i64, u8p, i64, i32p, i32, i64, i64, i64, i64,
                                               i64, i32p]
        lib.oracle_banded_doubling_blocks.restype = i64
        lib.oracle_banded_doubling_blocks.argtypes = [u8p, i64, u8p, i64, i32p, i32, i64, i64,
                                                      i64, i64, i64p, i64p, i32p]
        lib.oracle_band_ub.restype = i64
        lib.oracle_band_ub.argtypes = [i64, i64, i64, i64, i64, i64]
        lib.oracle_banded_doubling.restype = i64
        lib.oracle_banded_doubling.argtypes = [u8p, i64, u8p, i64, i32p, i32, i64, i64, i64,
                                               i64p, i64p, i32p]
        lib.oracle_min_certified_w.restype = i64
        lib.oracle_min_certified_w.argtypes = [u8p, i64, u8p, i64, i32p, i32, i64, i64, i32p]
        lib.oracle_min_certified_w_blocks.restype = i64
        lib.oracle_min_certified_w_blocks.argtypes = [u8p, i64, u8p, i64, i32p, i32, i64, i64, i64,
                                                      i32p]
        lib.oracle_batch.restype = i32
        lib.oracle_batch.argtypes = [u8p, i64p, u8p, i64p, i64, i32p, i32, i64, i64, i32, i64p,
                                     i32p, i32]
        lib.oracle_cross.restype = i32
        lib.oracle_cross.argtypes = [u8p, i64p, i64, u8p, i64p, i64, i32p, i32, i64, i64, i32,
                                     i64p, i32p, i32]
        _lib = lib
        return lib


class OracleError(RuntimeError):
    pass


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _sigma(matrix):
    s = np.ascontiguousarray(np.asarray(matrix, dtype=np.int32))
    if s.ndim != 2 or s.shape[0] != s.shape[1]:
        raise ValueError("substitution matrix must be square")
    return s, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(s.shape[0])


def _mode(mode):
    return MODES[mode] if isinstance(mode, str) else int(mode)


_ERRS = {1: "argument", 2: "residue code >= alphabet size", 3: "out of memory"}


def score(q, s, matrix, alpha, beta, mode, flags: int = 0) -> int:
    """Score of one pair (query codes q: rows, target codes s: columns)."""
    lib = _load()
    q, qp = _u8(q)
    s, sp = _u8(s)
    sig, sgp, A = _sigma(matrix)
    err = ctypes.c_int32(0)
    r = lib.oracle_score_ex(qp, len(q), sp, len(s), sgp, A, int(alpha), int(beta), _mode(mode),
                            int(flags), ctypes.byref(err))
    if err.value:
        raise OracleError(_ERRS.get(err.value, str(err.value)))
    return int(r)


def score_matrix(q, s, matrix, alpha, beta, mode):
    """(score, H) with H the full (m+1) x (n+1) matrix of Eq. H (small inputs)."""
    lib = _load()
    q, qp = _u8(q)
    s, sp = _u8(s)
    sig, sgp, A = _sigma(matrix)
    H = np.zeros((len(q) + 1, len(s) + 1), dtype=np.int64)
    err = ctypes.c_int32(0)
    r = lib.oracle_matrix(qp, len(q), sp, len(s), sgp, A, int(alpha), int(beta), _mode(mode),
                          H.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(err))
    if err.value:
        raise OracleError(_ERRS.get(err.value, str(err.value)))
    return int(r), H


def score_banded(q, s, matrix, alpha, beta, lo, hi) -> int:
    """Global score restricted to diagonals lo <= j - i <= hi."""
    lib = _load()
    q, qp = _u8(q)
    s, sp = _u8(s)
    sig, sgp, A = _sigma(matrix)
    err = ctypes.c_int32(0)
    r = lib.oracle_score_banded(qp, len(q), sp, len(s), sgp, A, int(alpha), int(beta), int(lo),
                                int(hi), ctypes.byref(err))
    if err.value:
        raise OracleError(_ERRS.get(err.value, str(err.value)))
    return int(r)


def score_blockband(q, s, matrix, alpha, beta, lo, hi, block) -> int:
    """Global score on the band [lo, hi] rounded out to blocks of `block` columns."""
    lib = _load()
    q, qp = _u8(q)
    s, sp = _u8(s)
    sig, sgp, A = _sigma(matrix)
    err = ctypes.c_int32(0)
    r = lib.oracle_score_blockband(qp, len(q), sp, len(s), sgp, A, int(alpha), int(beta),
                                   int(lo), int(hi), int(block), ctypes.byref(err))
    if err.value:
        raise OracleError(_ERRS.get(err.value, str(err.value)))
    return int(r)


def banded_doubling_blocks(q, s, matrix, alpha, beta, w0, block):
    """(score, w_used, retries) of band doubling on block-rounded regions."""
    lib = _load()
    q, qp = _u8(q)
    s, sp = _u8(s)
    sig, sgp, A = _sigma(matrix)
    err = ctypes.c_int32(0)
    w = ctypes.c_int64(0)
    t = ctypes.c_int64(0)
    r = lib.oracle_banded_doubling_blocks(qp, len(q), sp, len(s), sgp, A, int(alpha), int(beta),
                                          int(w0), int(block), ctypes.byref(w), ctypes.byref(t),
                                          ctypes.byref(err))
    if err.value:
        raise OracleError(_ERRS.get(err.value, str(err.value)))
    return int(r), int(w.value), int(t.value)


def band_ub(m, n, sigma_max, alpha, beta, d) -> int:
    """Upper bound on any global path visiting diagonal d (certificate)."""
    return int(_load().oracle_band_ub(int(m), int(n), int(sigma_max), int(alpha), int(beta), int(d)))


def banded_doubling(q, s, matrix, alpha, beta, w0):
    """(score, w_used, retries) of the certified band-doubling procedure."""
    lib = _load()
    q, qp = _u8(q)
    s, sp = _u8(s)
    sig, sgp, A = _sigma(matrix)
    err = ctypes.c_int32(0)
    w = ctypes.c_int64(0)
    t = ctypes.c_int64(0)
    r = lib.oracle_banded_doubling(qp, len(q), sp, len(s), sgp, A, int(alpha), int(beta), int(w0),
                                   ctypes.byref(w), ctypes.byref(t), ctypes.byref(err))
    if err.value:
        raise OracleError(_ERRS.get(err.value, str(err.value)))
    return int(r), int(w.value), int(t.value)


def min_certified_w(q, s, matrix, alpha, beta) -> int:
    lib = _load()
    q, qp = _u8(q)
    s, sp = _u8(s)
    sig, sgp, A = _sigma(matrix)
    err = ctypes.c_int32(0)
    r = lib.oracle_min_certified_w(qp, len(q), sp, len(s), sgp, A, int(alpha), int(beta),
                                   ctypes.byref(err))
    if err.value:
        raise OracleError(_ERRS.get(err.value, str(err.value)))
    return int(r)


def min_certified_w_blocks(q, s, matrix, alpha, beta, block) -> int:
    """Smallest w whose band, rounded out to blocks of `block` columns, certifies."""
    lib = _load()
    q, qp = _u8(q)
    s, sp = _u8(s)
    sig, sgp, A = _sigma(matrix)
    err = ctypes.c_int32(0)
    r = lib.oracle_min_certified_w_blocks(qp, len(q), sp, len(s), sgp, A, int(alpha), int(beta),
                                          int(block), ctypes.byref(err))
    if err.value:
        raise OracleError(_ERRS.get(err.value, str(err.value)))
    return int(r)


def batch(q_codes, q_off, t_codes, t_off, matrix, alpha, beta, mode, nthreads: int = 1):
    """Scores (int64) and per-pair error codes for pairs p: (q_p, t_p) in CSR form."""
    lib = _load()
    qc, qcp = _u8(q_codes)
    qo, qop = _i64(q_off)
    tc, tcp = _u8(t_codes)
    to, top = _i64(t_off)
    npairs = len(qo) - 1
    if len(to) - 1 != npairs:
        raise ValueError("q_off and t_off describe different pair counts")
    sig, sgp, A = _sigma(matrix)
    out = np.zeros(npairs, dtype=np.int64)
    errs = np.zeros(npairs, dtype=np.int32)
    lib.oracle_batch(qcp, qop, tcp, top, npairs, sgp, A, int(alpha), int(beta), _mode(mode),
                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                     errs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(nthreads))
    return out, errs


def cross(q_codes, q_off, t_codes, t_off, matrix, alpha, beta, mode, nthreads: int = 1):
    """Scores [nq, nt] (int64) for every (query, target) combination."""
    lib = _load()
    qc, qcp = _u8(q_codes)
    qo, qop = _i64(q_off)
    tc, tcp = _u8(t_codes)
    to, top = _i64(t_off)
    nq, nt = len(qo) - 1, len(to) - 1
    sig, sgp, A = _sigma(matrix)
    out = np.zeros((nq, nt), dtype=np.int64)
    errs = np.zeros((nq, nt), dtype=np.int32)
    lib.oracle_cross(qcp, qop, nq, tcp, top, nt, sgp, A, int(alpha), int(beta), _mode(mode),
                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                     errs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(nthreads))
    return out, errs
