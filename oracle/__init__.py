"""CPU oracle for Smith-Waterman/Gotoh database search -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product path (``paper_1702_07195_gb300``) never imports it and has
no CPU fallback.

The arithmetic lives in ``sw_oracle.c`` (plain int64 loops over Eqs. sw2-sw4 of the paper's
Section 2); this module only compiles it with gcc and marshals numpy arrays through ctypes.

Parity status: pinned.  ``tests/test_oracle_pins.py`` checks the oracle against brute-force
enumeration of every local alignment on tiny inputs, hand-worked examples, closed forms
(self-score, ungapped Kadane limit, linear-gap recurrence, single residue, empty input) and
invariants (transposition symmetry, monotonicity in the gap costs, bounds, concatenation).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sw_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_sw.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i8p = ctypes.POINTER(ctypes.c_int8)


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the shared-library path."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src],
                   check=True)
    os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """Load (building first if needed) and return the ctypes library."""
    global _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        lib = ctypes.CDLL(path or build())
        lib.oracle_sw_score.restype = ctypes.c_int64
        lib.oracle_sw_score.argtypes = [_u8p, ctypes.c_int64, _u8p, ctypes.c_int64, _i8p,
                                        ctypes.c_int32, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_sw_search.restype = ctypes.c_int32
        lib.oracle_sw_search.argtypes = [_u8p, ctypes.c_int64, _u8p, _i64p, ctypes.c_int64,
                                         _i8p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                         _i64p, ctypes.c_int32]
        lib.oracle_sw_pairs.restype = ctypes.c_int32
        lib.oracle_sw_pairs.argtypes = [_u8p, _i64p, _u8p, _i64p, _i64p, _i64p, ctypes.c_int64,
                                        _i8p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                        _i64p, ctypes.c_int32]
        if path is None:
            _lib = lib
        return lib


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(_u8p)


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_i64p)


def _mat(matrix):
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    assert m.ndim == 2 and m.shape[0] == m.shape[1], "matrix must be square (A x A)"
    return m, m.ctypes.data_as(_i8p), int(m.shape[0])


def sw_score(query, subject, matrix, goe: int, ge: int, lib=None) -> int:
    """Best local score of ``query`` vs ``subject``; a gap of length k costs goe + (k-1)*ge."""
    lib = lib or load()
    q, qp = _u8(query)
    d, dp = _u8(subject)
    mm, mp, a = _mat(matrix)
    r = lib.oracle_sw_score(qp, q.shape[0], dp, d.shape[0], mp, a, int(goe), int(ge))
    if r < 0:
        raise MemoryError("oracle scratch allocation failed")
    return int(r)


def sw_search(query, residues, offsets, matrix, goe: int, ge: int, threads: int = 0,
              lib=None):
    """Scores of ``query`` against every database sequence (int64, original order).

    Returns ``(scores, threads_used)``.
    """
    lib = lib or load()
    q, qp = _u8(query)
    r, rp = _u8(residues)
    o, op = _i64(offsets)
    mm, mp, a = _mat(matrix)
    n = o.shape[0] - 1
    out = np.zeros(n, dtype=np.int64)
    used = lib.oracle_sw_search(qp, q.shape[0], rp, op, n, mp, a, int(goe), int(ge),
                                out.ctypes.data_as(_i64p), int(threads))
    if n and out.min() < 0:
        raise MemoryError("oracle scratch allocation failed")
    return out, int(used)


def sw_pairs(queries, residues, offsets, qsel, dsel, matrix, goe: int, ge: int,
             threads: int = 0, lib=None):
    """Scores for the pairs (queries[qsel[p]], database sequence dsel[p]).  Returns int64."""
    lib = lib or load()
    qlens = np.array([len(x) for x in queries], dtype=np.int64)
    qoff = np.zeros(len(queries) + 1, dtype=np.int64)
    np.cumsum(qlens, out=qoff[1:])
    qres = np.concatenate([np.asarray(x, dtype=np.uint8) for x in queries]) if len(queries) \
        else np.zeros(1, dtype=np.uint8)
    qr, qrp = _u8(qres if qres.size else np.zeros(1, dtype=np.uint8))
    qo, qop = _i64(qoff)
    r, rp = _u8(residues if len(residues) else np.zeros(1, dtype=np.uint8))
    o, op = _i64(offsets)
    qs, qsp = _i64(qsel)
    ds, dsp = _i64(dsel)
    mm, mp, a = _mat(matrix)
    out = np.zeros(qs.shape[0], dtype=np.int64)
    lib.oracle_sw_pairs(qrp, qop, rp, op, qsp, dsp, qs.shape[0], mp, a, int(goe), int(ge),
                        out.ctypes.data_as(_i64p), int(threads))
    if out.size and out.min() < 0:
        raise MemoryError("oracle scratch allocation failed")
    return out
