"""ORACLE — test infrastructure, not part of the library.

Python front end of the plain C skip-BF oracle (``motif_oracle.c``, Perera & Ragel Sec. III.A
with the index-range split of Sec. IV.A).  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.  It imports nothing from the library
package and the library never imports it.

``search`` returns the ascending candidate indices (2l-bit codes, base i of the l-mer in bits
[2(l-1-i), 2(l-1-i)+1], A=0 C=1 G=2 T=3) of every l-mer that has a window within Hamming
distance d in every sequence, together with the canonical algorithmic window-compare tally.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "motif_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the C oracle with gcc into oracle/_build/liboracle.so and returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i64p = ctypes.POINTER(ctypes.c_longlong)
            lib.oracle_skipbf_range.argtypes = [ctypes.c_int] * 4 + [
                ctypes.c_char_p, ctypes.c_longlong, ctypes.c_uint64, ctypes.c_uint64, u64p,
                ctypes.c_longlong, i64p, u64p]
            lib.oracle_skipbf_threads.argtypes = [ctypes.c_int] * 4 + [
                ctypes.c_char_p, ctypes.c_longlong, ctypes.c_uint64, ctypes.c_uint64,
                ctypes.c_int, u64p, ctypes.c_longlong, i64p, u64p]
            lib.oracle_skipbf_var.argtypes = [
                ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                ctypes.c_char_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_uint64,
                ctypes.c_uint64, u64p, ctypes.c_longlong, i64p, u64p]
            lib.oracle_lmer_from_index.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_char_p]
            lib.oracle_lmer_from_index.restype = None
            _lib = lib
    return _lib


def _as_rows(seqs) -> tuple[bytes, int, int]:
    """Returns (buffer, n, t) for a list of equal-length strings/bytes or an (n, t) uint8 array."""
    if isinstance(seqs, np.ndarray):
        a = np.ascontiguousarray(seqs, dtype=np.uint8)
        if a.ndim != 2:
            raise ValueError("expected an (n, t) array of characters")
        return a.tobytes(), a.shape[0], a.shape[1]
    rows = [s.encode() if isinstance(s, str) else bytes(s) for s in seqs]
    if not rows or len({len(r) for r in rows}) != 1:
        raise ValueError("expected n >= 1 sequences of one common length")
    return b"".join(rows), len(rows), len(rows[0])


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__("oracle error %d" % code)
        self.code = code


def search(seqs, l: int, d: int, lo: int = 0, hi: int | None = None, threads: int = 1):
    """Skip-BF over candidate indices [lo, hi) (default: all 4^l).

    Returns (codes: np.ndarray[uint64] ascending, compares: int)."""
    lib = _load()
    buf, n, t = _as_rows(seqs)
    if hi is None:
        hi = 4 ** l
    count = ctypes.c_longlong(0)
    cmp = ctypes.c_uint64(0)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    # One pass with room for 65536 codes; a larger result is searched again with exact room.
    cap = 1 << 16
    while True:
        out = np.zeros(cap, dtype=np.uint64)
        ptr = out.ctypes.data_as(u64p)
        if threads == 1:
            rc = lib.oracle_skipbf_range(n, t, l, d, buf, t, lo, hi, ptr, cap,
                                         ctypes.byref(count), ctypes.byref(cmp))
        else:
            rc = lib.oracle_skipbf_threads(n, t, l, d, buf, t, lo, hi, threads, ptr, cap,
                                           ctypes.byref(count), ctypes.byref(cmp))
        if rc != 0:
            raise OracleError(rc)
        if count.value <= cap:
            return out[:count.value].copy(), int(cmp.value)
        cap = count.value


def search_var(seqs, l: int, d: int, mask_unknown: bool = True, lo: int = 0,
               hi: int | None = None):
    """Skip-BF for sequences of different lengths (strings or bytes); with mask_unknown a window
    containing a character outside ACGTacgt never matches.  Returns (codes, compares)."""
    lib = _load()
    rows = [s.encode() if isinstance(s, str) else bytes(s) for s in seqs]
    if not rows:
        raise ValueError("expected n >= 1 sequences")
    stride = max(1, max(len(r) for r in rows))
    buf = b"".join(r.ljust(stride, b"\0") for r in rows)
    lens = (ctypes.c_int * len(rows))(*[len(r) for r in rows])
    if hi is None:
        hi = 4 ** l
    count = ctypes.c_longlong(0)
    cmp = ctypes.c_uint64(0)
    cap = 1 << 16
    while True:
        out = np.zeros(cap, dtype=np.uint64)
        rc = lib.oracle_skipbf_var(len(rows), lens, l, d, buf, stride, 1 if mask_unknown else 0,
                                   lo, hi, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                   cap, ctypes.byref(count), ctypes.byref(cmp))
        if rc != 0:
            raise OracleError(rc)
        if count.value <= cap:
            return out[:count.value].copy(), int(cmp.value)
        cap = count.value


def lmer(code: int, l: int) -> str:
    """The l-mer string of a candidate index, as the oracle generates it."""
    lib = _load()
    buf = ctypes.create_string_buffer(l + 1)
    lib.oracle_lmer_from_index(code, l, buf)
    return buf.raw[:l].decode()
