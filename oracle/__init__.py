"""Shouji CPU oracle -- test infrastructure only.

A ctypes wrapper around ``shouji_oracle.c``: a plain, single-pair-at-a-time C
restatement of the Shouji filter (arXiv 1809.07858, Sec. 2.2 and Algorithms
1-2), of MAGNET (Supplementary Sec. 7, Algorithms 3-4), plus the global edit distance used as ground truth for false-accept /
false-reject counts (Sec. 3.2).  Only the tests, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg may import this package.  It shares no
code with the CUDA library and never imports it.

Parity status of each function (what pins it is in ``tests/test_oracle_pins.py``):
  neighborhood_map  pinned (Eq. 1 cells vs. a brute-force character compare,
                    orientation vs. the printed diagonals of Fig. 6)
  shouji            pinned (Fig. 1 caption, Fig. 6(b) printed count, E = 0
                    Hamming reduction, identical pairs, shifted-copy closed
                    forms, tiny brute force); the one Fig. 6(a) vector is
                    "parity unpinned" (the printed vector is garbled)
  count_mode        pinned (hand cases of the local / glocal rules); the Fig. 6(c)
                    local count is "parity unpinned" (3 here, 2 printed)
  magnet            pinned (Fig. 6(a),(b) printed counts, hand-traced cases per
                    reading, E = 0 identity test, shift / substitution closed
                    forms; tests/test_magnet_oracle.py); the Fig. 6(c) local
                    count is "parity unpinned" (5 here, 4 printed)
  edit_distance     pinned (textbook identities and brute force on tiny inputs)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shouji_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_shouji.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no vector intrinsics)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
             "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.oracle_shouji.argtypes = [ctypes.c_char_p, ctypes.c_char_p,
                                      ctypes.c_int, ctypes.c_int, u8p]
        lib.oracle_shouji.restype = ctypes.c_int
        lib.oracle_neighborhood_map.argtypes = [ctypes.c_char_p, ctypes.c_char_p,
                                                ctypes.c_int, ctypes.c_int, u8p]
        lib.oracle_neighborhood_map.restype = None
        lib.oracle_edit_distance.argtypes = [ctypes.c_char_p, ctypes.c_int,
                                             ctypes.c_char_p, ctypes.c_int]
        lib.oracle_edit_distance.restype = ctypes.c_int
        lib.oracle_shouji_batch.argtypes = [ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_size_t, ctypes.c_int,
                                            ctypes.c_size_t, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int]
        lib.oracle_shouji_batch.restype = ctypes.c_int
        lib.oracle_magnet_batch.argtypes = lib.oracle_shouji_batch.argtypes
        lib.oracle_magnet_batch.restype = ctypes.c_int
        lib.oracle_count_mode.argtypes = [u8p, ctypes.c_int, ctypes.c_int]
        lib.oracle_count_mode.restype = ctypes.c_int
        lib.oracle_shouji_mode.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_char_p,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, u8p]
        lib.oracle_shouji_mode.restype = ctypes.c_int
        lib.oracle_magnet_mode.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_char_p,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, u8p]
        lib.oracle_magnet_mode.restype = ctypes.c_int
        _lib = lib
    return _lib


def _as_bytes(s) -> bytes:
    if isinstance(s, str):
        return s.encode("ascii")
    if isinstance(s, np.ndarray):
        return s.astype(np.uint8, copy=False).tobytes()
    return bytes(s)


def neighborhood_map(P, T, E: int) -> np.ndarray:
    """(2E+1, m) uint8 array; row d+E is diagonal d (Eq. 1, readings R1/R3/R8)."""
    P, T = _as_bytes(P), _as_bytes(T)
    m = len(P)
    assert len(T) == m
    out = np.zeros((2 * E + 1, m), dtype=np.uint8)
    _load().oracle_neighborhood_map(
        P, T, m, E, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return out


def shouji(P, T, E: int):
    """Return (bit-vector as uint8 array of 0/1, ones, accept) for one pair."""
    P, T = _as_bytes(P), _as_bytes(T)
    m = len(P)
    assert len(T) == m and m > 0
    S = np.zeros(m, dtype=np.uint8)
    ones = _load().oracle_shouji(P, T, m, E,
                                 S.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    if ones < 0:
        raise MemoryError("oracle_shouji failed")
    return S, ones, ones <= E


GLOBAL, LOCAL, GLOCAL_START, GLOCAL_END = 0, 1, 2, 3


def count_mode(S, mode: int) -> int:
    """Ones of a Shouji bit-vector under a count mode (Sec. 2.2.3, Supp. Sec. 8):
    0 all, 1 not the runs at both ends, 2 not the leading run, 3 not the
    trailing run; a vector with no zero counts its length (reading R10)."""
    S = np.ascontiguousarray(S, dtype=np.uint8)
    return _load().oracle_count_mode(S.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), len(S),
                                     mode)


def shouji_mode(P, T, E: int, mode: int):
    """The filter for a pattern P no longer than the text T (P past its end
    reads as out of the band) with a count mode.  Returns (vector, count)."""
    P, T = _as_bytes(P), _as_bytes(T)
    m = len(T)
    assert len(P) <= m and m > 0
    S = np.zeros(m, dtype=np.uint8)
    c = _load().oracle_shouji_mode(P, len(P), T, m, E, mode,
                                   S.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    if c < 0:
        raise ValueError("oracle_shouji_mode: bad argument")
    return S, c


def magnet(P, T, E: int, mode: int = 0):
    """MAGNET (Supp. Sec. 7, Algorithms 3-4) for a pattern P no longer than the
    text T, with a count mode.  Returns (MAGNET vector, count)."""
    P, T = _as_bytes(P), _as_bytes(T)
    m = len(T)
    assert len(P) <= m and m > 0
    V = np.zeros(m, dtype=np.uint8)
    c = _load().oracle_magnet_mode(P, len(P), T, m, E, mode,
                                   V.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    if c < 0:
        raise ValueError("oracle_magnet_mode: bad argument")
    return V, c


def edit_distance(a, b) -> int:
    """Global (end-to-end) Levenshtein distance by the full DP table."""
    a, b = _as_bytes(a), _as_bytes(b)
    d = _load().oracle_edit_distance(a, len(a), b, len(b))
    if d < 0:
        raise MemoryError("oracle_edit_distance failed")
    return d


def shouji_batch(reads: np.ndarray, refs: np.ndarray, E: int,
                 E_per_pair: np.ndarray | None = None, threads: int = 1, magnet: bool = False):
    """Filter n pairs given as (n, m) uint8 arrays (row i = pair i) with Shouji,
    or with MAGNET (global count) when ``magnet``.

    Returns (accept bool[n], count uint8[n]).  ``threads`` splits the pairs
    into contiguous ranges, one POSIX thread each.
    """
    reads = np.ascontiguousarray(reads, dtype=np.uint8)
    refs = np.ascontiguousarray(refs, dtype=np.uint8)
    assert reads.shape == refs.shape and reads.ndim == 2
    n, m = reads.shape
    accept = np.zeros(n, dtype=np.uint8)
    count = np.zeros(n, dtype=np.uint8)
    ep = None
    if E_per_pair is not None:
        E_per_pair = np.ascontiguousarray(E_per_pair, dtype=np.uint8)
        assert E_per_pair.shape == (n,)
        ep = E_per_pair.ctypes.data
    fn = _load().oracle_magnet_batch if magnet else _load().oracle_shouji_batch
    rc = fn(reads.ctypes.data, refs.ctypes.data, m, m, n, E, ep, accept.ctypes.data,
            count.ctypes.data, int(threads))
    if rc != 0:
        raise MemoryError("oracle_shouji_batch failed")
    return accept.astype(bool), count
