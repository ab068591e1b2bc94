"""Seeded synthetic read/reference pairs shaped like the Shouji paper's workloads.

Thin ctypes wrapper over ``csrc/synth.c`` (SplitMix64, counter-style: pair i
always gets the same bytes, whatever sub-range or thread count generates it).
It holds none of the filter's arithmetic; the CUDA path's tests and benchmark
and the CPU oracle's tests all take their inputs from here.

The paper's datasets (Sec. 3.1: 30M mrFAST candidate pairs per set, read
lengths 100/150/250, thresholds 0-10% of the length) are not available; the
``workload`` helpers below reproduce their shapes:

* ``small``  -- 10,000 pairs, m=100, k ~ U{0..10}, seed 0;
* ``sweep``  -- m=100, threshold E: half near (k ~ U{0..E}), half far
  (k ~ U{E+1..25}), seed 1000+E;
* ``long``   -- m in {150, 250}, threshold E: near k ~ U{0..E}, far
  k ~ U{E+1..ceil(m/4)}, 0.1% 'N' bases on each side, seed 2000+m+E.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "synth.c")
_LIB_PATH = os.path.join(_HERE, "libshouji_synth.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
        lib.synth_pairs.argtypes = [u64, u64, u64, u32, u64, u32, u32, u32, u32,
                                    ctypes.c_double, ctypes.c_double, vp, vp, vp,
                                    vp, vp, ctypes.c_int]
        lib.synth_pairs.restype = ctypes.c_int
        lib.synth_mixed_shape.argtypes = [u64, u64, u64, vp, vp, ctypes.c_int,
                                          u32, u32, vp, vp]
        lib.synth_mixed_shape.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return int(a.data_ptr())  # a CPU torch tensor (e.g. pinned memory)


def default_threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def pairs(n: int, m: int, *, seed: int, near=(0, 10), far=None,
          far_fraction: float = 0.0, n_rate: float = 0.0, first: int = 0,
          lengths=None, out=None, stride: int | None = None,
          with_meta: bool = False, threads: int | None = None):
    """Generate pairs ``first .. first+n-1``.

    Returns ``(reads, refs)`` as (n, stride) uint8 arrays (or the ``out``
    buffers, numpy arrays or CPU torch tensors of n*stride bytes), plus
    ``(kind, k)`` arrays when ``with_meta``.
    """
    stride = m if stride is None else stride
    if out is None:
        reads = np.zeros((n, stride), dtype=np.uint8)
        refs = np.zeros((n, stride), dtype=np.uint8)
    else:
        reads, refs = out
    far = far if far is not None else (0, 0)
    kind = np.zeros(n, dtype=np.uint8) if with_meta else None
    kk = np.zeros(n, dtype=np.uint8) if with_meta else None
    if lengths is not None:
        lengths = np.ascontiguousarray(lengths, dtype=np.uint16)
        assert lengths.shape == (n,) and int(lengths.max(initial=0)) <= m
    rc = _load().synth_pairs(seed, first, n, m, stride, near[0], near[1],
                             far[0], far[1], float(far_fraction), float(n_rate),
                             _ptr(lengths), _ptr(reads), _ptr(refs), _ptr(kind),
                             _ptr(kk), threads or default_threads())
    if rc != 0:
        raise ValueError("synth_pairs: bad arguments or allocation failure")
    if with_meta:
        return reads, refs, kind, kk
    return reads, refs


def workload(name: str, n: int | None = None, *, E: int = 5, m: int = 100,
             first: int = 0, **kw):
    """The named workload recipes of the module docstring."""
    if name == "small":
        return pairs(10_000 if n is None else n, 100, seed=0, near=(0, 10),
                     first=first, **kw)
    if name == "sweep":
        return pairs(30_000_000 if n is None else n, 100, seed=1000 + E,
                     near=(0, E), far=(E + 1, 25), far_fraction=0.5,
                     first=first, **kw)
    if name == "long":
        assert m in (150, 250)
        return pairs(10_000_000 if n is None else n, m, seed=2000 + m + E,
                     near=(0, E), far=(E + 1, math.ceil(m / 4)),
                     far_fraction=0.5, n_rate=0.001, first=first, **kw)
    raise ValueError(name)


def mixed_shape(n: int, *, seed: int, choices=(100, 150, 250),
                weights=(0.4, 0.4, 0.2), e_range=(2, 12), first: int = 0):
    """Per-pair (length, E) for a mixed batch: length drawn from ``choices``
    with ``weights``, E uniform in ``e_range``."""
    ch = np.ascontiguousarray(choices, dtype=np.uint16)
    cum = np.ascontiguousarray(np.cumsum(weights) / np.sum(weights), dtype=np.float64)
    cum[-1] = 1.0
    lengths = np.zeros(n, dtype=np.uint16)
    Es = np.zeros(n, dtype=np.uint8)
    rc = _load().synth_mixed_shape(seed, first, n, ch.ctypes.data, cum.ctypes.data,
                                   len(ch), e_range[0], e_range[1],
                                   lengths.ctypes.data, Es.ctypes.data)
    if rc != 0:
        raise ValueError("synth_mixed_shape: bad arguments")
    return lengths, Es
