"""ctypes binding of libshouji.so: argument marshalling only.

Every function here forwards to the C ABI declared in ``include/shouji.h``
with the same name; torch tensors supply device memory and the current CUDA
stream.  No step of the filter runs in Python.  The library is loaded on
first use and a missing or unloadable library raises ``ShoujiError`` (there
is no fallback).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libshouji.so")

SHOUJI_TILE = 1024
SHOUJI_MAX_M = 255
SHOUJI_MAX_E = 31
SHOUJI_NOALLOC_MAX_PAIRS = 1 << 29

__all__ = [
    "ShoujiError", "SHOUJI_TILE", "SHOUJI_MAX_M", "SHOUJI_MAX_E", "LIB_PATH",
    "load_library", "shouji_status_string", "shouji_last_cuda_error", "shouji_wait_failures",
    "shouji_selftest_pack_wait", "shouji_alu_probe", "PROBE_OPS", "shouji_unmasked_n",
    "shouji_packed_words", "shouji_nmask_words", "shouji_pack", "shouji_filter",
    "shouji_pack_filter", "shouji_pack_filter_fused", "shouji_pack_filter_results",
    "shouji_pack_filter_workspace_size",
    "shouji_compact_workspace_size", "shouji_compact", "filter_pairs",
    "accept_to_bool", "Pipeline", "shouji_compact_noalloc", "SHOUJI_NOALLOC_MAX_PAIRS",
    "Batch", "Server", "shouji_count", "COUNT_GLOBAL", "COUNT_LOCAL", "COUNT_GLOCAL_START",
    "COUNT_GLOCAL_END", "shouji_magnet", "magnet_pairs", "SERVE_DEVICE_RESULTS",
]

COUNT_GLOBAL, COUNT_LOCAL, COUNT_GLOCAL_START, COUNT_GLOCAL_END = 0, 1, 2, 3

_lib = None


class ShoujiError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = "%s: %s" % (where, shouji_status_string(status) if _lib else status)
        if status == 3 and _lib is not None:
            msg += " (cudaError %d)" % _lib.shouji_last_cuda_error()
        super().__init__(msg)


def load_library(path: str = LIB_PATH):
    """Load libshouji.so (built in-tree by ``paper_1809_07858_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ShoujiError(-1, "libshouji.so not built at %s (run __graft_entry__.build())" % path)
    lib = ctypes.CDLL(path)
    vp, sz, u32, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint64
    lib.shouji_status_string.argtypes = [ctypes.c_int]
    lib.shouji_status_string.restype = ctypes.c_char_p
    lib.shouji_last_cuda_error.argtypes = []
    lib.shouji_last_cuda_error.restype = ctypes.c_int
    lib.shouji_wait_failures.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
    lib.shouji_wait_failures.restype = ctypes.c_int
    lib.shouji_selftest_pack_wait.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
    lib.shouji_selftest_pack_wait.restype = ctypes.c_int
    lib.shouji_unmasked_n.argtypes = [ctypes.POINTER(ctypes.c_int)]
    lib.shouji_unmasked_n.restype = ctypes.c_int
    lib.shouji_alu_probe.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.shouji_alu_probe.restype = ctypes.c_int
    lib.shouji_packed_words.argtypes = [sz, u32]
    lib.shouji_packed_words.restype = sz
    lib.shouji_nmask_words.argtypes = [sz, u32]
    lib.shouji_nmask_words.restype = sz
    lib.shouji_pack.argtypes = [vp, u64, sz, u32, vp, vp, vp]
    lib.shouji_pack.restype = ctypes.c_int
    lib.shouji_filter.argtypes = [vp, vp, vp, vp, u32, sz, ctypes.c_int, vp, vp, vp, vp, vp]
    lib.shouji_filter.restype = ctypes.c_int
    lib.shouji_magnet.argtypes = [vp, vp, vp, vp, u32, sz, ctypes.c_int, vp, vp, vp, vp, vp]
    lib.shouji_magnet.restype = ctypes.c_int
    lib.shouji_pack_filter.argtypes = [vp, vp, u64, sz, u32, ctypes.c_int, vp, vp, vp, vp, vp]
    lib.shouji_pack_filter.restype = ctypes.c_int
    lib.shouji_pack_filter_fused.argtypes = [vp, vp, u64, u32, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int)]
    lib.shouji_pack_filter_fused.restype = ctypes.c_int
    lib.shouji_pack_filter_workspace_size.argtypes = [vp, vp, u64, sz, u32, ctypes.c_int,
                                                      ctypes.POINTER(sz)]
    lib.shouji_pack_filter_workspace_size.restype = ctypes.c_int
    lib.shouji_pack_filter_results.argtypes = [vp, vp, u64, sz, u32, ctypes.c_int, vp, sz, vp,
                                               vp, vp]
    lib.shouji_pack_filter_results.restype = ctypes.c_int
    lib.shouji_compact_workspace_size.argtypes = [sz]
    lib.shouji_compact_workspace_size.restype = sz
    lib.shouji_compact.argtypes = [vp, sz, vp, vp, vp, sz, vp]
    lib.shouji_compact.restype = ctypes.c_int
    lib.shouji_compact_noalloc.argtypes = [vp, sz, vp, vp, vp]
    lib.shouji_compact_noalloc.restype = ctypes.c_int
    lib.shouji_batch_create.argtypes = [sz, u32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_char_p, ctypes.POINTER(vp)]
    lib.shouji_batch_create.restype = ctypes.c_int
    lib.shouji_batch_run.argtypes = [vp, vp, vp, u64, vp, vp, sz, vp, vp, vp]
    lib.shouji_batch_run.restype = ctypes.c_int
    lib.shouji_batch_invalid.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.shouji_batch_invalid.restype = ctypes.c_int
    ip = ctypes.POINTER(ctypes.c_int)
    lib.shouji_batch_shape.argtypes = [vp, ctypes.c_int, ip, ip, ip, ip]
    lib.shouji_batch_shape.restype = ctypes.c_int
    lib.shouji_batch_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    lib.shouji_batch_timing.restype = ctypes.c_int
    lib.shouji_batch_tune.argtypes = [vp, vp, vp, u64, vp, vp, sz, vp, vp, ctypes.c_char_p, vp]
    lib.shouji_batch_tune.restype = ctypes.c_int
    lib.shouji_batch_destroy.argtypes = [vp]
    lib.shouji_batch_destroy.restype = None
    lib.shouji_server_create.argtypes = [sz, u32, u64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         sz, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(vp)]
    lib.shouji_server_create.restype = ctypes.c_int
    lib.shouji_server_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_uint64)]
    lib.shouji_server_info.restype = ctypes.c_int
    lib.shouji_server_submit.argtypes = [vp, vp, vp, u64, vp, vp, sz, vp, vp,
                                         ctypes.POINTER(ctypes.c_uint64)]
    lib.shouji_server_submit.restype = ctypes.c_int
    lib.shouji_server_wait.argtypes = [vp, u64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.shouji_server_wait.restype = ctypes.c_int
    lib.shouji_server_wait_timed.argtypes = [vp, u64, ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_double)]
    lib.shouji_server_wait_timed.restype = ctypes.c_int
    lib.shouji_server_submit_request.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.shouji_server_submit_request.restype = ctypes.c_int
    lib.shouji_server_add_reference.argtypes = [vp, vp, u64, ctypes.POINTER(ctypes.c_uint32)]
    lib.shouji_server_add_reference.restype = ctypes.c_int
    lib.shouji_server_stats_read.argtypes = [vp, vp]
    lib.shouji_server_stats_read.restype = ctypes.c_int
    lib.shouji_batch_run_at.argtypes = [vp, vp, u64, vp, vp, vp, vp, sz, vp, vp, vp]
    lib.shouji_batch_run_at.restype = ctypes.c_int
    lib.shouji_batch_device_bytes.argtypes = [sz, u32, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.shouji_batch_device_bytes.restype = sz
    lib.shouji_server_destroy.argtypes = [vp]
    lib.shouji_server_destroy.restype = None
    lib.shouji_count.argtypes = [vp, u32, sz, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp]
    lib.shouji_count.restype = ctypes.c_int
    lib.shouji_pipeline_create.argtypes = [u32, sz, sz, ctypes.c_int, ctypes.POINTER(vp)]
    lib.shouji_pipeline_create.restype = ctypes.c_int
    lib.shouji_pipeline_run.argtypes = [vp, vp, vp, u64, sz, ctypes.c_int, vp, vp, vp,
                                        ctypes.POINTER(ctypes.c_uint64)]
    lib.shouji_pipeline_run.restype = ctypes.c_int
    lib.shouji_pipeline_run_packed.argtypes = [vp, vp, vp, vp, vp, sz, ctypes.c_int, vp, vp, vp,
                                               ctypes.POINTER(ctypes.c_uint64)]
    lib.shouji_pipeline_run_packed.restype = ctypes.c_int
    lib.shouji_pipeline_destroy.argtypes = [vp]
    lib.shouji_pipeline_destroy.restype = None
    _lib = lib
    return lib


def shouji_status_string(status: int) -> str:
    return load_library().shouji_status_string(int(status)).decode()


def shouji_last_cuda_error() -> int:
    return load_library().shouji_last_cuda_error()


def shouji_wait_failures() -> int:
    """Synchronize the device; return and reset the number of bounded pack
    staging waits that ran out (0 in normal operation)."""
    c = ctypes.c_uint32(0)
    _check(load_library().shouji_wait_failures(ctypes.byref(c)), "shouji_wait_failures")
    return c.value


def shouji_selftest_pack_wait() -> int:
    """Run the pack with every staging wait made to run out (about a second);
    return the failures counted (4)."""
    c = ctypes.c_uint32(0)
    _check(load_library().shouji_selftest_pack_wait(ctypes.byref(c)), "shouji_selftest_pack_wait")
    return c.value


def shouji_unmasked_n() -> bool:
    """Synchronize the device; whether a pack without an N mask has read an
    'N' (as 'G') since the last call, and reset that flag."""
    v = ctypes.c_int(0)
    st = load_library().shouji_unmasked_n(ctypes.byref(v))
    if st not in (0, 1) or (st == 1 and not v.value):
        _check(st, "shouji_unmasked_n")
    return bool(v.value)


PROBE_OPS = {"lop3": 0, "shf": 1, "prmt": 2, "iadd3": 3, "imad": 4, "popc": 5, "lop3+imad": 6}


def shouji_alu_probe(op: str = "lop3") -> float:
    """Measured lane-operations per SM clock of one integer instruction kind
    (see ``PROBE_OPS``) on the current device; synchronizes the device."""
    r = ctypes.c_double(0.0)
    _check(load_library().shouji_alu_probe(PROBE_OPS[op], ctypes.byref(r)), "shouji_alu_probe")
    return r.value


def shouji_packed_words(n: int, m: int) -> int:
    return load_library().shouji_packed_words(n, m)


def shouji_nmask_words(n: int, m: int) -> int:
    return load_library().shouji_nmask_words(n, m)


def _torch():
    import torch
    return torch


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(status: int, where: str):
    if status != 0:
        raise ShoujiError(status, where)


def shouji_pack(seqs, m: int, *, n: int | None = None, stride: int | None = None,
                with_n: bool = False, packed=None, nmask=None, stream=None):
    """ASCII sequences -> packed bit-sliced planes (and N mask).

    ``seqs``: CUDA uint8 tensor, (n, stride) or flat with ``n`` and ``stride``.
    Returns ``(packed, nmask)`` (``nmask`` is None unless ``with_n``).
    """
    torch = _torch()
    lib = load_library()
    if seqs.dim() == 2:
        n = seqs.shape[0] if n is None else n
        stride = seqs.shape[1] if stride is None else stride
    assert n is not None and stride is not None
    dev = seqs.device
    if packed is None:
        packed = torch.empty(max(1, lib.shouji_packed_words(n, m)), dtype=torch.int32, device=dev)
    if with_n and nmask is None:
        nmask = torch.empty(max(1, lib.shouji_nmask_words(n, m)), dtype=torch.int32, device=dev)
    _check(lib.shouji_pack(_ptr(seqs), stride, n, m, _ptr(packed),
                           _ptr(nmask) if with_n else None, _stream(stream)), "shouji_pack")
    return packed, (nmask if with_n else None)


def shouji_filter(reads, refs, m: int, n_pairs: int, E: int, *, reads_nmask=None,
                  refs_nmask=None, E_per_pair=None, out_accept=None, out_count=None,
                  count: bool = True, out_vectors=None, vectors: bool = False,
                  stream=None):
    """Filter packed pairs.  Returns ``(accept_words, count, vectors)``.

    ``accept_words``: int32 tensor of ceil(n_pairs/32) words (bit i%32 of word
    i//32 = pair i accepted); ``count``: uint8[n_pairs] or None; ``vectors``:
    bit-sliced Shouji bit-vectors or None.
    """
    torch = _torch()
    lib = load_library()
    dev = reads.device
    if out_accept is None:
        out_accept = torch.empty(max(1, (n_pairs + 31) // 32), dtype=torch.int32, device=dev)
    if out_count is None and count:
        out_count = torch.empty(max(1, n_pairs), dtype=torch.uint8, device=dev)
    if out_vectors is None and vectors:
        out_vectors = torch.empty(max(1, lib.shouji_nmask_words(n_pairs, m)), dtype=torch.int32,
                                  device=dev)
    _check(lib.shouji_filter(_ptr(reads), _ptr(refs), _ptr(reads_nmask), _ptr(refs_nmask),
                             m, n_pairs, E, _ptr(E_per_pair), _ptr(out_accept),
                             _ptr(out_count), _ptr(out_vectors), _stream(stream)),
           "shouji_filter")
    return out_accept, out_count, out_vectors


def shouji_pack_filter(reads, refs, m: int, E: int, *, n: int | None = None,
                       stride: int | None = None, packed_reads=None, packed_refs=None,
                       out_accept=None, out_count=None, count: bool = True, stream=None):
    """Pack both ASCII sets and filter them (one fused kernel where it
    applies).  ``reads``/``refs``: CUDA uint8, (n, stride) or flat with ``n``
    and ``stride``.  Returns ``(packed_reads, packed_refs, accept_words,
    count)``."""
    torch = _torch()
    lib = load_library()
    if reads.dim() == 2:
        n = reads.shape[0] if n is None else n
        stride = reads.shape[1] if stride is None else stride
    assert n is not None and stride is not None
    dev = reads.device
    words = max(1, lib.shouji_packed_words(n, m))
    if packed_reads is None:
        packed_reads = torch.empty(words, dtype=torch.int32, device=dev)
    if packed_refs is None:
        packed_refs = torch.empty(words, dtype=torch.int32, device=dev)
    if out_accept is None:
        out_accept = torch.empty(max(1, (n + 31) // 32), dtype=torch.int32, device=dev)
    if out_count is None and count:
        out_count = torch.empty(max(1, n), dtype=torch.uint8, device=dev)
    _check(lib.shouji_pack_filter(_ptr(reads), _ptr(refs), stride, n, m, E, _ptr(packed_reads),
                                  _ptr(packed_refs), _ptr(out_accept), _ptr(out_count),
                                  _stream(stream)),
           "shouji_pack_filter")
    return packed_reads, packed_refs, out_accept, out_count


def shouji_pack_filter_workspace_size(reads, refs, m: int, E: int, n: int, *,
                                      stride: int | None = None) -> int:
    """Bytes of the workspace ``shouji_pack_filter_results`` needs."""
    stride = (reads.shape[1] if reads.dim() == 2 else m) if stride is None else stride
    b = ctypes.c_size_t(0)
    _check(load_library().shouji_pack_filter_workspace_size(_ptr(reads), _ptr(refs), stride, n, m,
                                                            E, ctypes.byref(b)),
           "shouji_pack_filter_workspace_size")
    return b.value


def shouji_pack_filter_results(reads, refs, m: int, E: int, *, n: int | None = None,
                               stride: int | None = None, workspace=None, out_accept=None,
                               out_count=None, count: bool = True, stream=None):
    """``shouji_pack_filter`` without the packed outputs (the packed tiles go
    through per-CTA rings in ``workspace``, a CUDA uint8 tensor of at least
    ``shouji_pack_filter_workspace_size`` bytes).  Returns ``(accept_words,
    count)``."""
    torch = _torch()
    if reads.dim() == 2:
        n = reads.shape[0] if n is None else n
        stride = reads.shape[1] if stride is None else stride
    assert n is not None and stride is not None
    dev = reads.device
    if workspace is None:
        need = shouji_pack_filter_workspace_size(reads, refs, m, E, n, stride=stride)
        workspace = torch.empty(max(16, need), dtype=torch.uint8, device=dev)
    if out_accept is None:
        out_accept = torch.empty(max(1, (n + 31) // 32), dtype=torch.int32, device=dev)
    if out_count is None and count:
        out_count = torch.empty(max(1, n), dtype=torch.uint8, device=dev)
    _check(load_library().shouji_pack_filter_results(
        _ptr(reads), _ptr(refs), stride, n, m, E, _ptr(workspace),
        workspace.numel() * workspace.element_size(), _ptr(out_accept), _ptr(out_count),
        _stream(stream)), "shouji_pack_filter_results")
    return out_accept, out_count


def shouji_pack_filter_fused(reads, refs, m: int, E: int, *, stride: int | None = None) -> bool:
    """Whether ``shouji_pack_filter`` on these rows runs as the one fused
    kernel (True) or as separate pack and filter launches (False)."""
    stride = (reads.shape[1] if reads.dim() == 2 else m) if stride is None else stride
    f = ctypes.c_int(0)
    _check(load_library().shouji_pack_filter_fused(_ptr(reads), _ptr(refs), stride, m, E,
                                                   ctypes.byref(f)), "shouji_pack_filter_fused")
    return bool(f.value)


def shouji_magnet(reads, refs, m: int, n_pairs: int, E: int, *, reads_nmask=None,
                  refs_nmask=None, E_per_pair=None, out_accept=None, out_count=None,
                  count: bool = True, out_vectors=None, vectors: bool = False,
                  stream=None):
    """MAGNET on packed pairs, same arguments and results as ``shouji_filter``
    (``vectors`` are the MAGNET bit-vectors)."""
    torch = _torch()
    lib = load_library()
    dev = reads.device
    if out_accept is None:
        out_accept = torch.empty(max(1, (n_pairs + 31) // 32), dtype=torch.int32, device=dev)
    if out_count is None and count:
        out_count = torch.empty(max(1, n_pairs), dtype=torch.uint8, device=dev)
    if out_vectors is None and vectors:
        out_vectors = torch.empty(max(1, lib.shouji_nmask_words(n_pairs, m)), dtype=torch.int32,
                                  device=dev)
    _check(lib.shouji_magnet(_ptr(reads), _ptr(refs), _ptr(reads_nmask), _ptr(refs_nmask),
                             m, n_pairs, E, _ptr(E_per_pair), _ptr(out_accept),
                             _ptr(out_count), _ptr(out_vectors), _stream(stream)),
           "shouji_magnet")
    return out_accept, out_count, out_vectors


def shouji_count(vectors, m: int, n_pairs: int, E: int, mode: int, *, E_per_pair=None,
                 out_accept=None, out_count=None, count: bool = True, stream=None):
    """Recount Shouji bit-vectors (from ``shouji_filter(..., vectors=True)``)
    under a count mode.  Returns ``(accept_words, count)``."""
    torch = _torch()
    dev = vectors.device
    if out_accept is None:
        out_accept = torch.empty(max(1, (n_pairs + 31) // 32), dtype=torch.int32, device=dev)
    if out_count is None and count:
        out_count = torch.empty(max(1, n_pairs), dtype=torch.uint8, device=dev)
    _check(load_library().shouji_count(_ptr(vectors), m, n_pairs, E, _ptr(E_per_pair), mode,
                                       _ptr(out_accept), _ptr(out_count), _stream(stream)),
           "shouji_count")
    return out_accept, out_count


def shouji_compact_workspace_size(n_pairs: int) -> int:
    return load_library().shouji_compact_workspace_size(n_pairs)


def shouji_compact(accept, n_pairs: int, *, out_idx=None, out_n=None, workspace=None,
                   stream=None):
    """Indices of accepted pairs in input order.  Returns ``(idx, n_dev)``;
    the first ``int(n_dev)`` entries of ``idx`` are valid."""
    torch = _torch()
    lib = load_library()
    dev = accept.device
    if out_idx is None:
        out_idx = torch.empty(max(1, n_pairs), dtype=torch.int32, device=dev)
    if out_n is None:
        out_n = torch.empty(1, dtype=torch.int32, device=dev)
    ws_bytes = lib.shouji_compact_workspace_size(n_pairs)
    if workspace is None:
        workspace = torch.empty(max(16, ws_bytes), dtype=torch.uint8, device=dev)
    _check(lib.shouji_compact(_ptr(accept), n_pairs, _ptr(out_idx), _ptr(out_n),
                              _ptr(workspace), workspace.numel() * workspace.element_size(),
                              _stream(stream)), "shouji_compact")
    return out_idx, out_n


def shouji_compact_noalloc(accept, n_pairs: int, *, out_idx=None, out_n=None, stream=None):
    """Like ``shouji_compact`` but with the library's own fixed device
    workspace (no allocation by the library).  Returns ``(idx, n_dev)``."""
    torch = _torch()
    lib = load_library()
    dev = accept.device
    if out_idx is None:
        out_idx = torch.empty(max(1, n_pairs), dtype=torch.int32, device=dev)
    if out_n is None:
        out_n = torch.empty(1, dtype=torch.int32, device=dev)
    _check(lib.shouji_compact_noalloc(_ptr(accept), n_pairs, _ptr(out_idx), _ptr(out_n),
                                      _stream(stream)), "shouji_compact_noalloc")
    return out_idx, out_n


def accept_to_bool(accept_words, n_pairs: int):
    """Expand accept words to a bool tensor of n_pairs entries (on the words' device)."""
    torch = _torch()
    w = accept_words[: (n_pairs + 31) // 32].to(torch.int64) & 0xFFFFFFFF
    bits = (w.unsqueeze(1) >> torch.arange(32, device=w.device)) & 1
    return bits.reshape(-1)[:n_pairs].bool()


def _pack_pairs(reads, refs, m: int, with_n, stream):
    """Pack both sets; ``with_n=None`` packs without N masks first and packs
    again with them when the device saw an 'N' (shouji_unmasked_n)."""
    if with_n is None:
        shouji_unmasked_n()  # clear the flag
        pr, _ = shouji_pack(reads, m, stream=stream)
        pt, _ = shouji_pack(refs, m, stream=stream)
        if not shouji_unmasked_n():
            return pr, None, pt, None
        with_n = True
    pr, nr = shouji_pack(reads, m, with_n=with_n, stream=stream)
    pt, nt = shouji_pack(refs, m, with_n=with_n, stream=stream)
    return pr, nr, pt, nt


def filter_pairs(reads, refs, E: int, *, with_n: bool | None = None, E_per_pair=None,
                 stream=None):
    """Pack and filter (n, m) uint8 CUDA tensors of reads and references.

    Returns ``(accept_bool[n], count_uint8[n])``.  ``with_n=None`` (the
    default) filters without N masks and runs again with them when the
    device saw an 'N'.  Without N masks or per-pair thresholds this is one
    ``shouji_pack_filter`` call.
    """
    n, m = reads.shape
    assert refs.shape == reads.shape
    if not with_n and E_per_pair is None:
        if with_n is None:
            shouji_unmasked_n()  # clear the flag
        _, _, acc, cnt = shouji_pack_filter(reads, refs, m, E, stream=stream)
        if with_n is not None or not shouji_unmasked_n():
            return accept_to_bool(acc, n), cnt[:n]
        with_n = True
    pr, nr, pt, nt = _pack_pairs(reads, refs, m, with_n, stream)
    acc, cnt, _ = shouji_filter(pr, pt, m, n, E, reads_nmask=nr, refs_nmask=nt,
                                E_per_pair=E_per_pair, stream=stream)
    return accept_to_bool(acc, n), cnt[:n]


def magnet_pairs(reads, refs, E: int, *, with_n: bool | None = None, E_per_pair=None,
                 stream=None):
    """Pack (n, m) uint8 CUDA tensors of reads and references and run MAGNET.

    Returns ``(accept_bool[n], count_uint8[n])`` like ``filter_pairs``.
    """
    n, m = reads.shape
    assert refs.shape == reads.shape
    pr, nr, pt, nt = _pack_pairs(reads, refs, m, with_n, stream)
    acc, cnt, _ = shouji_magnet(pr, pt, m, n, E, reads_nmask=nr, refs_nmask=nt,
                                E_per_pair=E_per_pair, stream=stream)
    return accept_to_bool(acc, n), cnt[:n]


def _host_ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert not a.is_cuda and a.is_contiguous()
        return a.data_ptr()
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


class Pipeline:
    """``shouji_pipeline_*``: the whole filter for pairs held in host memory.

    Buffers are numpy arrays or CPU torch tensors (pin them for overlap).
    """

    def __init__(self, m: int, chunk_pairs: int = 1 << 22, max_pairs: int = 0,
                 with_n: bool = False):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.shouji_pipeline_create(m, chunk_pairs, max_pairs, int(with_n),
                                          ctypes.byref(h)), "shouji_pipeline_create")
        self._h = h
        self.m = m
        self.max_pairs = max_pairs

    def run(self, reads, refs, n_pairs: int, E: int, accept, *, count=None, idx=None,
            stride: int | None = None) -> int:
        """Filter; fills ``accept`` (uint32[ceil(n/32)]) and optionally
        ``count`` and ``idx``; returns the number of accepted pairs."""
        n_acc = ctypes.c_uint64(0)
        _check(load_library().shouji_pipeline_run(
            self._h, _host_ptr(reads), _host_ptr(refs), self.m if stride is None else stride,
            n_pairs, E, _host_ptr(accept), _host_ptr(count), _host_ptr(idx),
            ctypes.byref(n_acc)), "shouji_pipeline_run")
        return n_acc.value

    def run_packed(self, reads, refs, n_pairs: int, E: int, accept, *, reads_n=None,
                   refs_n=None, count=None, idx=None) -> int:
        """The same for pairs already in the packed layout (host uint32
        arrays of ``shouji_packed_words(n_pairs, m)`` words; N masks of
        ``shouji_nmask_words(n_pairs, m)`` words, or None)."""
        n_acc = ctypes.c_uint64(0)
        _check(load_library().shouji_pipeline_run_packed(
            self._h, _host_ptr(reads), _host_ptr(refs), _host_ptr(reads_n), _host_ptr(refs_n),
            n_pairs, E, _host_ptr(accept), _host_ptr(count), _host_ptr(idx),
            ctypes.byref(n_acc)), "shouji_pipeline_run_packed")
        return n_acc.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().shouji_pipeline_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """``shouji_batch_*``: pairs of mixed lengths and thresholds, bucketed,
    packed and filtered on the device in one CUDA-graph launch per batch.

    Tensors are CUDA tensors: ``reads``/``refs`` (n, stride) uint8, ``lens``
    int16/uint16-compatible int16 tensor or numpy-converted, ``E_per_pair``
    uint8.
    """

    def __init__(self, max_pairs: int, max_m: int, e_min: int, e_max: int,
                 with_n: bool = False, tune_cache: str | None = None):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.shouji_batch_create(max_pairs, max_m, e_min, e_max, int(with_n),
                                       tune_cache.encode() if tune_cache else None,
                                       ctypes.byref(h)), "shouji_batch_create")
        self._h = h
        self.max_pairs = max_pairs

    def _args(self, reads, refs, lens, E_per_pair, n_pairs, stride, out_accept, out_count):
        torch = _torch()
        dev = reads.device
        n = reads.shape[0] if n_pairs is None else n_pairs
        stride = reads.shape[1] if stride is None else stride
        if out_accept is None:
            out_accept = torch.empty(max(1, (n + 31) // 32), dtype=torch.int32, device=dev)
        return n, stride, out_accept, out_count

    def run(self, reads, refs, lens, E_per_pair, *, n_pairs=None, stride=None,
            out_accept=None, out_count=None, count: bool = True, stream=None):
        """Returns ``(accept_words, count)``."""
        torch = _torch()
        n, stride, out_accept, out_count = self._args(reads, refs, lens, E_per_pair, n_pairs,
                                                      stride, out_accept, out_count)
        if out_count is None and count:
            out_count = torch.empty(max(1, n), dtype=torch.uint8, device=reads.device)
        _check(load_library().shouji_batch_run(
            self._h, _ptr(reads), _ptr(refs), stride, _ptr(lens), _ptr(E_per_pair), n,
            _ptr(out_accept), _ptr(out_count), _stream(stream)), "shouji_batch_run")
        return out_accept, out_count

    def run_at(self, reads, ref_text, ref_offsets, lens, E_per_pair, *, n_pairs=None,
               stride=None, out_accept=None, out_count=None, count: bool = True, stream=None):
        """Like ``run``, with pair i's reference segment read from the device
        text ``ref_text`` at byte ``ref_offsets[i]`` (CUDA int64 tensor)."""
        torch = _torch()
        n, stride, out_accept, out_count = self._args(reads, None, lens, E_per_pair, n_pairs,
                                                      stride, out_accept, out_count)
        if out_count is None and count:
            out_count = torch.empty(max(1, n), dtype=torch.uint8, device=reads.device)
        _check(load_library().shouji_batch_run_at(
            self._h, _ptr(reads), stride, _ptr(ref_text), _ptr(ref_offsets), _ptr(lens),
            _ptr(E_per_pair), n, _ptr(out_accept), _ptr(out_count), _stream(stream)),
            "shouji_batch_run_at")
        return out_accept, out_count

    def tune(self, reads, refs, lens, E_per_pair, *, n_pairs=None, stride=None,
             cache: str | None = None, stream=None):
        n, stride, out_accept, _ = self._args(reads, refs, lens, E_per_pair, n_pairs, stride,
                                              None, None)
        _check(load_library().shouji_batch_tune(
            self._h, _ptr(reads), _ptr(refs), stride, _ptr(lens), _ptr(E_per_pair), n,
            _ptr(out_accept), None, cache.encode() if cache else None, _stream(stream)),
            "shouji_batch_tune")

    def timing(self) -> dict:
        """Stage durations (ms) the last run's graph recorded: ``graph``,
        ``bucketing``, ``pack``, ``filters``, ``finalize`` and ``filter_E``
        ({E: ms} for the thresholds in range)."""
        n = 5 + SHOUJI_MAX_E + 1
        buf = (ctypes.c_float * n)()
        _check(load_library().shouji_batch_timing(self._h, buf, n), "shouji_batch_timing")
        v = list(buf)
        return {"graph": v[0], "bucketing": v[1], "pack": v[2], "filters": v[3],
                "finalize": v[4], "filter_E": {E: v[5 + E] for E in range(SHOUJI_MAX_E + 1)
                                               if v[5 + E] >= 0}}

    def shape(self, E: int) -> dict:
        """Launch shape of threshold E's filter kernel (defaults or tuned)."""
        v = [ctypes.c_int(0) for _ in range(4)]
        _check(load_library().shouji_batch_shape(self._h, E, *[ctypes.byref(x) for x in v]),
               "shouji_batch_shape")
        return {"threads": v[0].value, "ctas_per_sm": v[1].value, "schedule": v[2].value,
                "windows": v[3].value}

    def invalid(self) -> int:
        v = ctypes.c_uint64(0)
        _check(load_library().shouji_batch_invalid(self._h, ctypes.byref(v)),
               "shouji_batch_invalid")
        return v.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().shouji_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _ServerRequest(ctypes.Structure):
    _fields_ = [("reads", ctypes.c_void_p), ("refs", ctypes.c_void_p),
                ("stride", ctypes.c_uint64), ("ref_id", ctypes.c_uint32),
                ("ref_offsets", ctypes.c_void_p), ("lens", ctypes.c_void_p),
                ("E_per_pair", ctypes.c_void_p), ("n_pairs", ctypes.c_size_t),
                ("accept", ctypes.c_void_p), ("count", ctypes.c_void_p),
                ("flags", ctypes.c_int)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("used_bytes", ctypes.c_uint64),
                ("peak_used_bytes", ctypes.c_uint64), ("reference_bytes", ctypes.c_uint64),
                ("workers", ctypes.c_int), ("busy_workers", ctypes.c_int),
                ("peak_busy_workers", ctypes.c_int), ("queued", ctypes.c_int),
                ("admitted", ctypes.c_uint64), ("workers_made", ctypes.c_uint64),
                ("workers_released", ctypes.c_uint64)]


SERVE_DEVICE_RESULTS = 1


class Server:
    """``shouji_server_*``: requests of mixed lengths and thresholds filtered as
    they arrive, admitted by device memory (continuous batching).

    Host buffers are numpy arrays or CPU torch tensors (pinned for overlap)
    and must stay alive until ``wait`` returns for the request; with
    ``device_results`` the outputs are CUDA tensors written on the device.
    """

    def __init__(self, max_request_pairs: int, max_m: int, e_min: int, e_max: int, *,
                 max_stride: int | None = None, with_n: bool = False,
                 memory_budget: int = 40 << 30, max_slots: int = 64,
                 tune_cache: str | None = None):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.shouji_server_create(max_request_pairs, max_m,
                                        max_m if max_stride is None else max_stride, e_min,
                                        e_max, int(with_n), memory_budget, max_slots,
                                        tune_cache.encode() if tune_cache else None,
                                        ctypes.byref(h)), "shouji_server_create")
        self._h = h
        self._keep = {}

    def info(self):
        """(workers held now, device bytes of a worker for the largest request)."""
        slots = ctypes.c_int(0)
        bps = ctypes.c_uint64(0)
        _check(load_library().shouji_server_info(self._h, ctypes.byref(slots), ctypes.byref(bps)),
               "shouji_server_info")
        return slots.value, bps.value

    def stats(self) -> dict:
        st = _ServerStats()
        _check(load_library().shouji_server_stats_read(self._h, ctypes.byref(st)),
               "shouji_server_stats_read")
        return {name: getattr(st, name) for name, _ in _ServerStats._fields_}

    def add_reference(self, text) -> int:
        """Make a reference text (host bytes) resident on the device; its id."""
        rid = ctypes.c_uint32(0)
        _check(load_library().shouji_server_add_reference(
            self._h, _host_ptr(text), int(text.nbytes if hasattr(text, "nbytes") else len(text)),
            ctypes.byref(rid)), "shouji_server_add_reference")
        return rid.value

    def _submit(self, req, keep) -> int:
        rid = ctypes.c_uint64(0)
        _check(load_library().shouji_server_submit_request(self._h, ctypes.byref(req),
                                                           ctypes.byref(rid)),
               "shouji_server_submit_request")
        self._keep[rid.value] = keep
        return rid.value

    def _outs(self, accept, count, device_results):
        if device_results:
            return _ptr(accept), _ptr(count), SERVE_DEVICE_RESULTS
        return _host_ptr(accept), _host_ptr(count), 0

    def submit(self, reads, refs, lens, E_per_pair, accept, count=None, *, n_pairs=None,
               stride=None, device_results: bool = False) -> int:
        """Pairs given as host rows of reads and reference segments."""
        n = len(lens) if n_pairs is None else n_pairs
        stride = reads.shape[1] if stride is None else stride
        acc, cnt, flags = self._outs(accept, count, device_results)
        req = _ServerRequest(_host_ptr(reads), _host_ptr(refs), stride, 0, None,
                             _host_ptr(lens), _host_ptr(E_per_pair), n, acc, cnt, flags)
        return self._submit(req, (reads, refs, lens, E_per_pair, accept, count))

    def submit_at(self, reads, ref_id: int, ref_offsets, lens, E_per_pair, accept, count=None,
                  *, n_pairs=None, stride=None, device_results: bool = False) -> int:
        """Pairs given as host rows of reads and offsets (host uint64) of
        their reference segments in the resident text ``ref_id``."""
        n = len(lens) if n_pairs is None else n_pairs
        stride = reads.shape[1] if stride is None else stride
        acc, cnt, flags = self._outs(accept, count, device_results)
        req = _ServerRequest(_host_ptr(reads), None, stride, ref_id, _host_ptr(ref_offsets),
                             _host_ptr(lens), _host_ptr(E_per_pair), n, acc, cnt, flags)
        return self._submit(req, (reads, ref_offsets, lens, E_per_pair, accept, count))

    def wait_timed(self, request_id: int, timeout: float = 60.0):
        """Block until done; returns (latency, gpu_start, gpu_end) in seconds
        (GPU times since the server was created).  Raises ``ShoujiError`` with
        status 4 (SHOUJI_ETIMEOUT) when the deadline passes."""
        t = (ctypes.c_double * 3)(-1.0, -1.0, -1.0)
        st = load_library().shouji_server_wait_timed(self._h, request_id, float(timeout), t)
        if st != 4:
            self._keep.pop(request_id, None)
        _check(st, "shouji_server_wait_timed")
        return t[0], t[1], t[2]

    def wait(self, request_id: int, timeout: float = 60.0) -> float:
        """Block until done; returns the latency in seconds."""
        return self.wait_timed(request_id, timeout)[0]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().shouji_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
