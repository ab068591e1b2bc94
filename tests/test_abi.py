"""The C-ABI library loads and exports what include/shouji.h declares; host-side
argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_1809_07858_gb300 as sj

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "shouji.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(shouji_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for fn in ("shouji_pack", "shouji_filter", "shouji_magnet", "shouji_compact",
               "shouji_compact_workspace_size", "shouji_status_string"):
        assert fn in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(sj.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_size_helpers():
    assert sj.shouji_packed_words(0, 100) == 0
    assert sj.shouji_packed_words(1, 100) == 100 * 64
    assert sj.shouji_packed_words(1024, 100) == 100 * 64
    assert sj.shouji_packed_words(1025, 100) == 2 * 100 * 64
    assert sj.shouji_nmask_words(30_000_000, 100) == 29297 * 100 * 32
    assert sj.shouji_compact_workspace_size(0) == 0
    ws = sj.shouji_compact_workspace_size(30_000_000)
    assert ws % 16 == 0 and ws >= 4 * ((30_000_000 // 32 + 4095) // 4096)


def test_status_strings():
    for s in range(5):
        assert sj.shouji_status_string(s).startswith("SHOUJI")


def test_host_argument_checks_return_einval():
    lib = sj.load_library()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: every call below fails its checks
    EINVAL, OK = 1, 0
    # pack: m out of range, stride < m, null pointers
    assert lib.shouji_pack(fake, 100, 10, 0, fake, None, None) == EINVAL
    assert lib.shouji_pack(fake, 300, 10, 256, fake, None, None) == EINVAL
    assert lib.shouji_pack(fake, 99, 10, 100, fake, None, None) == EINVAL
    assert lib.shouji_pack(None, 100, 10, 100, fake, None, None) == EINVAL
    assert lib.shouji_pack(fake, 100, 10, 100, None, None, None) == EINVAL
    assert lib.shouji_pack(None, 100, 0, 100, None, None, None) == OK   # n = 0
    # filter: E range, m range, one-sided N mask, nulls, misalignment
    assert lib.shouji_filter(fake, fake, None, None, 100, 10, -1, None, fake, None, None, None) == EINVAL
    assert lib.shouji_filter(fake, fake, None, None, 100, 10, 32, None, fake, None, None, None) == EINVAL
    assert lib.shouji_filter(fake, fake, None, None, 0, 10, 5, None, fake, None, None, None) == EINVAL
    assert lib.shouji_filter(fake, fake, fake, None, 100, 10, 5, None, fake, None, None, None) == EINVAL
    assert lib.shouji_filter(None, fake, None, None, 100, 10, 5, None, fake, None, None, None) == EINVAL
    assert lib.shouji_filter(fake, fake, None, None, 100, 10, 5, None, None, None, None, None) == EINVAL
    assert lib.shouji_filter(ctypes.c_void_p(0x1004), fake, None, None, 100, 10, 5, None, fake,
                             None, None, None) == EINVAL
    assert lib.shouji_filter(None, None, None, None, 100, 0, 5, None, None, None, None, None) == OK
    # magnet: the checks of the filter
    assert lib.shouji_magnet(fake, fake, None, None, 100, 10, -1, None, fake, None, None, None) == EINVAL
    assert lib.shouji_magnet(fake, fake, None, None, 100, 10, 32, None, fake, None, None, None) == EINVAL
    assert lib.shouji_magnet(fake, fake, None, None, 256, 10, 5, None, fake, None, None, None) == EINVAL
    assert lib.shouji_magnet(fake, fake, None, fake, 100, 10, 5, None, fake, None, None, None) == EINVAL
    assert lib.shouji_magnet(fake, None, None, None, 100, 10, 5, None, fake, None, None, None) == EINVAL
    assert lib.shouji_magnet(fake, fake, None, None, 100, 10, 5, None, None, None, None, None) == EINVAL
    assert lib.shouji_magnet(fake, ctypes.c_void_p(0x1004), None, None, 100, 10, 5, None, fake,
                             None, None, None) == EINVAL
    assert lib.shouji_magnet(None, None, None, None, 100, 0, 5, None, None, None, None, None) == OK
    assert lib.shouji_wait_failures(None) == EINVAL
    # pack_filter: m, stride or E out of range, nulls, misaligned packed arrays; n = 0 is OK
    u64, sz = ctypes.c_uint64, ctypes.c_size_t
    pf = lib.shouji_pack_filter
    assert pf(fake, fake, u64(100), sz(10), 0, 5, fake, fake, fake, None, None) == EINVAL
    assert pf(fake, fake, u64(300), sz(10), 256, 5, fake, fake, fake, None, None) == EINVAL
    assert pf(fake, fake, u64(99), sz(10), 100, 5, fake, fake, fake, None, None) == EINVAL
    assert pf(fake, fake, u64(100), sz(10), 100, -1, fake, fake, fake, None, None) == EINVAL
    assert pf(fake, fake, u64(100), sz(10), 100, 32, fake, fake, fake, None, None) == EINVAL
    assert pf(None, fake, u64(100), sz(10), 100, 5, fake, fake, fake, None, None) == EINVAL
    assert pf(fake, None, u64(100), sz(10), 100, 5, fake, fake, fake, None, None) == EINVAL
    assert pf(fake, fake, u64(100), sz(10), 100, 5, None, fake, fake, None, None) == EINVAL
    assert pf(fake, fake, u64(100), sz(10), 100, 5, fake, None, fake, None, None) == EINVAL
    assert pf(fake, fake, u64(100), sz(10), 100, 5, fake, fake, None, None, None) == EINVAL
    assert pf(fake, fake, u64(100), sz(10), 100, 5, ctypes.c_void_p(0x1004), fake, fake, None,
              None) == EINVAL
    assert pf(None, None, u64(100), sz(0), 100, 5, None, None, None, None, None) == OK
    # pack_filter_results / its workspace size: nulls, short or misaligned
    # workspace, m, stride or E out of range (none of these needs a device)
    pr = lib.shouji_pack_filter_results
    assert pr(fake, fake, u64(100), sz(10), 0, 5, fake, sz(1 << 20), fake, None, None) == EINVAL
    assert pr(fake, fake, u64(99), sz(10), 100, 5, fake, sz(1 << 20), fake, None, None) == EINVAL
    assert pr(fake, fake, u64(100), sz(10), 100, 32, fake, sz(1 << 20), fake, None, None) == EINVAL
    assert pr(None, fake, u64(100), sz(10), 100, 5, fake, sz(1 << 20), fake, None, None) == EINVAL
    assert pr(fake, fake, u64(100), sz(10), 100, 5, None, sz(1 << 20), fake, None, None) == EINVAL
    assert pr(fake, fake, u64(100), sz(10), 100, 5, fake, sz(1 << 20), None, None, None) == EINVAL
    assert pr(fake, fake, u64(100), sz(10), 100, 5, ctypes.c_void_p(0x1008), sz(1 << 20), fake,
              None, None) == EINVAL
    assert pr(None, None, u64(100), sz(0), 100, 5, None, sz(0), None, None, None) == OK
    ws = lib.shouji_pack_filter_workspace_size
    b = sz(7)
    assert ws(fake, fake, u64(100), sz(10), 100, 5, None) == EINVAL
    assert ws(fake, fake, u64(100), sz(10), 256, 5, ctypes.byref(b)) == EINVAL and b.value == 0
    assert ws(fake, fake, u64(100), sz(10), 100, -1, ctypes.byref(b)) == EINVAL
    assert ws(fake, fake, u64(100), sz(0), 100, 5, ctypes.byref(b)) == OK and b.value == 0
    # rows that are not contiguous never take the fused kernel: both packed arrays
    assert ws(fake, fake, u64(112), sz(5000), 100, 5, ctypes.byref(b)) == OK
    assert b.value == 2 * 4 * sj.shouji_packed_words(5000, 100)
    assert lib.shouji_selftest_pack_wait(None) == EINVAL
    # host pipelines: no pipeline
    assert lib.shouji_pipeline_run(None, fake, fake, 100, 10, 5, fake, None, None, None) == EINVAL
    assert lib.shouji_pipeline_run_packed(None, fake, fake, None, None, 10, 5, fake, None, None,
                                          None) == EINVAL
    # compact: short or misaligned workspace, too many pairs, nulls
    assert lib.shouji_compact(fake, 1000, fake, fake, fake, 0, None) == EINVAL
    assert lib.shouji_compact(fake, 1000, fake, fake, ctypes.c_void_p(0x1008), 1 << 20, None) == EINVAL
    assert lib.shouji_compact(fake, 1 << 32, fake, fake, fake, 1 << 30, None) == EINVAL
    assert lib.shouji_compact(None, 1000, fake, fake, fake, 1 << 20, None) == EINVAL


def test_query_and_probe_argument_checks():
    lib = sj.load_library()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced
    EINVAL = 1
    f = ctypes.c_int(7)
    u64 = ctypes.c_uint64
    pff = lib.shouji_pack_filter_fused
    assert pff(fake, fake, u64(100), 100, 5, None) == EINVAL
    assert pff(fake, fake, u64(100), 0, 5, ctypes.byref(f)) == EINVAL and f.value == 0
    assert pff(fake, fake, u64(99), 100, 5, ctypes.byref(f)) == EINVAL
    assert pff(fake, fake, u64(100), 100, 32, ctypes.byref(f)) == EINVAL
    # rows that are not contiguous or not on 16 bytes never take the fused kernel;
    # this needs no device
    f.value = 7
    assert pff(fake, fake, u64(112), 100, 5, ctypes.byref(f)) == 0 and f.value == 0
    f.value = 7
    assert pff(ctypes.c_void_p(0x1004), fake, u64(100), 100, 5, ctypes.byref(f)) == 0
    assert f.value == 0
    assert lib.shouji_unmasked_n(None) == EINVAL
    assert lib.shouji_batch_timing(None, None, 0) == EINVAL
