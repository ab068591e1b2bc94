"""shouji_compact_noalloc: the compaction variant for callers that cannot
allocate device memory (their memory belongs to another allocator, or they
must not call cudaMalloc/cudaFree in a latency-bound loop).  It keeps its
workspace in a fixed array inside the library; its results must equal those
of shouji_compact, which uses a caller-allocated workspace, and the indices
of the set accept bits.

This file is collected last on purpose (it runs after every other test when
the suite stops at the first failure)."""
import ctypes
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import paper_1809_07858_gb300 as sj

torch = pytest.importorskip("torch")


def _words_from_positions(n, positions):
    """Accept words (bit i % 32 of word i / 32) with the given bits set."""
    words = np.zeros((n + 31) // 32, np.uint32)
    np.bitwise_or.at(words, positions // 32, (np.uint32(1) << (positions % 32).astype(np.uint32)))
    return words


def _random_positions(n, density, seed):
    rng = np.random.default_rng(seed)
    if density >= 0.05:
        return np.flatnonzero(rng.random(n) < density)
    k = int(n * density)
    return np.unique(rng.integers(0, n, size=k, dtype=np.int64))


def _noalloc(lib, acc, n, stream):
    dev = acc.device
    idx = torch.full((n,), -1, dtype=torch.int32, device=dev)
    cnt = torch.full((1,), -1, dtype=torch.int32, device=dev)
    status = lib.shouji_compact_noalloc(acc.data_ptr(), n, idx.data_ptr(), cnt.data_ptr(),
                                        stream.cuda_stream)
    assert status == 0, sj.shouji_status_string(status)
    return idx, cnt


@pytest.mark.gpu
def test_noalloc_matches_compact_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    lib = sj.load_library()
    for call, (n, density) in enumerate([(5_000_001, 0.4), (777_777, 0.9)]):
        pos = _random_positions(n, density, seed=call)
        acc = torch.from_numpy(_words_from_positions(n, pos).view(np.int32)).to(dev)
        idx_ref, n_ref = sj.shouji_compact(acc, n)
        idx, cnt = _noalloc(lib, acc, n, torch.cuda.current_stream())
        torch.cuda.synchronize()
        k = int(n_ref.item())
        assert k == len(pos)
        assert int(cnt.item()) == k
        assert torch.equal(idx[:k], idx_ref[:k])
        assert np.array_equal(idx[:k].cpu().numpy(), pos)


@pytest.mark.gpu
def test_noalloc_at_its_size_limit_on_a_side_stream():
    """n = SHOUJI_NOALLOC_MAX_PAIRS fills every slice sum of the array; the
    call runs on a non-default stream."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    lib = sj.load_library()
    n = sj.SHOUJI_NOALLOC_MAX_PAIRS
    pos = _random_positions(n, 1e-3, seed=7)
    pos = np.union1d(pos, np.array([0, 31, 32, n - 33, n - 1]))  # first and last words
    acc = torch.from_numpy(_words_from_positions(n, pos).view(np.int32)).to(dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        idx, cnt = _noalloc(lib, acc, n, side)
        idx_ref, n_ref = sj.shouji_compact(acc, n, stream=side)
    side.synchronize()
    k = len(pos)
    assert int(cnt.item()) == k and int(n_ref.item()) == k
    got = idx[:k].cpu().numpy()
    assert np.array_equal(got, pos)
    assert torch.equal(idx[:k], idx_ref[:k])
    del idx, idx_ref, acc
    torch.cuda.empty_cache()


_CONTEXT_SCRIPT = textwrap.dedent(r"""
    import ctypes, sys
    import numpy as np
    lib = ctypes.CDLL(sys.argv[1])
    cu = ctypes.CDLL("libcuda.so.1")
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    lib.shouji_compact_noalloc.argtypes = [vp, sz, vp, vp, vp]
    lib.shouji_compact.argtypes = [vp, sz, vp, vp, vp, sz, vp]
    lib.shouji_compact_workspace_size.argtypes = [sz]
    lib.shouji_compact_workspace_size.restype = sz

    def ok(r, what):
        if r != 0:
            raise SystemExit("%s failed: %d" % (what, r))

    ok(cu.cuInit(0), "cuInit")
    dev = ctypes.c_int(0)
    ok(cu.cuDeviceGet(ctypes.byref(dev), 0), "cuDeviceGet")
    n = 3_000_017
    rng = np.random.default_rng(11)
    bits = rng.random(n) < 0.3
    pos = np.flatnonzero(bits)
    words = np.zeros((n + 31) // 32, np.uint32)
    np.bitwise_or.at(words, pos // 32, (np.uint32(1) << (pos % 32).astype(np.uint32)))

    def alloc(nbytes):
        p = ctypes.c_uint64(0)
        ok(cu.cuMemAlloc_v2(ctypes.byref(p), ctypes.c_size_t(nbytes)), "cuMemAlloc")
        return p.value

    def run_in_current_context(tag):
        d_acc, d_idx, d_n = alloc(words.nbytes), alloc(4 * n), alloc(4)
        ws_bytes = lib.shouji_compact_workspace_size(n)
        d_ws, d_idx2, d_n2 = alloc(ws_bytes), alloc(4 * n), alloc(4)
        ok(cu.cuMemcpyHtoD_v2(ctypes.c_uint64(d_acc), words.ctypes.data_as(vp),
                              ctypes.c_size_t(words.nbytes)), "copy in")
        for call in range(2):
            ok(lib.shouji_compact_noalloc(d_acc, n, d_idx, d_n, None), tag + " noalloc")
            ok(lib.shouji_compact(d_acc, n, d_idx2, d_n2, d_ws, ws_bytes, None), tag + " compact")
            ok(cu.cuCtxSynchronize(), tag + " synchronize")
            for d_out, d_cnt, what in ((d_idx, d_n, "noalloc"), (d_idx2, d_n2, "compact")):
                k = np.zeros(1, np.uint32)
                ok(cu.cuMemcpyDtoH_v2(k.ctypes.data_as(vp), ctypes.c_uint64(d_cnt),
                                      ctypes.c_size_t(4)), "copy count")
                got = np.zeros(int(k[0]), np.uint32)
                if got.size:
                    ok(cu.cuMemcpyDtoH_v2(got.ctypes.data_as(vp), ctypes.c_uint64(d_out),
                                          ctypes.c_size_t(got.nbytes)), "copy indices")
                if not np.array_equal(got, pos):
                    raise SystemExit("%s %s call %d: wrong indices" % (tag, what, call))
        for p in (d_acc, d_idx, d_n, d_ws, d_idx2, d_n2):
            ok(cu.cuMemFree_v2(ctypes.c_uint64(p)), "cuMemFree")

    primary = ctypes.c_void_p(0)
    ok(cu.cuDevicePrimaryCtxRetain(ctypes.byref(primary), dev), "retain primary")
    ok(cu.cuCtxSetCurrent(primary), "set primary")
    run_in_current_context("primary")
    own = ctypes.c_void_p(0)
    ok(cu.cuCtxCreate_v4(ctypes.byref(own), None, 0, dev), "cuCtxCreate")
    run_in_current_context("own context")
    ok(cu.cuCtxSetCurrent(primary), "back to primary")
    run_in_current_context("primary again")
    ok(cu.cuCtxSetCurrent(own), "back to own context")
    run_in_current_context("own context again")
    ok(cu.cuCtxSetCurrent(primary), "primary before destroy")
    ok(cu.cuCtxDestroy_v2(own), "cuCtxDestroy")
    print("contexts ok")
""")


@pytest.mark.gpu
def test_noalloc_in_a_second_context_on_the_same_device():
    """The array's address belongs to a context: a call made while another
    context of the same GPU is current (here one the program created with
    the driver API) must look the address up in that context, and calls in
    the first context must still use the first context's address.  Runs in a
    fresh process that uses only the driver API and this library."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-c", _CONTEXT_SCRIPT, sj.LIB_PATH],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "contexts ok" in r.stdout


def test_noalloc_rejects_more_pairs_than_its_workspace_holds():
    lib = sj.load_library()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the size check comes first
    assert lib.shouji_compact_noalloc(fake, sj.SHOUJI_NOALLOC_MAX_PAIRS + 1, fake, fake, None) == 1
