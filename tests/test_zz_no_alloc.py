"""shouji_compact_noalloc: the compaction variant for callers that cannot
allocate device memory (their memory belongs to another allocator, or they
must not call cudaMalloc/cudaFree in a latency-bound loop).  It keeps its
workspace in a fixed array inside the library; its results must equal those
of shouji_compact, which uses a caller-allocated workspace.

This file is collected last on purpose (it runs after every other test when
the suite stops at the first failure)."""
import ctypes

import numpy as np
import pytest

import paper_1809_07858_gb300 as sj

torch = pytest.importorskip("torch")


def _random_accept(n, density, seed):
    rng = np.random.default_rng(seed)
    bits = np.zeros((n + 31) // 32 * 32, np.uint8)
    bits[:n] = rng.random(n) < density
    words = np.packbits(bits.reshape(-1, 32)[:, ::-1], axis=1).view(">u4").astype(np.uint32).ravel()
    return words.view(np.int32)


@pytest.mark.gpu
def test_noalloc_matches_compact_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    lib = sj.load_library()
    for call, (n, density) in enumerate([(5_000_001, 0.4), (777_777, 0.9)]):
        acc = torch.from_numpy(_random_accept(n, density, seed=call)).to(dev)
        idx_ref, n_ref = sj.shouji_compact(acc, n)
        idx = torch.full((n,), -1, dtype=torch.int32, device=dev)
        cnt = torch.full((1,), -1, dtype=torch.int32, device=dev)
        status = lib.shouji_compact_noalloc(acc.data_ptr(), n, idx.data_ptr(), cnt.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
        assert status == 0, sj.shouji_status_string(status)
        torch.cuda.synchronize()
        k = int(n_ref.item())
        assert int(cnt.item()) == k
        assert torch.equal(idx[:k], idx_ref[:k])


def test_noalloc_rejects_more_pairs_than_its_workspace_holds():
    lib = sj.load_library()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the size check comes first
    assert lib.shouji_compact_noalloc(fake, sj.SHOUJI_NOALLOC_MAX_PAIRS + 1, fake, fake, None) == 1
