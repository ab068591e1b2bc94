"""'N' bases at the C ABI.  The paper's filter compares bases (Eq. 1); an 'N'
matches nothing (reading R8), which needs N masks.  Every pack without a mask
reads an 'N' as 'G' and sets a device flag that shouji_unmasked_n() reports
as SHOUJI_EINVAL; N-free input leaves it clear, bytes past the end of a row
(stride padding) never set it, and the one-call helpers take the masked path
when the flag comes up, giving the oracle's results."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1809_07858_gb300 as sj
from paper_1809_07858_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = ord("N")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def flag_status():
    lib = sj.load_library()
    v = ctypes.c_int(-1)
    st = lib.shouji_unmasked_n(ctypes.byref(v))
    return st, v.value


def with_one_n(reads, refs, which, row, col):
    reads, refs = reads.copy(), refs.copy()
    (reads if which == "read" else refs)[row, col] = N
    return reads, refs


@pytest.fixture(autouse=True)
def clear_flag():
    dev()
    sj.shouji_unmasked_n()
    yield
    sj.shouji_unmasked_n()


def test_flag_query_checks_its_argument():
    assert sj.load_library().shouji_unmasked_n(None) == 1


@pytest.mark.parametrize("m", [100, 98, 150])
def test_pack_without_mask(m):
    d = dev()
    reads, _ = synth.pairs(5000, m, seed=3, near=(0, 5))
    sj.shouji_pack(torch.from_numpy(reads).to(d), m)
    assert flag_status() == (0, 0)
    bad = reads.copy()
    bad[4999, m - 1] = N  # the last base of the last row
    sj.shouji_pack(torch.from_numpy(bad).to(d), m)
    assert flag_status() == (1, 1)
    assert flag_status() == (0, 0)  # read and reset
    # with a mask the 'N' is represented: no flag
    sj.shouji_pack(torch.from_numpy(bad).to(d), m, with_n=True)
    assert flag_status() == (0, 0)


@pytest.mark.parametrize("m,E", [(100, 5), (100, 2), (96, 5), (98, 3), (150, 5), (100, 8)])
def test_pack_filter_fused_and_separate(m, E):
    d = dev()
    reads, refs = synth.pairs(20_000, m, seed=5, near=(0, E), far=(E + 1, 25), far_fraction=0.5)
    r, t = torch.from_numpy(reads).to(d), torch.from_numpy(refs).to(d)
    sj.shouji_pack_filter(r, t, m, E)
    assert flag_status() == (0, 0)
    for which, row, col in (("read", 0, 0), ("ref", 12_345, m // 2), ("ref", 19_999, m - 1)):
        br, bt = with_one_n(reads, refs, which, row, col)
        sj.shouji_pack_filter(torch.from_numpy(br).to(d), torch.from_numpy(bt).to(d), m, E)
        assert flag_status() == (1, 1), (which, row, col)


def test_stride_padding_is_not_read_as_a_base():
    """Rows at a stride with 'N' bytes after each row's m bases (the batched
    form reads whole 16-byte chunks): no flag, and the results are those of
    the N-free rows."""
    d = dev()
    n = 30_000
    lens, Es = synth.mixed_shape(n, seed=17)
    reads, refs = synth.pairs(n, 250, seed=17, near=(0, 6), far=(7, 40), far_fraction=0.5,
                              lengths=lens, stride=256)
    for a in (reads, refs):
        for i in range(n):
            a[i, lens[i]:] = N
    b = sj.Batch(n, 250, 2, 12)
    acc, cnt = b.run(torch.from_numpy(reads).to(d), torch.from_numpy(refs).to(d),
                     torch.from_numpy(lens.astype(np.int16)).to(d), torch.from_numpy(Es).to(d))
    torch.cuda.synchronize()
    assert flag_status() == (0, 0)
    b.close()


def test_batch_without_masks_flags_and_with_masks_does_not():
    d = dev()
    n = 20_000
    lens, Es = synth.mixed_shape(n, seed=21)
    reads, refs = synth.pairs(n, 250, seed=21, near=(0, 6), far=(7, 40), far_fraction=0.5,
                              lengths=lens, stride=256)
    args = [torch.from_numpy(lens.astype(np.int16)).to(d), torch.from_numpy(Es).to(d)]
    plain = sj.Batch(n, 250, 2, 12)
    plain.run(torch.from_numpy(reads).to(d), torch.from_numpy(refs).to(d), *args)
    torch.cuda.synchronize()
    assert flag_status() == (0, 0)
    i = int(np.flatnonzero(lens == 150)[0])
    refs[i, 149] = N
    plain.run(torch.from_numpy(reads).to(d), torch.from_numpy(refs).to(d), *args)
    assert flag_status() == (1, 1)
    plain.close()
    masked = sj.Batch(n, 250, 2, 12, with_n=True)
    masked.run(torch.from_numpy(reads).to(d), torch.from_numpy(refs).to(d), *args)
    assert flag_status() == (0, 0)
    masked.close()


def test_pipeline_without_masks_returns_einval_with_results_written():
    dev()
    m, E, n = 100, 5, 50_000
    reads, refs = synth.pairs(n, m, seed=8, near=(0, E), far=(E + 1, 25), far_fraction=0.5)
    acc = np.zeros((n + 31) // 32, np.uint32)
    pipe = sj.Pipeline(m, chunk_pairs=1 << 14, max_pairs=n)
    pipe.run(reads, refs, n, E, acc)  # no 'N': OK
    reads[777, 3] = N
    acc2 = np.zeros_like(acc)
    with pytest.raises(sj.ShoujiError) as ei:
        pipe.run(reads, refs, n, E, acc2)
    assert ei.value.status == 1
    # every result was written: the pairs without 'N' agree with the first run
    same = np.ones(n, bool)
    same[777] = False
    a1 = np.unpackbits(acc.view(np.uint8), bitorder="little")[:n]
    a2 = np.unpackbits(acc2.view(np.uint8), bitorder="little")[:n]
    assert (a1[same] == a2[same]).all()
    pipe.close()
    masked = sj.Pipeline(m, chunk_pairs=1 << 14, max_pairs=n, with_n=True)
    acc3 = np.zeros_like(acc)
    masked.run(reads, refs, n, E, acc3)
    acc_o, _ = oracle.shouji_batch(reads, refs, E, threads=8)
    assert (np.unpackbits(acc3.view(np.uint8), bitorder="little")[:n] == acc_o).all()
    masked.close()


@pytest.mark.parametrize("helper", ["filter", "magnet"])
def test_helpers_take_the_masked_path_on_n(helper):
    d = dev()
    m, E, n = 100, 5, 8_000
    reads, refs = synth.pairs(n, m, seed=31, near=(0, E), far=(E + 1, 25), far_fraction=0.5)
    reads[5, 7] = N
    refs[4000, 99] = N
    refs[4001, 50] = N
    reads[4001, 50] = N  # 'N' against 'N' matches nothing either
    fn = sj.filter_pairs if helper == "filter" else sj.magnet_pairs
    acc, cnt = fn(torch.from_numpy(reads).to(d), torch.from_numpy(refs).to(d), E)
    acc_o, cnt_o = oracle.shouji_batch(reads, refs, E, threads=8, magnet=helper == "magnet")
    assert (acc.cpu().numpy() == acc_o).all()
    assert (cnt.cpu().numpy() == cnt_o).all()
    assert flag_status() == (0, 0)  # the helper read and cleared it
