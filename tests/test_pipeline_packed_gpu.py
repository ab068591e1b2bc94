"""The host pipeline on pairs the caller already holds in the packed 2-bit
layout (shouji_pipeline_run_packed) against the CPU oracle, bit-exact.

The packed inputs are written here by a plain numpy packer that follows the
layout stated in include/shouji.h (A=00, C=01, G=11, T=10 as hi, lo bits;
sequence s in tile s // 1024, lane (s % 1024) // 32, bit s % 32), so that
nothing of the input comes from the CUDA path."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1809_07858_gb300 as sj
from paper_1809_07858_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CODE = np.zeros(256, np.uint8)
for ch, c in zip(b"ACGTN", (0, 1, 3, 2, 3)):
    CODE[ch] = c


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def pack_numpy(seqs):
    """(packed words, N-mask words) of n rows of m ASCII bases."""
    n, m = seqs.shape
    tiles = (n + 1023) // 1024
    codes = np.zeros((tiles * 1024, m), np.uint8)   # rows past n: code 0, no N
    codes[:n] = CODE[seqs]
    isn = np.zeros((tiles * 1024, m), np.uint8)
    isn[:n] = seqs == ord("N")
    weight = (np.uint64(1) << np.arange(32, dtype=np.uint64))[None, None, :, None]

    def slice_words(bits):        # (tiles*1024, m) bits -> (tiles, m, 32 lanes) words
        b = bits.reshape(tiles, 32, 32, m).astype(np.uint64)
        return (b * weight).sum(axis=2).astype(np.uint32).transpose(0, 2, 1)

    hi = slice_words(codes >> 1)
    lo = slice_words(codes & 1)
    packed = np.ascontiguousarray(np.stack([hi, lo], axis=-1).reshape(-1))
    nmask = np.ascontiguousarray(slice_words(isn).reshape(-1))
    return packed, nmask


def accept_bits(acc, n):
    return ((acc[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:n].astype(bool)


def test_numpy_packer_follows_the_header_layout():
    """Pins the test's own packer: sequence 1029 (tile 1, lane 0, bit 5),
    position 2 holds 'G' = 11 and 'N'."""
    seqs = np.full((1030, 3), ord("A"), np.uint8)
    seqs[1029, 2] = ord("G")
    seqs[1029, 1] = ord("N")
    packed, nmask = pack_numpy(seqs)
    assert len(packed) == sj.shouji_packed_words(1030, 3)
    assert len(nmask) == sj.shouji_nmask_words(1030, 3)
    m = 3
    for p, want_hi, want_lo in ((2, 1, 1), (1, 1, 1), (0, 0, 0)):
        w = ((1 * m + p) * 32 + 0) * 2
        assert (packed[w] >> 5) & 1 == want_hi and (packed[w + 1] >> 5) & 1 == want_lo
    assert nmask[(1 * m + 1) * 32] == 1 << 5
    assert int(np.count_nonzero(packed)) == 4 and int(np.count_nonzero(nmask)) == 1


@pytest.mark.parametrize("n,chunk", [(1, 1024), (5000, 1024), (70_001, 16384)])
def test_packed_pipeline_bit_exact(n, chunk):
    need_gpu()
    reads, refs = synth.workload("sweep", n, E=5)
    acc_o, cnt_o = oracle.shouji_batch(reads, refs, 5, threads=8)
    pr, _ = pack_numpy(reads)
    pt, _ = pack_numpy(refs)
    pipe = sj.Pipeline(100, chunk_pairs=chunk, max_pairs=n)
    acc = np.zeros((n + 31) // 32, np.uint32)
    cnt = np.zeros(n, np.uint8)
    idx = np.zeros(n, np.uint32)
    k = pipe.run_packed(pr, pt, n, 5, acc, count=cnt, idx=idx)
    # and the ASCII entry of the same pipeline gives the same
    acc2 = np.zeros_like(acc)
    k2 = pipe.run(reads, refs, n, 5, acc2)
    pipe.close()
    assert k == int(acc_o.sum()) == k2
    assert (accept_bits(acc, n) == acc_o).all() and (acc2 == acc).all()
    assert (cnt == cnt_o).all()
    assert (idx[:k] == np.flatnonzero(acc_o)).all()


def test_packed_pipeline_with_N_masks():
    need_gpu()
    n, m, E = 9000, 150, 7
    reads, refs = synth.workload("long", n, m=m, E=E)
    assert (reads == ord("N")).any()
    acc_o, cnt_o = oracle.shouji_batch(reads, refs, E, threads=8)
    pr, nr = pack_numpy(reads)
    pt, nt = pack_numpy(refs)
    pipe = sj.Pipeline(m, chunk_pairs=4096, max_pairs=0, with_n=True)
    acc = np.zeros((n + 31) // 32, np.uint32)
    cnt = np.zeros(n, np.uint8)
    k = pipe.run_packed(pr, pt, n, E, acc, reads_n=nr, refs_n=nt, count=cnt)
    assert k == int(acc_o.sum())
    assert (accept_bits(acc, n) == acc_o).all() and (cnt == cnt_o).all()
    # only one of the two masks, or masks on a pipeline made without them: EINVAL
    with pytest.raises(sj.ShoujiError):
        pipe.run_packed(pr, pt, n, E, acc, reads_n=nr)
    pipe.close()
    plain = sj.Pipeline(m, chunk_pairs=4096)
    with pytest.raises(sj.ShoujiError):
        plain.run_packed(pr, pt, n, E, acc, reads_n=nr, refs_n=nt)
    plain.close()


def test_packed_pipeline_zero_pairs():
    need_gpu()
    pipe = sj.Pipeline(100, chunk_pairs=1024)
    lib = sj.load_library()
    n_acc = ctypes.c_uint64(7)
    assert lib.shouji_pipeline_run_packed(pipe._h, None, None, None, None, 0, 5, None, None,
                                          None, ctypes.byref(n_acc)) == 0
    assert n_acc.value == 0
    pipe.close()
