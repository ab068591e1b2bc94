"""shouji_magnet (MAGNET, Supplementary Sec. 7, Algorithms 3-4) against the
oracle, pair by pair: counts, accept bits and the MAGNET bit-vectors."""
import os

import numpy as np
import pytest

import oracle
import paper_1809_07858_gb300 as sj
from paper_1809_07858_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _bits(acc, n):
    w = acc.cpu().numpy().view(np.uint32)
    return ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:n].astype(bool)


def _vector(vec, m, i):
    """Column bits of pair i from the bit-sliced vector words."""
    t, l, b = i // 1024, (i % 1024) // 32, i % 32
    cols = vec[(t * m + np.arange(m)) * 32 + l]
    return ((cols >> np.uint32(b)) & 1).astype(np.uint8)


def _run(reads, refs, m, E, *, with_n, E_per_pair=None):
    dev = _dev()
    n = reads.shape[0]
    pr, nr = sj.shouji_pack(torch.from_numpy(np.ascontiguousarray(reads)).to(dev), m, with_n=with_n)
    pt, nt = sj.shouji_pack(torch.from_numpy(np.ascontiguousarray(refs)).to(dev), m, with_n=with_n)
    ep = None if E_per_pair is None else torch.from_numpy(E_per_pair).to(dev)
    acc, cnt, vec = sj.shouji_magnet(pr, pt, m, n, E, reads_nmask=nr, refs_nmask=nt,
                                     E_per_pair=ep, vectors=True)
    # Without vectors: the same accept words and counts.
    acc2, cnt2, _ = sj.shouji_magnet(pr, pt, m, n, E, reads_nmask=nr, refs_nmask=nt,
                                     E_per_pair=ep)
    torch.cuda.synchronize()
    assert torch.equal(acc, acc2)
    assert torch.equal(cnt[:n], cnt2[:n])
    return (_bits(acc, n), cnt[:n].cpu().numpy(),
            vec.cpu().numpy().view(np.uint32), acc.cpu().numpy().view(np.uint32))


def _check(reads, refs, m, E, bits, cnt, vec, E_per_pair=None, idx=None):
    idx = range(reads.shape[0]) if idx is None else idx
    for i in idx:
        e = E if E_per_pair is None else min(int(E_per_pair[i]), E)
        V, c = oracle.magnet(reads[i].tobytes(), refs[i].tobytes(), e)
        assert cnt[i] == c, (i, cnt[i], c)
        assert bits[i] == (c <= e), i
        assert (_vector(vec, m, i) == V).all(), i


@pytest.mark.parametrize("m,E,with_n", [(100, 5, False), (100, 5, True), (100, 2, False),
                                        (150, 7, False), (250, 12, True), (33, 3, False),
                                        (64, 0, False), (96, 9, False), (255, 31, False)])
def test_magnet_bit_exact(m, E, with_n):
    n = 2500  # three tiles, the last one ragged
    reads, refs = synth.pairs(n, m, seed=7 * m + E, near=(0, E + 1), far=(E + 1, m // 3 + 2),
                              far_fraction=0.5, n_rate=0.01 if with_n else 0.0)
    bits, cnt, vec, words = _run(reads, refs, m, E, with_n=with_n)
    _check(reads, refs, m, E, bits, cnt, vec)
    assert (words[-1] >> np.uint32(n % 32)) == 0 if n % 32 else True


def test_magnet_per_pair_threshold():
    m, E, n = 100, 10, 3000
    reads, refs = synth.pairs(n, m, seed=91, near=(0, 10), far=(11, 30), far_fraction=0.4)
    ep = np.random.default_rng(5).integers(0, E + 4, size=n).astype(np.uint8)  # some above E
    bits, cnt, vec, _ = _run(reads, refs, m, E, with_n=False, E_per_pair=ep)
    _check(reads, refs, m, E, bits, cnt, vec, E_per_pair=ep)


def test_magnet_edge_cases():
    rng = np.random.default_rng(11)
    for m in (1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 224, 255):
        for E in (0, 1, 4, 31):
            n = 70
            reads = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=(n, m))
            refs = reads.copy()
            refs[10:40] = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=(30, m))  # random
            refs[40:50] = rng.choice(np.frombuffer(b"GT", np.uint8), size=(10, m))
            reads[40:50] = rng.choice(np.frombuffer(b"AC", np.uint8), size=(10, m))  # disjoint
            refs[50:70, :] = np.roll(reads[50:70], 1 + (m // 7), axis=1)  # shifted copies
            bits, cnt, vec, _ = _run(reads, refs, m, E, with_n=False)
            _check(reads, refs, m, E, bits, cnt, vec)


def test_magnet_many_long_runs():
    """Pairs with more runs of 8 or more matching columns than the kernel lists
    (a read of one letter against a reference with a mismatch every 9
    columns: every diagonal then has a run of 8 between each two mismatches)."""
    rng = np.random.default_rng(12)
    for m in (100, 255):
        for E in (2, 5, 31):
            n = 64
            reads = np.full((n, m), ord("A"), np.uint8)
            refs = np.full((n, m), ord("A"), np.uint8)
            for i in range(n):
                period = 9 + (i % 4)
                refs[i, (i % period)::period] = ord("C")
                if i % 3 == 0:  # a few extra differences
                    refs[i, rng.integers(0, m, size=3)] = ord("G")
            bits, cnt, vec, _ = _run(reads, refs, m, E, with_n=False)
            _check(reads, refs, m, E, bits, cnt, vec)


def test_magnet_count_modes_with_short_reads():
    """MAGNET vectors recounted by shouji_count (local / glocal), with reads
    shorter than their reference packed as 'N' padding."""
    dev = _dev()
    m, E, n = 100, 4, 2000
    rng = np.random.default_rng(3)
    reads, refs = synth.pairs(n, m, seed=33, near=(0, E), far=(E + 1, 30), far_fraction=0.5)
    short = rng.random(n) < 0.4
    mp = np.where(short, rng.integers(m // 2, m + 1, size=n), m)
    for i in np.flatnonzero(short):
        reads[i, mp[i]:] = ord("N")
    bits, cnt, vec, _ = _run(reads, refs, m, E, with_n=True)
    vec_t = torch.from_numpy(vec.view(np.int32)).to(dev)
    for mode in range(4):
        acc, c = sj.shouji_count(vec_t, m, n, E, mode)
        torch.cuda.synchronize()
        c = c[:n].cpu().numpy()
        b = _bits(acc, n)
        for i in range(n):
            _, co = oracle.magnet(reads[i, :mp[i]].tobytes(), refs[i].tobytes(), E, mode)
            assert c[i] == co, (mode, i)
            assert b[i] == (co <= E)


def test_magnet_full_size(host_buffers):
    """The benchmark's MAGNET workload (30M pairs, m = 100, E = 5, half of them
    near, half far) in one launch, every pair checked against the oracle (run
    on all host cores)."""
    dev = _dev()
    n, m, E = 30_000_000, 100, 5
    reads, refs = synth.workload("sweep", n, E=E, out=host_buffers.views(n, m))
    pr, _ = sj.shouji_pack(torch.from_numpy(reads).to(dev), m)
    pt, _ = sj.shouji_pack(torch.from_numpy(refs).to(dev), m)
    acc, cnt, _ = sj.shouji_magnet(pr, pt, m, n, E)
    torch.cuda.synchronize()
    bits = _bits(acc, n)
    cnt = cnt.cpu().numpy()
    acc_o, cnt_o = oracle.shouji_batch(reads, refs, E, threads=max(1, os.cpu_count() or 1),
                                       magnet=True)
    bad = np.flatnonzero((cnt != cnt_o) | (bits != acc_o))
    assert bad.size == 0, "%d pairs differ, first %s" % (bad.size, bad[:10])
    del pr, pt, acc
    torch.cuda.empty_cache()


def test_magnet_random_configurations():
    """Random lengths, thresholds, N densities, alphabets and per-pair
    thresholds, every pair's count and accept bit against the oracle."""
    dev = _dev()
    rng = np.random.default_rng(2024)
    for trial in range(40):
        m = int(rng.choice([int(rng.integers(1, 256)), 100, 150, 250]))
        E = int(rng.integers(0, 32))
        n = int(rng.integers(1, 3000))
        alphabet = np.frombuffer(rng.choice([b"ACGT", b"AC", b"AAAC", b"ACGTN"]), np.uint8)
        reads = rng.choice(alphabet, size=(n, m)).astype(np.uint8)
        refs = reads.copy()
        # near pairs: a few substitutions and shifts; far pairs: random
        k = rng.integers(0, max(1, E + 3), size=n)
        for i in range(n):
            if rng.random() < 0.3:
                refs[i] = rng.choice(alphabet, size=m)
                continue
            for _ in range(int(k[i])):
                pos = int(rng.integers(0, m))
                if rng.random() < 0.6:
                    refs[i, pos] = rng.choice(alphabet)
                else:
                    refs[i, pos:] = np.roll(refs[i, pos:], 1 if rng.random() < 0.5 else -1)
        with_n = bool((reads == ord("N")).any() or (refs == ord("N")).any() or rng.random() < 0.3)
        ep = rng.integers(0, E + 2, size=n).astype(np.uint8) if rng.random() < 0.3 else None
        pr, nr = sj.shouji_pack(torch.from_numpy(reads).to(dev), m, with_n=with_n)
        pt, nt = sj.shouji_pack(torch.from_numpy(refs).to(dev), m, with_n=with_n)
        acc, cnt, _ = sj.shouji_magnet(pr, pt, m, n, E, reads_nmask=nr, refs_nmask=nt,
                                       E_per_pair=None if ep is None else torch.from_numpy(ep).to(dev))
        torch.cuda.synchronize()
        bits, cnt = _bits(acc, n), cnt[:n].cpu().numpy()
        # without N masks an 'N' is read as 'G'
        r_o = reads if with_n else np.where(reads == ord("N"), ord("G"), reads).astype(np.uint8)
        t_o = refs if with_n else np.where(refs == ord("N"), ord("G"), refs).astype(np.uint8)
        e_o = None if ep is None else np.minimum(ep, E).astype(np.uint8)
        acc_o, cnt_o = oracle.shouji_batch(r_o, t_o, E, E_per_pair=e_o, threads=8, magnet=True)
        bad = np.flatnonzero((cnt != cnt_o) | (bits != acc_o))
        assert bad.size == 0, (trial, m, E, n, with_n, ep is not None, bad[:5])


def test_magnet_pairs_convenience():
    """magnet_pairs (pack + MAGNET in one call) on ASCII tensors, with 'N'."""
    dev = _dev()
    n, m, E = 1500, 120, 6
    reads, refs = synth.pairs(n, m, seed=77, near=(0, 6), far=(7, 30), far_fraction=0.5,
                              n_rate=0.01)
    acc, cnt = sj.magnet_pairs(torch.from_numpy(reads).to(dev), torch.from_numpy(refs).to(dev), E)
    torch.cuda.synchronize()
    acc_o, cnt_o = oracle.shouji_batch(reads, refs, E, threads=8, magnet=True)
    assert (acc.cpu().numpy() == acc_o).all()
    assert (cnt.cpu().numpy() == cnt_o).all()
