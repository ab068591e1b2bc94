"""The batched path (mixed lengths and thresholds in one CUDA-graph launch)
against the oracle, pair by pair: accept bits and counts bit-exact."""
import os

import numpy as np
import pytest

import oracle
import paper_1809_07858_gb300 as sj
from paper_1809_07858_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def oracle_mixed(reads, refs, lens, Es, threads=8):
    """Per pair: the oracle on the first lens[i] bases at threshold Es[i]."""
    n = len(lens)
    acc = np.zeros(n, bool)
    cnt = np.zeros(n, np.uint8)
    for L in np.unique(lens):
        idx = np.flatnonzero(lens == L)
        a, c = oracle.shouji_batch(reads[idx, :L], refs[idx, :L], 0,
                                   E_per_pair=Es[idx].astype(np.uint8), threads=threads)
        acc[idx], cnt[idx] = a, c
    return acc, cnt


def accept_bits(words, n):
    w = words.view(np.uint32)
    return ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:n].astype(bool)


def run_batch(b, reads, refs, lens, Es, stride=None):
    d = dev()
    acc, cnt = b.run(torch.from_numpy(np.ascontiguousarray(reads)).to(d),
                     torch.from_numpy(np.ascontiguousarray(refs)).to(d),
                     torch.from_numpy(lens.astype(np.int16)).to(d),
                     torch.from_numpy(Es.astype(np.uint8)).to(d), stride=stride)
    torch.cuda.synchronize()
    n = len(lens)
    return accept_bits(acc.cpu().numpy(), n), cnt[:n].cpu().numpy()


def mixed_batch(n, seed, n_rate=0.0, choices=(100, 150, 250), weights=(0.4, 0.4, 0.2),
                e_range=(2, 12), stride=256):
    lens, Es = synth.mixed_shape(n, seed=seed, choices=choices, weights=weights, e_range=e_range)
    reads, refs = synth.pairs(n, max(choices), seed=seed, near=(0, 6), far=(7, 40),
                              far_fraction=0.5, n_rate=n_rate, lengths=lens, stride=stride)
    return reads, refs, lens, Es


def test_mixed_lengths_and_thresholds_bit_exact():
    reads, refs, lens, Es = mixed_batch(20_000, seed=1)
    b = sj.Batch(50_000, 255, 2, 12)
    acc, cnt = run_batch(b, reads, refs, lens, Es)
    acc_o, cnt_o = oracle_mixed(reads, refs, lens, Es)
    assert (cnt == cnt_o).all(), np.flatnonzero(cnt != cnt_o)[:10]
    assert (acc == acc_o).all()
    assert b.invalid() == 0
    # the same object again, another batch of another size (graph reuse)
    reads, refs, lens, Es = mixed_batch(7_777, seed=2)
    acc, cnt = run_batch(b, reads, refs, lens, Es)
    acc_o, cnt_o = oracle_mixed(reads, refs, lens, Es)
    assert (cnt == cnt_o).all() and (acc == acc_o).all()
    b.close()


def test_every_length_and_threshold_with_N():
    rng = np.random.default_rng(3)
    n = 12_000
    lens = rng.integers(1, 256, size=n).astype(np.uint16)
    Es = rng.integers(0, 32, size=n).astype(np.uint8)
    reads, refs = synth.pairs(n, 255, seed=3, near=(0, 8), far=(9, 60), far_fraction=0.5,
                              n_rate=0.01, lengths=lens, stride=255)
    b = sj.Batch(n, 255, 0, 31, with_n=True)
    acc, cnt = run_batch(b, reads, refs, lens, Es)
    acc_o, cnt_o = oracle_mixed(reads, refs, lens, Es)
    assert (cnt == cnt_o).all(), np.flatnonzero(cnt != cnt_o)[:10]
    assert (acc == acc_o).all()
    b.close()


def test_out_of_range_pairs_are_rejected_and_counted():
    n = 3000
    lens, Es = synth.mixed_shape(n, seed=4)
    lens[::97] = 0          # length 0: out of range
    lens[5::101] = 250      # in range
    Es[7::89] = 13          # threshold above e_max
    reads, refs = synth.pairs(n, 250, seed=4, near=(0, 6), far=(7, 40), far_fraction=0.5,
                              lengths=lens, stride=256)
    bad = (lens == 0) | (Es > 12)
    b = sj.Batch(n, 250, 2, 12)
    acc, cnt = run_batch(b, reads, refs, lens, Es)
    assert b.invalid() == int(bad.sum())
    assert (~acc[bad]).all() and (cnt[bad] == 255).all()
    ok = ~bad
    acc_o, cnt_o = oracle_mixed(reads[ok], refs[ok], lens[ok], Es[ok])
    assert (cnt[ok] == cnt_o).all() and (acc[ok] == acc_o).all()
    b.close()


def test_tuned_shapes_give_identical_results(tmp_path):
    reads, refs, lens, Es = mixed_batch(40_000, seed=5)
    d = dev()
    args = (torch.from_numpy(reads).to(d), torch.from_numpy(refs).to(d),
            torch.from_numpy(lens.astype(np.int16)).to(d), torch.from_numpy(Es).to(d))
    cache = str(tmp_path / "tune.txt")
    b = sj.Batch(40_000, 255, 2, 12)
    acc0, cnt0 = b.run(*args)
    torch.cuda.synchronize()
    acc0, cnt0 = acc0.cpu().clone(), cnt0.cpu().clone()
    b.tune(*args, cache=cache)
    acc1, cnt1 = b.run(*args)
    torch.cuda.synchronize()
    assert torch.equal(acc0, acc1.cpu()) and torch.equal(cnt0, cnt1.cpu())
    lines = [l.split() for l in open(cache).read().split("\n") if l.strip()]
    assert len(lines) == 11     # E = 2..12 present in the batch
    b2 = sj.Batch(40_000, 255, 2, 12, tune_cache=cache)   # reads the cache back
    for f in lines:
        E = int(f[1])
        want = {"threads": int(f[2]), "ctas_per_sm": int(f[3]), "schedule": int(f[4]),
                "windows": int(f[5])}
        assert b.shape(E) == want and b2.shape(E) == want
        assert want["windows"] in (4, 8) and (want["windows"] == 4 or E <= 6)
    acc2, cnt2 = b2.run(*args)
    torch.cuda.synchronize()
    assert torch.equal(acc0, acc2.cpu()) and torch.equal(cnt0, cnt2.cpu())
    b.close()
    b2.close()


@pytest.mark.parametrize("with_n", [False, True])
def test_eight_windows_per_chunk_bit_exact(tmp_path, with_n):
    """The filter kernels with 8 windows per chunk (thresholds up to 6),
    forced through a tuning cache, against the oracle."""
    reads, refs, lens, Es = mixed_batch(30_000, seed=8, n_rate=0.002 if with_n else 0.0,
                                        choices=(1, 7, 33, 100, 150, 255),
                                        weights=(0.05, 0.1, 0.15, 0.3, 0.3, 0.1), e_range=(0, 6))
    cache = tmp_path / "u8.txt"
    gpu = torch.cuda.get_device_name(0).replace(" ", "_")
    cache.write_text("".join("%s %d 64 4 2 8 1.0\n" % (gpu, E) for E in range(0, 7)))
    b = sj.Batch(30_000, 255, 0, 6, with_n=with_n, tune_cache=str(cache))
    assert all(b.shape(E)["windows"] == 8 for E in range(0, 7))
    acc, cnt = run_batch(b, reads, refs, lens, Es)
    acc_o, cnt_o = oracle_mixed(reads, refs, lens, Es)
    assert (cnt == cnt_o).all() and (acc == acc_o).all()
    b.close()


def test_runs_queued_back_to_back_use_their_own_arguments():
    """Runs alternate between two argument blocks: three batches queued on one
    stream without waiting (outputs into separate buffers) each give the
    results they give alone."""
    d = dev()
    batches = [mixed_batch(30_000, seed=s) for s in (31, 32, 33)]
    b = sj.Batch(30_000, 250, 2, 12)
    outs = []
    for reads, refs, lens, Es in batches:
        outs.append(b.run(torch.from_numpy(reads).to(d), torch.from_numpy(refs).to(d),
                          torch.from_numpy(lens.astype(np.int16)).to(d),
                          torch.from_numpy(Es).to(d)))
    torch.cuda.synchronize()
    for (reads, refs, lens, Es), (acc, cnt) in zip(batches, outs):
        acc_o, cnt_o = oracle_mixed(reads, refs, lens, Es)
        assert (accept_bits(acc.cpu().numpy(), len(lens)) == acc_o).all()
        assert (cnt[:len(lens)].cpu().numpy() == cnt_o).all()
    b.close()


def test_stage_timing_recorded_by_the_graph():
    reads, refs, lens, Es = mixed_batch(200_000, seed=34)
    b = sj.Batch(200_000, 250, 2, 12)
    t0 = b.timing()
    assert t0["graph"] == -1 and t0["filter_E"] == {}   # before the first run
    run_batch(b, reads, refs, lens, Es)
    t = b.timing()
    assert t["graph"] > 0 and t["filters"] > 0 and t["pack"] > 0
    assert t["bucketing"] >= 0 and t["finalize"] >= 0
    parts = t["bucketing"] + t["pack"] + t["filters"] + t["finalize"]
    assert abs(parts - t["graph"]) <= 0.05 * t["graph"] + 0.02
    assert sorted(t["filter_E"]) == list(range(2, 13))
    for E, ms in t["filter_E"].items():
        assert 0 < ms <= t["filters"] + 1e-3, (E, ms)
    b.close()


def test_unaligned_stride_byte_path():
    reads, refs, lens, Es = mixed_batch(5000, seed=6, stride=251)
    b = sj.Batch(5000, 250, 2, 12)
    acc, cnt = run_batch(b, reads, refs, lens, Es)
    acc_o, cnt_o = oracle_mixed(reads, refs, lens, Es)
    assert (cnt == cnt_o).all() and (acc == acc_o).all()
    b.close()


@pytest.mark.slow
def test_full_size_batch_every_pair(host_buffers):
    """The benchmark's batched workload at its full size (50M pairs, lengths
    40% 100 / 40% 150 / 20% 250, E uniform in 2..12, unsorted, stride 256) in one
    graph launch: properties over every pair, and every pair against the
    oracle (run on all host cores, in chunks)."""
    d = dev()
    n = 50_000_000
    lens, Es = synth.mixed_shape(n, seed=4242)
    reads, refs = synth.pairs(n, 250, seed=4242, near=(0, 6), far=(7, 40), far_fraction=0.5,
                              lengths=lens, stride=256, out=host_buffers.views(n, 256))
    b = sj.Batch(n, 250, 2, 12)
    acc, cnt = b.run(torch.from_numpy(reads).to(d), torch.from_numpy(refs).to(d),
                     torch.from_numpy(lens.astype(np.int16)).to(d), torch.from_numpy(Es).to(d))
    torch.cuda.synchronize()
    invalid = b.invalid()
    b.close()
    bits = accept_bits(acc.cpu().numpy(), n)
    cnt = cnt[:n].cpu().numpy()
    assert invalid == 0
    assert (cnt <= lens).all()
    assert (bits == (cnt <= Es)).all()
    del acc
    torch.cuda.empty_cache()
    threads = max(1, os.cpu_count() or 1)
    chunk = 4_000_000
    for s0 in range(0, n, chunk):
        sl = slice(s0, min(n, s0 + chunk))
        acc_o, cnt_o = oracle_mixed(reads[sl], refs[sl], lens[sl], Es[sl], threads=threads)
        bad = np.flatnonzero((cnt[sl] != cnt_o) | (bits[sl] != acc_o))
        assert bad.size == 0, "pairs %d.. : %d differ, first %s" % (s0, bad.size, bad[:10] + s0)
