"""shouji_pack_filter: both packs and the filter in one call (a fused
warp-specialized kernel when rows are contiguous on 16-byte boundaries, E <= 5
and m is within the staging rings; the separate launches otherwise).  Accept
bits and counts are compared with the oracle pair by pair, and the packed
words with an independent unpack of the ASCII input, across lengths,
thresholds, ragged sizes, sizes that give a CTA one tile or hundreds, and the
fallback layouts."""
import numpy as np
import pytest

import oracle
import paper_1809_07858_gb300 as sj
from paper_1809_07858_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CODE = np.zeros(256, np.uint8)
for ch, v in ((b"A", 0), (b"C", 1), (b"G", 3), (b"T", 2), (b"N", 3)):
    CODE[ch[0]] = v


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def unpack_planes(words, n, m):
    tiles = (n + 1023) // 1024
    w = words[: tiles * m * 64].view(np.uint32).reshape(tiles, m, 32, 2)
    b = np.arange(32, dtype=np.uint32)
    hi = (w[..., 0][..., None] >> b) & 1
    lo = (w[..., 1][..., None] >> b) & 1
    return (hi * 2 + lo).transpose(0, 2, 3, 1).reshape(tiles * 1024, m)[:n].astype(np.uint8)


def accept_bits(acc, n):
    return sj.accept_to_bool(acc, n).cpu().numpy()


def check(reads, refs, m, E, *, stride_pad=0, offset=0, packing=True):
    d = dev()
    n = len(reads)
    if stride_pad or offset:
        stride = m + stride_pad
        def place(a):
            buf = torch.zeros(offset + n * stride + 64, dtype=torch.uint8, device=d)
            rows = np.zeros((n, stride), np.uint8)
            rows[:, :m] = a
            buf[offset: offset + n * stride] = torch.from_numpy(rows.reshape(-1)).to(d)
            return buf[offset: offset + n * stride]
        r, t = place(reads), place(refs)
        pr, pt, acc, cnt = sj.shouji_pack_filter(r, t, m, E, n=n, stride=stride)
    else:
        r = torch.from_numpy(np.ascontiguousarray(reads)).to(d)
        t = torch.from_numpy(np.ascontiguousarray(refs)).to(d)
        pr, pt, acc, cnt = sj.shouji_pack_filter(r, t, m, E)
    assert sj.shouji_wait_failures() == 0
    acc_o, cnt_o = oracle.shouji_batch(reads, refs, E, threads=8)
    got_cnt = cnt[:n].cpu().numpy()
    bad = np.flatnonzero((got_cnt != cnt_o) | (accept_bits(acc, n) != acc_o))
    assert bad.size == 0, "%d pairs differ, first %s" % (bad.size, bad[:10])
    words = acc.cpu().numpy().view(np.uint32)
    if n % 32:
        assert words[-1] >> (n % 32) == 0, "accept bits past n"
    if packing:
        assert (unpack_planes(pr.cpu().numpy(), n, m) == CODE[reads]).all()
        assert (unpack_planes(pt.cpu().numpy(), n, m) == CODE[refs]).all()
        tiles = (n + 1023) // 1024
        assert (unpack_planes(pr.cpu().numpy(), tiles * 1024, m)[n:] == 0).all()


def pairs(n, m, E, seed):
    return synth.pairs(n, m, seed=seed, near=(0, max(E, 1)), far=(E + 1, max(E + 8, m // 4)),
                       far_fraction=0.5)


@pytest.mark.parametrize("E", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_thresholds_m100(E):
    reads, refs = pairs(70_001, 100, E, 100 + E)
    check(reads, refs, 100, E)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7, 31, 33, 64, 65, 150, 250, 255])
def test_lengths(m):
    E = 5 if m > 12 else 1
    reads, refs = pairs(20_000 + m, m, E, 200 + m)
    check(reads, refs, m, E)


@pytest.mark.parametrize("m", list(range(4, 200, 8)) + [8, 16, 24, 40, 56, 72, 96, 128, 136, 160,
                                                         192, 198, 199, 200])
def test_layouts_of_the_fused_producer(m):
    """Every length with an odd number of 4-base words per row (m % 8 == 4,
    the transposition that visits rows in rotated groups of 4), other
    multiples of 4, lengths on either side of the largest that the staging
    rings take (199), each with a ragged last tile."""
    E = 5 if m > 12 else 2
    reads, refs = pairs(3_000 + m, m, E, 400 + m)
    check(reads, refs, m, E)


@pytest.mark.parametrize("m", [1, 4, 12, 33, 36, 64, 65, 100, 124, 128, 131, 132, 133, 140])
@pytest.mark.parametrize("E", [6, 8])
def test_above_the_fused_thresholds(m, E):
    """Thresholds above 5 take the separate launches at every length."""
    reads, refs = pairs(5_000 + m, m, E, 700 + m + E)
    check(reads, refs, m, E)


@pytest.mark.parametrize("n", [1, 1025, 155_649, 311_297, 1_000_001])
def test_above_the_fused_thresholds_ragged_sizes(n):
    reads, refs = pairs(n, 100, 7, 800 + n % 1000)
    check(reads, refs, 100, 7, packing=n < 500_000)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 255, 256, 257, 1023, 1024, 1025, 4097, 155_648,
                               155_649, 311_297])
def test_ragged_sizes(n):
    """Fewer tiles than SMs (some CTAs idle), exactly one tile per CTA, one
    more, and two-plus tiles per CTA with a ragged last tile."""
    reads, refs = pairs(n, 100, 5, n % 1000)
    check(reads, refs, 100, 5)


def test_many_tiles_per_cta():
    """About 26 tiles per CTA: each consumer warp takes several tiles, and
    the producers lap the ring of staging buffers many times."""
    reads, refs = pairs(4_000_003, 100, 5, 7)
    check(reads, refs, 100, 5, packing=False)


@pytest.mark.parametrize("stride_pad,offset,E", [(0, 4, 5), (12, 0, 5), (0, 0, 12), (3, 1, 9)])
def test_fallback_layouts(stride_pad, offset, E):
    """Rows with padding, a base off the 16-byte boundary, or E > 8 take the
    separate launches: same results."""
    reads, refs = pairs(30_001, 100, E, 300 + stride_pad + offset)
    check(reads, refs, 100, E, stride_pad=stride_pad, offset=offset)


def test_zero_pairs_and_bad_arguments():
    d = dev()
    x = torch.zeros(1000, dtype=torch.uint8, device=d)
    lib = sj.load_library()
    buf = torch.zeros(64, dtype=torch.int32, device=d)
    p = buf.data_ptr()
    assert lib.shouji_pack_filter(p, p, 100, 0, 100, 5, p, p, p, None, None) == 0
    assert lib.shouji_pack_filter(p, p, 100, 10, 100, 32, p, p, p, None, None) == 1
    assert lib.shouji_pack_filter(p, p, 99, 10, 100, 5, p, p, p, None, None) == 1
    assert lib.shouji_pack_filter(p, p, 100, 10, 100, 5, p + 4, p, p, None, None) == 1
    assert lib.shouji_pack_filter(None, p, 100, 10, 100, 5, p, p, p, None, None) == 1
    del x


def test_without_counts_on_a_side_stream_with_reused_outputs():
    """Counts left out (NULL), a non-default stream, and the same output
    buffers reused across calls that take the fused kernel (E = 5, 2) and the
    separate launches (E = 7, 12) in turn."""
    d = dev()
    n, m = 50_001, 100
    words = sj.shouji_packed_words(n, m)
    pr = torch.full((words,), -1, dtype=torch.int32, device=d)
    pt = torch.full((words,), -1, dtype=torch.int32, device=d)
    acc = torch.full(((n + 31) // 32,), -1, dtype=torch.int32, device=d)
    side = torch.cuda.Stream(device=d)
    for E in (5, 7, 12, 2):
        reads, refs = pairs(n, m, E, 600 + E)
        r = torch.from_numpy(reads).to(d)
        t = torch.from_numpy(refs).to(d)
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            _, _, _, cnt = sj.shouji_pack_filter(r, t, m, E, packed_reads=pr, packed_refs=pt,
                                                 out_accept=acc, count=False, stream=side)
        side.synchronize()
        assert cnt is None
        assert sj.shouji_wait_failures() == 0
        acc_o, _ = oracle.shouji_batch(reads, refs, E, threads=8)
        assert (accept_bits(acc, n) == acc_o).all()
        assert (unpack_planes(pr.cpu().numpy(), n, m) == CODE[reads]).all()
        assert (unpack_planes(pt.cpu().numpy(), n, m) == CODE[refs]).all()


# ---------------------------------------------------------------- results only
def check_results(reads, refs, m, E):
    """shouji_pack_filter_results: the packed tiles go through per-CTA rings in
    a workspace that starts out as garbage; accept bits and counts against
    the oracle."""
    d = dev()
    n = len(reads)
    r = torch.from_numpy(np.ascontiguousarray(reads)).to(d)
    t = torch.from_numpy(np.ascontiguousarray(refs)).to(d)
    need = sj.shouji_pack_filter_workspace_size(r, t, m, E, n)
    if sj.shouji_pack_filter_fused(r, t, m, E):
        # 12 tiles of 256 m bytes per CTA (one per SM, at most one per tile) and side
        sms = torch.cuda.get_device_properties(d).multi_processor_count
        assert need == 2 * min((n + 1023) // 1024, sms) * 12 * 256 * m
    else:
        assert need == 2 * 4 * sj.shouji_packed_words(n, m)
    ws = torch.full((need,), 0xAB, dtype=torch.uint8, device=d)
    acc, cnt = sj.shouji_pack_filter_results(r, t, m, E, workspace=ws)
    torch.cuda.synchronize()
    assert sj.shouji_wait_failures() == 0
    acc_o, cnt_o = oracle.shouji_batch(reads, refs, E, threads=8)
    got_cnt = cnt[:n].cpu().numpy()
    bad = np.flatnonzero((got_cnt != cnt_o) | (accept_bits(acc, n) != acc_o))
    assert bad.size == 0, "%d pairs differ, first %s" % (bad.size, bad[:10])
    words = acc.cpu().numpy().view(np.uint32)
    if n % 32:
        assert words[-1] >> (n % 32) == 0, "accept bits past n"


@pytest.mark.parametrize("n,m,E", [
    (1, 100, 5), (1025, 100, 5), (155_649, 100, 5),
    (2_500_003, 100, 5),      # about 16 tiles per CTA: every ring entry is reused
    (300_001, 64, 3), (200_000, 37, 5), (100_000, 199, 4), (120_000, 100, 0),
    (50_000, 100, 7),         # above the fused thresholds: the separate launches
])
def test_results_without_packed_outputs(n, m, E):
    reads, refs = pairs(n, m, E, 900 + n % 1000 + m)
    check_results(reads, refs, m, E)


def test_results_workspace_checks():
    d = dev()
    reads, refs = pairs(5000, 100, 5, 5)
    r = torch.from_numpy(reads).to(d)
    t = torch.from_numpy(refs).to(d)
    need = sj.shouji_pack_filter_workspace_size(r, t, 100, 5, 5000)
    ws = torch.empty(need + 64, dtype=torch.uint8, device=d)
    with pytest.raises(sj.ShoujiError):          # one byte short
        sj.shouji_pack_filter_results(r, t, 100, 5, workspace=ws[:need - 1])
    with pytest.raises(sj.ShoujiError):          # off the 16-byte boundary
        sj.shouji_pack_filter_results(r, t, 100, 5, workspace=ws[8:need + 8])
    assert sj.shouji_pack_filter_workspace_size(r, t, 100, 5, 0) == 0
