"""The serving loop: requests admitted while others run on the GPU give the
same results as when each runs alone (bit-exact: integer path) and overlap on
the device; admission is by device memory (a request holds memory in
proportion to its size, never more than the budget in total); host waits
honour their deadlines; requests may name their reference segments by offset
into a resident reference text and may leave their results on the device."""
import threading

import numpy as np
import pytest

import oracle
import paper_1809_07858_gb300 as sj
from paper_1809_07858_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def make_request(n, seed, stride=256, pinned=False):
    lens, Es = synth.mixed_shape(n, seed=seed)
    reads, refs = synth.pairs(n, 250, seed=seed, near=(0, 6), far=(7, 40), far_fraction=0.5,
                              lengths=lens, stride=stride)
    acc = np.zeros((n + 31) // 32, np.uint32)
    cnt = np.zeros(n, np.uint8)
    if pinned:  # page-locked host buffers, viewed as numpy arrays
        def pin(a):
            t = torch.empty(max(1, a.nbytes), dtype=torch.uint8, pin_memory=True)
            v = t.numpy()[:a.nbytes].view(a.dtype).reshape(a.shape)
            v[...] = a
            return v
        reads, refs, lens, Es, acc, cnt = (pin(x) for x in (reads, refs, lens, Es, acc, cnt))
    return reads, refs, lens, Es, acc, cnt


def oracle_request(r, t, L, E):
    n = len(L)
    acc_o = np.zeros(n, bool)
    cnt_o = np.zeros(n, np.uint8)
    for m in np.unique(L):
        idx = np.flatnonzero(L == m)
        x, y = oracle.shouji_batch(r[idx, :m], t[idx, :m], 0, E_per_pair=E[idx], threads=8)
        acc_o[idx], cnt_o[idx] = x, y
    return acc_o, cnt_o


def bits_of(words, n):
    return ((words[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:n].astype(bool)


def union_length(intervals):
    total, end = 0.0, -1.0
    for a, b in sorted(intervals):
        if a > end:
            total += b - a
            end = b
        elif b > end:
            total += b - end
            end = b
    return total


def test_each_result_is_the_same_alone_and_in_the_mix():
    need_gpu()
    sizes = [1000, 250_000, 3_000, 120_000, 47_777, 999, 200_000, 64_000, 5_000, 150_000]
    # pinned host buffers (the copies of one request overlap the others' work)
    # for all but the last two, which take the staged path of pageable memory
    reqs = [make_request(n, seed=100 + i, pinned=i < 8) for i, n in enumerate(sizes)]
    srv = sj.Server(250_000, 250, 2, 12, max_stride=256, max_slots=6)
    assert srv.info()[0] == 0 and srv.info()[1] > 0   # workers are made on demand
    # alone: one at a time (this also makes the workers of every size class)
    alone = []
    for r, t, L, E, a, c in reqs:
        srv.wait(srv.submit(r, t, L, E, a, c), timeout=120)
        alone.append((a.copy(), c.copy()))
        a[:] = 0
        c[:] = 0
    # in the mix: all submitted at once from two threads (twice: the first
    # mix may still make workers for requests that now run side by side)
    ids = [None] * len(reqs)

    def submit(idx):
        for i in idx:
            r, t, L, E, a, c = reqs[i]
            ids[i] = srv.submit(r, t, L, E, a, c)

    for _ in range(2):
        made = srv.stats()["workers_made"]
        th = [threading.Thread(target=submit, args=(range(k, len(reqs), 2),)) for k in (0, 1)]
        [t.start() for t in th]
        [t.join() for t in th]
        timed = [srv.wait_timed(i, timeout=120) for i in ids]
    assert all(lat > 0 and 0 <= g0 < g1 for lat, g0, g1 in timed)
    st = srv.stats()
    assert 2 <= st["peak_busy_workers"] <= 6 and st["workers"] <= 6
    assert st["peak_used_bytes"] <= st["budget_bytes"]
    assert st["workers_made"] - made <= 2   # the second mix ran (almost) on workers it found
    # their work overlapped on the device: the summed GPU time of the requests
    # exceeds the time during which any of them was on the GPU
    spans = [(g0, g1) for _, g0, g1 in timed]
    assert sum(b - a for a, b in spans) > 1.2 * union_length(spans)
    for k, (r, t, L, E, a, c) in enumerate(reqs):
        assert (a == alone[k][0]).all() and (c == alone[k][1]).all(), "request %d differs" % k
    srv.close()
    # and the small ones against the oracle
    for k in (0, 5):
        r, t, L, E, a, c = reqs[k]
        acc_o, cnt_o = oracle_request(r, t, L, E)
        assert (c == cnt_o).all() and (bits_of(a, len(L)) == acc_o).all()


def test_admission_by_memory():
    need_gpu()
    big = sj.Server(400_000, 250, 2, 12, max_stride=256)
    _, per_big = big.info()
    big.close()
    # a budget below one worker for the largest request admits nothing
    with pytest.raises(sj.ShoujiError) as err:
        sj.Server(400_000, 250, 2, 12, max_stride=256, memory_budget=per_big // 2)
    assert err.value.status == 2
    budget = int(2.5 * per_big)
    srv = sj.Server(400_000, 250, 2, 12, max_stride=256, memory_budget=budget)
    # largest requests: at most two fit in the budget at once
    bigs = [make_request(400_000, seed=40 + k) for k in range(4)]
    ids = [srv.submit(*q) for q in bigs]
    rid = ids[-1]
    with pytest.raises(sj.ShoujiError) as err:
        srv.wait(rid, timeout=0.0)          # not done yet: the deadline passes
    assert err.value.status == 4
    for i in ids:
        assert srv.wait(i, timeout=120) > 0  # the timed-out one can be waited for again
    st = srv.stats()
    assert st["peak_busy_workers"] <= 2 and st["peak_used_bytes"] <= budget
    # small requests hold little memory: in the same budget many run at once
    small = [make_request(20_000, seed=60 + k) for k in range(24)]
    ids = [srv.submit(*q) for q in small]
    for i in ids:
        srv.wait(i, timeout=120)
    st = srv.stats()
    assert st["peak_busy_workers"] > 2, st
    assert st["peak_used_bytes"] <= budget
    for (r, t, L, E, a, c) in small[:2]:
        acc_o, cnt_o = oracle_request(r, t, L, E)
        assert (c == cnt_o).all() and (bits_of(a, len(L)) == acc_o).all()
    srv.close()


def test_resident_reference_and_device_results():
    """Pairs whose reference segments are read from a resident text by offset
    give the results of the same pairs sent as rows; results left on the
    device equal those copied back."""
    need_gpu()
    d = torch.device("cuda:0")
    n = 60_000
    reads, refs, lens, Es, acc, cnt = make_request(n, seed=77)
    # a reference text holding every segment at a scattered offset
    rng = np.random.default_rng(5)
    gaps = rng.integers(0, 40, size=n)
    offs = np.zeros(n, np.uint64)
    pos = 0
    for i in range(n):
        pos += int(gaps[i])
        offs[i] = pos
        pos += int(lens[i])
    text = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=pos + 64)
    for i in range(n):
        o, L = int(offs[i]), int(lens[i])
        text[o:o + L] = refs[i, :L]
    srv = sj.Server(100_000, 250, 2, 12, max_stride=256)
    ref_id = srv.add_reference(text)
    assert srv.stats()["reference_bytes"] == text.nbytes
    srv.wait(srv.submit(reads, refs, lens, Es, acc, cnt), timeout=120)
    acc2, cnt2 = np.zeros_like(acc), np.zeros_like(cnt)
    srv.wait(srv.submit_at(reads, ref_id, offs, lens, Es, acc2, cnt2), timeout=120)
    assert (acc2 == acc).all() and (cnt2 == cnt).all()
    dacc = torch.zeros(len(acc), dtype=torch.int32, device=d)
    dcnt = torch.zeros(n, dtype=torch.uint8, device=d)
    srv.wait(srv.submit_at(reads, ref_id, offs, lens, Es, dacc, dcnt, device_results=True),
             timeout=120)
    assert (dacc.cpu().numpy().view(np.uint32) == acc).all()
    assert (dcnt.cpu().numpy() == cnt).all()
    # a segment past the end of the text is rejected on the host
    bad = offs.copy()
    bad[17] = np.uint64(pos + 64 - int(lens[17]) + 1)
    with pytest.raises(sj.ShoujiError):
        srv.submit_at(reads, ref_id, bad, lens, Es, acc2, cnt2)
    srv.close()
    acc_o, cnt_o = oracle_request(reads[:3000], refs[:3000], lens[:3000], Es[:3000])
    assert (cnt[:3000] == cnt_o).all() and (bits_of(acc, n)[:3000] == acc_o).all()


def test_submit_rejects_bad_requests():
    need_gpu()
    srv = sj.Server(1000, 100, 2, 12, max_stride=128, max_slots=1)
    r, t, L, E, a, c = make_request(10, seed=3, stride=256)
    with pytest.raises(sj.ShoujiError):
        srv.submit(r, t, L, E, a, c)        # stride 256 > max_stride 128
    with pytest.raises(sj.ShoujiError):
        srv.submit_at(r[:, :128].copy(), 0, np.zeros(10, np.uint64), L, E, a, c)  # no reference
    srv.close()
