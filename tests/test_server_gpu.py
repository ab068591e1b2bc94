"""The serving loop: requests admitted while others run on the GPU give the
same results as when each runs alone (bit-exact: integer path), host waits
honour their deadlines, and admission is bounded by the memory budget."""
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


def make_request(n, seed, stride=256):
    lens, Es = synth.mixed_shape(n, seed=seed)
    reads, refs = synth.pairs(n, 250, seed=seed, near=(0, 6), far=(7, 40), far_fraction=0.5,
                              lengths=lens, stride=stride)
    acc = np.zeros((n + 31) // 32, np.uint32)
    cnt = np.zeros(n, np.uint8)
    return reads, refs, lens, Es, acc, cnt


def test_each_result_is_the_same_alone_and_in_the_mix():
    need_gpu()
    sizes = [1000, 250_000, 3_000, 120_000, 47_777, 999, 200_000, 64_000, 5_000, 150_000]
    reqs = [make_request(n, seed=100 + i) for i, n in enumerate(sizes)]
    srv = sj.Server(250_000, 250, 2, 12, max_stride=256, max_slots=4)
    slots, per_slot = srv.info()
    assert slots == 4 and per_slot > 0
    # in the mix: all submitted at once from two threads
    ids = [None] * len(reqs)

    def submit(idx):
        for i in idx:
            r, t, L, E, a, c = reqs[i]
            ids[i] = srv.submit(r, t, L, E, a, c)

    th = [threading.Thread(target=submit, args=(range(k, len(reqs), 2),)) for k in (0, 1)]
    [t.start() for t in th]
    [t.join() for t in th]
    lat = [srv.wait(i, timeout=120) for i in ids]
    assert all(x > 0 for x in lat)
    mixed = [(a.copy(), c.copy()) for (_, _, _, _, a, c) in reqs]
    # alone: one at a time
    for k, (r, t, L, E, a, c) in enumerate(reqs):
        a[:] = 0
        c[:] = 0
        srv.wait(srv.submit(r, t, L, E, a, c), timeout=120)
        assert (a == mixed[k][0]).all() and (c == mixed[k][1]).all(), "request %d differs" % k
    srv.close()
    # and the small ones against the oracle
    for k in (0, 5):
        r, t, L, E, a, c = reqs[k]
        n = len(L)
        acc_o = np.zeros(n, bool)
        cnt_o = np.zeros(n, np.uint8)
        for m in np.unique(L):
            idx = np.flatnonzero(L == m)
            x, y = oracle.shouji_batch(r[idx, :m], t[idx, :m], 0, E_per_pair=E[idx])
            acc_o[idx], cnt_o[idx] = x, y
        bits = ((a[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:n].astype(bool)
        assert (c == cnt_o).all() and (bits == acc_o).all()


def test_wait_deadline_and_memory_bounded_slots():
    need_gpu()
    r, t, L, E, a, c = make_request(400_000, seed=7)
    one = sj.Server(400_000, 250, 2, 12, max_stride=256, max_slots=8)
    _, per_slot = one.info()
    one.close()
    # a budget below one slot admits nothing: SHOUJI_ENOMEM, and nothing is kept
    with pytest.raises(sj.ShoujiError) as err:
        sj.Server(400_000, 250, 2, 12, max_stride=256, max_slots=8,
                  memory_budget=per_slot // 2)
    assert err.value.status == 2
    # a budget for two slots gives two slots
    srv = sj.Server(400_000, 250, 2, 12, max_stride=256, max_slots=8,
                    memory_budget=int(2.5 * per_slot))
    assert srv.info()[0] == 2
    rid = srv.submit(r, t, L, E, a, c)
    with pytest.raises(sj.ShoujiError) as err:
        srv.wait(rid, timeout=0.0)          # not done yet: the deadline passes
    assert err.value.status == 4
    assert srv.wait(rid, timeout=120) > 0   # the same request can be waited for again
    many = [make_request(30_000, seed=20 + k) for k in range(6)]
    ids = [srv.submit(*q) for q in many]
    for i in ids:
        srv.wait(i, timeout=120)
    srv.close()


def test_submit_rejects_bad_requests():
    need_gpu()
    srv = sj.Server(1000, 100, 2, 12, max_stride=128, max_slots=1)
    r, t, L, E, a, c = make_request(10, seed=3, stride=256)
    with pytest.raises(sj.ShoujiError):
        srv.submit(r, t, L, E, a, c)        # stride 256 > max_stride 128
    srv.close()
