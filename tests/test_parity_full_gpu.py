"""Parity at full workload sizes, in the launch sequence bench.py times.

30M pairs at m=100 (sweep recipe, E = 0, 5, 10) and 10M pairs at m=150 / 250
with 'N' bases: every pair is filtered on the GPU and recomputed by the oracle
(one pair at a time, on all host cores), and the two must match bit for bit on
every pair; properties that hold for every pair are checked as well.  Without
N masks the fused pack + filter (shouji_pack_filter) is checked the same way,
and its packed words against shouji_pack's, and so is the benchmark's step
(shouji_pack_filter_results: the same kernel with the packed tiles in per-CTA
rings instead of packed outputs).
"""
import os
import numpy as np
import pytest

import oracle
import paper_1809_07858_gb300 as sj
from paper_1809_07858_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

THREADS = max(1, os.cpu_count() or 1)


def run_full(reads, refs, m, E, with_n):
    """The separate launches (pack, pack, filter, compact) and, without N
    masks, the fused pack + filter on the same rows."""
    dev = torch.device("cuda:0")
    n = len(reads)
    r = torch.from_numpy(reads).to(dev)
    t = torch.from_numpy(refs).to(dev)
    pr, nr = sj.shouji_pack(r, m, with_n=with_n)
    pt, nt = sj.shouji_pack(t, m, with_n=with_n)
    fused = results = None
    if not with_n:
        fr, ft, facc, fcnt = sj.shouji_pack_filter(r, t, m, E)
        torch.cuda.synchronize()
        same_packing = bool(torch.equal(fr, pr)) and bool(torch.equal(ft, pt))
        fused = (sj.accept_to_bool(facc, n).cpu().numpy(), fcnt[:n].cpu().numpy(), same_packing)
        del fr, ft, facc, fcnt
        # the same without packed outputs (per-CTA rings in a workspace)
        racc, rcnt = sj.shouji_pack_filter_results(r, t, m, E)
        torch.cuda.synchronize()
        results = (sj.accept_to_bool(racc, n).cpu().numpy(), rcnt[:n].cpu().numpy())
        del racc, rcnt
    del r, t
    acc, cnt, _ = sj.shouji_filter(pr, pt, m, n, E, reads_nmask=nr, refs_nmask=nt)
    idx, n_acc = sj.shouji_compact(acc, n)
    torch.cuda.synchronize()
    accept = sj.accept_to_bool(acc, n).cpu().numpy()
    count = cnt[:n].cpu().numpy()
    k = int(n_acc.item())
    survivors = idx[:k].cpu().numpy()
    assert sj.shouji_wait_failures() == 0
    return accept, count, survivors, fused, results


def check(reads, refs, m, E, with_n):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = len(reads)
    accept, count, survivors, fused, results = run_full(reads, refs, m, E, with_n)
    # properties over every pair
    assert (count <= m).all()
    assert (accept == (count <= E)).all()
    assert len(survivors) == int(accept.sum())
    assert (np.diff(survivors.astype(np.int64)) > 0).all()
    assert accept[survivors].all()
    # the oracle on every pair
    acc_o, cnt_o = oracle.shouji_batch(reads, refs, E, threads=THREADS)
    bad = np.flatnonzero((count != cnt_o) | (accept != acc_o))
    assert bad.size == 0, "%d pairs differ, first %s" % (bad.size, bad[:10])
    if fused is not None:
        f_acc, f_cnt, same_packing = fused
        assert same_packing, "fused pack + filter wrote other packed words"
        bad = np.flatnonzero((f_cnt != cnt_o) | (f_acc != acc_o))
        assert bad.size == 0, "fused: %d pairs differ, first %s" % (bad.size, bad[:10])
    if results is not None:
        r_acc, r_cnt = results
        bad = np.flatnonzero((r_cnt != cnt_o) | (r_acc != acc_o))
        assert bad.size == 0, "results only: %d pairs differ, first %s" % (bad.size, bad[:10])


@pytest.mark.parametrize("E", [0, 5, 10])
def test_sweep_30M(E, host_buffers):
    reads, refs = synth.workload("sweep", 30_000_000, E=E,
                                 out=host_buffers.views(30_000_000, 100))
    check(reads, refs, 100, E, False)


@pytest.mark.parametrize("m,E", [(150, 15), (250, 15)])
def test_long_10M_with_N(m, E, host_buffers):
    reads, refs = synth.workload("long", 10_000_000, m=m, E=E,
                                 out=host_buffers.views(10_000_000, m))
    check(reads, refs, m, E, True)
