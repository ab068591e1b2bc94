"""The one-call helpers of the binding, filter_pairs and magnet_pairs, against
the oracle: without 'N' (filter_pairs then takes shouji_pack_filter), with 'N'
bases (N masks), and with per-pair thresholds."""
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


@pytest.mark.parametrize("with_N", [False, True])
@pytest.mark.parametrize("m,E", [(100, 5), (100, 3), (150, 7), (33, 2)])
def test_filter_pairs_and_magnet_pairs(m, E, with_N):
    d = dev()
    n = 12_345
    reads, refs = synth.pairs(n, m, seed=900 + m + E, near=(0, E), far=(E + 1, E + 12),
                              far_fraction=0.5)
    if with_N:
        rng = np.random.default_rng(m + E)
        reads[rng.random(reads.shape) < 0.01] = ord("N")
        refs[rng.random(refs.shape) < 0.01] = ord("N")
    r, t = torch.from_numpy(reads).to(d), torch.from_numpy(refs).to(d)
    acc, cnt = sj.filter_pairs(r, t, E)
    acc_o, cnt_o = oracle.shouji_batch(reads, refs, E, threads=8)
    assert (acc.cpu().numpy() == acc_o).all()
    assert (cnt.cpu().numpy() == cnt_o).all()
    macc, mcnt = sj.magnet_pairs(r, t, E)
    macc_o, mcnt_o = oracle.shouji_batch(reads, refs, E, threads=8, magnet=True)
    assert (macc.cpu().numpy() == macc_o).all()
    assert (mcnt.cpu().numpy() == mcnt_o).all()
    assert sj.shouji_wait_failures() == 0


def test_filter_pairs_per_pair_thresholds():
    d = dev()
    n, m, E = 9_999, 100, 6
    reads, refs = synth.pairs(n, m, seed=77, near=(0, E), far=(E + 1, 20), far_fraction=0.5)
    ep = np.random.default_rng(3).integers(0, E + 1, n).astype(np.uint8)
    acc, cnt = sj.filter_pairs(torch.from_numpy(reads).to(d), torch.from_numpy(refs).to(d), E,
                               E_per_pair=torch.from_numpy(ep).to(d))
    acc_o, cnt_o = oracle.shouji_batch(reads, refs, E, E_per_pair=ep, threads=8)
    assert (acc.cpu().numpy() == acc_o).all()
    assert (cnt.cpu().numpy() == cnt_o).all()
