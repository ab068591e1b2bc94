"""shouji_count (local / glocal counting of Shouji bit-vectors) against the
oracle, pair by pair, including reads shorter than their reference."""
import numpy as np
import pytest

import oracle
import paper_1809_07858_gb300 as sj
from paper_1809_07858_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,E", [(100, 4), (150, 7), (250, 12), (33, 2)])
def test_count_modes_bit_exact(m, E):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(m + E)
    n = 2500
    reads, refs = synth.pairs(n, m, seed=m * 7 + E, near=(0, E), far=(E + 1, m // 3 + 1),
                              far_fraction=0.5)
    # a third of the reads are shorter than their reference: padded with 'N'
    short = rng.random(n) < 0.33
    mp = np.where(short, rng.integers(max(1, m // 2), m + 1, size=n), m)
    for i in np.flatnonzero(short):
        reads[i, mp[i]:] = ord("N")
    pr, nr = sj.shouji_pack(torch.from_numpy(reads).to(dev), m, with_n=True)
    pt, nt = sj.shouji_pack(torch.from_numpy(refs).to(dev), m, with_n=True)
    _, _, vec = sj.shouji_filter(pr, pt, m, n, E, reads_nmask=nr, refs_nmask=nt, vectors=True)
    for mode in range(4):
        acc, cnt = sj.shouji_count(vec, m, n, E, mode)
        torch.cuda.synchronize()
        cnt = cnt[:n].cpu().numpy()
        w = acc.cpu().numpy().view(np.uint32)
        bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:n].astype(bool)
        for i in range(n):
            _, c = oracle.shouji_mode(reads[i, :mp[i]].tobytes(), refs[i].tobytes(), E, mode)
            assert cnt[i] == c, (mode, i, cnt[i], c)
            assert bits[i] == (c <= E)


def test_count_modes_per_pair_thresholds():
    """shouji_count with per-pair thresholds (values above E act as E)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    m, E, n = 100, 8, 3000
    reads, refs = synth.pairs(n, m, seed=808, near=(0, E), far=(E + 1, 30), far_fraction=0.5)
    ep = np.random.default_rng(9).integers(0, E + 3, size=n).astype(np.uint8)
    pr, _ = sj.shouji_pack(torch.from_numpy(reads).to(dev), m)
    pt, _ = sj.shouji_pack(torch.from_numpy(refs).to(dev), m)
    ep_d = torch.from_numpy(ep).to(dev)
    _, _, vec = sj.shouji_filter(pr, pt, m, n, E, E_per_pair=ep_d, vectors=True)
    for mode in range(4):
        acc, cnt = sj.shouji_count(vec, m, n, E, mode, E_per_pair=ep_d)
        torch.cuda.synchronize()
        cnt = cnt[:n].cpu().numpy()
        w = acc.cpu().numpy().view(np.uint32)
        bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:n].astype(bool)
        for i in range(0, n, 7):
            e = min(int(ep[i]), E)
            _, c = oracle.shouji_mode(reads[i].tobytes(), refs[i].tobytes(), e, mode)
            assert cnt[i] == c, (mode, i)
            assert bits[i] == (c <= e), (mode, i)
