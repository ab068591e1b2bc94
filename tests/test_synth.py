"""The seeded input generator: deterministic, sub-range stable, recipe-shaped."""
import numpy as np

import oracle
from paper_1809_07858_gb300 import synth


def test_subrange_regenerates_identical_bytes():
    r, t = synth.workload("sweep", 2000, E=5)
    r2, t2 = synth.workload("sweep", 500, E=5, first=1200, threads=3)
    assert (r[1200:1700] == r2).all() and (t[1200:1700] == t2).all()
    r3, t3 = synth.workload("sweep", 2000, E=5, threads=1)
    assert (r == r3).all() and (t == t3).all()


def test_alphabet_and_shape():
    r, t = synth.workload("small")
    assert r.shape == (10_000, 100) and t.shape == (10_000, 100)
    assert set(np.unique(r)) <= set(b"ACGT") and set(np.unique(t)) <= set(b"ACGT")
    rl, tl = synth.workload("long", 20_000, m=150, E=7)
    frac_n = (rl == ord("N")).mean()
    assert 0.0005 < frac_n < 0.002
    assert set(np.unique(tl)) <= set(b"ACGTN")


def test_edit_counts_bound_edit_distance():
    """Each ref is the read after k edits, then trimmed/padded: the global edit
    distance is at most k plus the length repair (|insertions - deletions|)."""
    r, t, kind, k = synth.pairs(400, 60, seed=9, near=(0, 3), far=(4, 12),
                                far_fraction=0.5, with_meta=True)
    assert 0.35 < kind.mean() < 0.65
    assert (k[kind == 0] <= 3).all() and (k[kind == 1] >= 4).all()
    for i in range(400):
        ed = oracle.edit_distance(r[i].tobytes(), t[i].tobytes())
        assert ed <= 2 * int(k[i])


def test_mixed_shape_distribution():
    lengths, Es = synth.mixed_shape(100_000, seed=4)
    frac = [(lengths == L).mean() for L in (100, 150, 250)]
    assert abs(frac[0] - 0.4) < 0.01 and abs(frac[1] - 0.4) < 0.01 and abs(frac[2] - 0.2) < 0.01
    assert Es.min() == 2 and Es.max() == 12
