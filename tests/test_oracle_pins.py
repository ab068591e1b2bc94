"""The CPU oracle against what the paper and mathematics fix (no GPU needed)."""
import itertools
import random

import numpy as np
import pytest

import oracle
from _pins import ALL_PINS, read_kv


def oracle_shouji(P, T, E):
    S, ones, _ = oracle.shouji(P, T, E)
    return "".join(map(str, S)), ones


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(pin):
    assert pin(oracle_shouji), pin.__doc__


def _printed_rows(g):
    rows = {}
    for k in range(1, 5):
        rows[+k] = g["upper%d" % k]
        rows[-k] = g["lower%d" % k]
    return rows


def _oracle_rows(P, T, E, swap=False):
    if swap:
        P, T = T, P
    m = len(T)
    mp = oracle.neighborhood_map(P, T, E)
    rows = {}
    for d in range(-E, E + 1):
        if d == 0:
            continue
        rows[d] = "".join("-" if not (0 <= c - d < m) else str(mp[d + E, c])
                          for c in range(m))
    return rows


@pytest.mark.parametrize("fig", ["fig6a.txt", "fig6b.txt"])
def test_map_orientation_matches_printed_diagonals(fig):
    """Fig. 6 prints the 8 off-main diagonals of two pairs (damaged by text
    extraction: characters dropped and inserted).  With upper diagonal d
    comparing P[c-d] to T[c] (reading R1), the oracle's rows sit much closer to
    the printed rows, in edit distance, than with P and T exchanged; and every
    upper row starts with d out-of-band dashes as printed."""
    g = read_kv(fig)
    printed = _printed_rows(g)
    ours = _oracle_rows(g["P"], g["T"], 4)
    swapped = _oracle_rows(g["P"], g["T"], 4, swap=True)
    d_ours = sum(oracle.edit_distance(ours[d], printed[d]) for d in printed)
    d_swap = sum(oracle.edit_distance(swapped[d], printed[d]) for d in printed)
    assert d_ours < 0.6 * d_swap, (d_ours, d_swap)
    for k in range(1, 5):
        assert printed[k].startswith("-" * k) and ours[k].startswith("-" * k)
        assert printed[-k].endswith("-" * k) and ours[-k].endswith("-" * k)
    # The first columns, before the first dropped character, agree exactly.
    main = "".join(str(x) for x in oracle.neighborhood_map(g["P"], g["T"], 4)[4])
    assert main[:20] == g["main"][:20]


def test_map_cells_follow_eq1():
    """Eq. 1 cell by cell on random pairs, against a direct character compare."""
    rng = random.Random(5)
    for _ in range(100):
        m = rng.randint(1, 20)
        E = rng.randint(0, 5)
        P = "".join(rng.choice("ACGTN") for _ in range(m))
        T = "".join(rng.choice("ACGTN") for _ in range(m))
        mp = oracle.neighborhood_map(P, T, E)
        for d in range(-E, E + 1):
            for c in range(m):
                i = c - d
                if 0 <= i < m:
                    want = 0 if (P[i] == T[c] and P[i] != "N") else 1
                else:
                    want = 1
                assert mp[d + E, c] == want


def test_fig6a_regression_parity_unpinned():
    """Fig. 6(a): parity unpinned.  The printed vector is damaged (89 of 100
    characters) and shows 3 ones; under the readings taken here the oracle finds
    4 ones at columns 19, 22, 23 and 93.  Kept as a regression value only."""
    g = read_kv("fig6a.txt")
    S, ones = oracle_shouji(g["P"], g["T"], 4)
    assert ones == 4
    assert [i for i, x in enumerate(S) if x == "1"] == [19, 22, 23, 93]


def _edit_distance_brute(a, b):
    """Levenshtein by its recursive definition (no table), for tiny inputs."""
    if not a:
        return len(b)
    if not b:
        return len(a)
    return min(_edit_distance_brute(a[1:], b) + 1,
               _edit_distance_brute(a, b[1:]) + 1,
               _edit_distance_brute(a[1:], b[1:]) + (a[0] != b[0]))


def test_edit_distance_brute_force():
    rng = random.Random(6)
    for _ in range(300):
        a = "".join(rng.choice("ACG") for _ in range(rng.randint(0, 6)))
        b = "".join(rng.choice("ACG") for _ in range(rng.randint(0, 6)))
        assert oracle.edit_distance(a, b) == _edit_distance_brute(a, b)


def test_edit_distance_identities():
    assert oracle.edit_distance("ACGT", "ACGT") == 0
    assert oracle.edit_distance("", "ACGT") == 4
    assert oracle.edit_distance("ACGTACGT", "ACCTACGT") == 1
    assert oracle.edit_distance("ACGTACGT", "CGTACGTA") == 2   # one deletion + one insertion
    assert oracle.edit_distance("kitten", "sitting") == 3


def test_batch_matches_single_pair_calls():
    rng = np.random.default_rng(7)
    reads = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=(300, 37))
    refs = reads.copy()
    flip = rng.random(refs.shape) < 0.1
    refs[flip] = rng.choice(np.frombuffer(b"ACGTN", np.uint8), size=int(flip.sum()))
    acc1, cnt1 = oracle.shouji_batch(reads, refs, 3, threads=1)
    acc4, cnt4 = oracle.shouji_batch(reads, refs, 3, threads=4)
    assert (acc1 == acc4).all() and (cnt1 == cnt4).all()
    for i in range(0, 300, 17):
        S, ones, acc = oracle.shouji(reads[i], refs[i], 3)
        assert ones == cnt1[i] and acc == acc1[i]
    Ep = rng.integers(0, 6, size=300).astype(np.uint8)
    accp, cntp = oracle.shouji_batch(reads, refs, 0, E_per_pair=Ep)
    for i in range(0, 300, 13):
        S, ones, acc = oracle.shouji(reads[i], refs[i], int(Ep[i]))
        assert ones == cntp[i] and acc == accp[i]


def test_false_accept_reject_report_tiny_brute_force(capsys):
    """All pairs over {A,C,G,T}^4 at E = 0..2, against exact global edit distance.
    The paper reports 0 false rejects on its real datasets (Sec. 3.2); that is an
    empirical claim, not a theorem, so the counts are reported, not asserted.  At
    E = 0 the filter is exact (it is the Hamming test; Hamming 0 <=> ED 0)."""
    seqs = ["".join(t) for t in itertools.product("ACGT", repeat=4)]
    reads = np.array([[ord(c) for c in a] for a in seqs for _ in seqs], np.uint8)
    refs = np.array([[ord(c) for c in b] for _ in seqs for b in seqs], np.uint8)
    ed = np.array([oracle.edit_distance(a, b) for a in seqs for b in seqs])
    for E in range(3):
        acc, _ = oracle.shouji_batch(reads, refs, E, threads=4)
        fa = int((acc & (ed > E)).sum())
        fr = int((~acc & (ed <= E)).sum())
        print("m=4 E=%d pairs=%d similar=%d FA=%d FR=%d" % (E, len(ed), int((ed <= E).sum()), fa, fr))
        if E == 0:
            assert fa == 0 and fr == 0


# ------------------------------------------------------------ count modes (N3)
def test_count_modes_hand_worked():
    """Sec. 2.2.3 / Supp. Sec. 8: local counting leaves out the runs of ones at
    both ends of the Shouji bit-vector, glocal the run at one end.  Worked by
    hand: 11010011 has ones at 0,1,3,6,7; first zero 2, last zero 5."""
    S = [1, 1, 0, 1, 0, 0, 1, 1]
    assert oracle.count_mode(S, oracle.GLOBAL) == 5
    assert oracle.count_mode(S, oracle.LOCAL) == 1          # only column 3
    assert oracle.count_mode(S, oracle.GLOCAL_START) == 3   # columns 3, 6, 7
    assert oracle.count_mode(S, oracle.GLOCAL_END) == 3     # columns 0, 1, 3
    for mode in range(4):
        assert oracle.count_mode([1, 1, 1, 1], mode) == 4   # reading R10: no zero counts m
        assert oracle.count_mode([0, 0, 0], mode) == 0
        assert oracle.count_mode([0, 1, 1, 0], mode) == 2
    assert [oracle.count_mode([1, 0, 0, 0], k) for k in range(4)] == [1, 0, 0, 1]


def test_short_pattern_is_out_of_band_past_its_end():
    """A pattern shorter than the text reads as out of the band past its end
    (the dashes of Fig. 6(c)); that is the same as padding it with 'N', which
    matches nothing (R8) -- the equivalence the GPU path relies on."""
    rng = random.Random(21)
    for _ in range(200):
        m = rng.randint(4, 60)
        mp = rng.randint(0, m)
        E = rng.randint(0, 5)
        T = "".join(rng.choice("ACGT") for _ in range(m))
        P = "".join(rng.choice("ACGT") for _ in range(mp))
        for mode in range(4):
            S1, c1 = oracle.shouji_mode(P, T, E, mode)
            S2, c2 = oracle.shouji_mode(P + "N" * (m - mp), T, E, mode)
            assert (S1 == S2).all() and c1 == c2
        S3, ones, _ = oracle.shouji(P + "N" * (m - mp), T, E)
        assert (S3 == S1).all() and ones == oracle.count_mode(S1, oracle.GLOBAL)


def test_fig6c_local_count_parity_unpinned():
    """Fig. 6(c) (68-base read, 100-base reference, E = 4, local): the figure
    states 2 edits; under the readings taken here (Algorithm 1's strict
    comparisons, lower before upper) the local count is 3, with ones at
    columns 1, 20 and 28 inside the end runs.  Kept as a regression value."""
    lines = [l for l in open(__import__("os").path.join(
        __import__("os").path.dirname(__file__), "golden", "fig6c.txt")) if not l.startswith("#")]
    d = dict(l.rstrip("\n").split(" ", 1) for l in lines if l.strip())
    S, local = oracle.shouji_mode(d["P"], d["T"], int(d["E"]), oracle.LOCAL)
    assert local == 3
    assert [i for i in range(len(S)) if S[i]][:3] == [1, 20, 28]
