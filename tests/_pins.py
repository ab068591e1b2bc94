"""Pins for the Shouji oracle: facts fixed by the paper or by mathematics.

Each pin takes a ``shouji(P, T, E) -> (vector_str, ones)`` callable so the same
checks can run against the oracle and against deliberately broken copies of it
(the mutation test plants mistakes in a copy of the oracle source).
"""
import os
import random

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_kv(name):
    d = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.rstrip("\n")
            if not line or line.startswith("#"):
                continue
            k, v = line.split(" ", 1)
            d[k] = v
    return d


def readings_cases():
    cases = []
    with open(os.path.join(GOLDEN, "readings.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            name, P, T, E, S, ones = line.split()
            cases.append((name, P, T, int(E), S, int(ones)))
    return cases


def pin_fig1(shouji):
    """Fig. 1: zeros exactly on GGTG, AGAG and T; three edits; accepted at E=3."""
    g = read_kv("fig1.txt")
    S, ones = shouji(g["P"], g["T"], int(g["E"]))
    return S == g["shouji"] and ones == int(g["ones"]) and (ones <= int(g["E"])) == bool(int(g["accept"]))


def pin_fig6b(shouji):
    """Fig. 6(b): the printed Shouji bit-vector has 4 ones and ends in 10000100."""
    g = read_kv("fig6b.txt")
    S, ones = shouji(g["P"], g["T"], int(g["E"]))
    p = g["printed_shouji"]
    return ones == p.count("1") and S.endswith(p[-8:]) and len(S) == len(g["P"])


def pin_readings(shouji):
    """The hand-worked tiny pairs of golden/readings.txt."""
    return all(shouji(P, T, E) == (S, ones) for _, P, T, E, S, ones in readings_cases())


def pin_identical(shouji):
    """Identical sequences share one common subsequence of length m: no ones."""
    rng = random.Random(11)
    for m in (1, 2, 3, 4, 5, 17, 64, 100, 150, 250):
        for E in (0, 1, 3, 5):
            P = "".join(rng.choice("ACGT") for _ in range(m))
            if shouji(P, P, E) != ("0" * m, 0):
                return False
    return True


def pin_no_common_base(shouji):
    """P over {A,C}, T over {G,T}: every cell of the map is a mismatch, so the
    Shouji bit-vector keeps its initial all-ones value."""
    rng = random.Random(12)
    for m in (1, 4, 9, 100):
        for E in (0, 2, 5):
            P = "".join(rng.choice("AC") for _ in range(m))
            T = "".join(rng.choice("GT") for _ in range(m))
            if shouji(P, T, E) != ("1" * m, m):
                return False
    return True


def pin_hamming_at_E0(shouji):
    """E = 0 leaves only the main diagonal: each window's choice is the main
    segment, every main-diagonal zero is written by its own window and no one is
    ever overwritten by a one, so the vector is the per-position mismatch string
    and the count is the Hamming distance."""
    rng = random.Random(13)
    for _ in range(200):
        m = rng.randint(1, 40)
        P = "".join(rng.choice("ACGT") for _ in range(m))
        T = "".join(rng.choice("ACGT") if rng.random() < 0.5 else P[i] for i in range(m))
        want = "".join("0" if a == b else "1" for a, b in zip(P, T))
        if shouji(P, T, 0) != (want, want.count("1")):
            return False
    return True


def pin_shifted_copies(shouji):
    """Closed forms.  P over {A,C}; T = G^d + P[:m-d] (a copy of P shifted right by
    d, the gap filled with a base P never has).  Columns < d hold G and match
    nothing; every column >= d matches on upper diagonal d, so each window from
    column d on finds 0000 and the windows just before it find the unique
    all-mismatch-then-match segment of diagonal d.  The vector is 1^d 0^(m-d)
    when d <= E.  Symmetrically T = P[d:] + G^d gives 0^(m-d) 1^d (lower
    diagonal d): the windows that reach past column m-d never beat the zeros
    already written, because the update needs strictly more zeros."""
    rng = random.Random(14)
    for m in (8, 33, 100):
        for E in (1, 3, 5):
            for d in range(1, E + 1):
                P = "".join(rng.choice("AC") for _ in range(m))
                up = shouji(P, "G" * d + P[: m - d], E)
                lo = shouji(P, P[d:] + "G" * d, E)
                if up != ("1" * d + "0" * (m - d), d):
                    return False
                if lo != ("0" * (m - d) + "1" * d, d):
                    return False
    return True


def pin_zero_needs_a_match(shouji):
    """Every bit of the Shouji bit-vector is a copy of some diagonal's bit or the
    initial 1.  So S[c] = 0 needs some P[c-d] == T[c] with |d| <= E, checked here by
    comparing characters directly."""
    rng = random.Random(15)
    for _ in range(300):
        m = rng.randint(1, 30)
        E = rng.randint(0, 4)
        P = "".join(rng.choice("ACGTN") for _ in range(m))
        T = "".join(rng.choice("ACGTN") for _ in range(m))
        S, ones = shouji(P, T, E)
        if len(S) != m or ones != S.count("1"):
            return False
        for c in range(m):
            match = any(0 <= c - d < m and P[c - d] == T[c] and T[c] != "N"
                        for d in range(-E, E + 1))
            if S[c] == "0" and not match:
                return False
    return True


def pin_large_E_accepts(shouji):
    """With E >= m the count (at most m) can never exceed E."""
    rng = random.Random(16)
    for m in (1, 3, 7, 12):
        P = "".join(rng.choice("ACGT") for _ in range(m))
        T = "".join(rng.choice("ACGT") for _ in range(m))
        S, ones = shouji(P, T, m)
        if not (ones <= m):
            return False
    return True


def pin_N_matches_nothing(shouji):
    """Reading R8: an 'N' is a mismatch against every base and against 'N'."""
    return (shouji("NNNN", "NNNN", 2) == ("1111", 4)
            and shouji("ANAA", "ANAA", 0) == ("0100", 1))


ALL_PINS = [pin_fig1, pin_fig6b, pin_readings, pin_identical, pin_no_common_base,
            pin_hamming_at_E0, pin_shifted_copies, pin_zero_needs_a_match,
            pin_large_E_accepts, pin_N_matches_nothing]
