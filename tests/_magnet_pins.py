"""Pins for the MAGNET oracle (Supplementary Sec. 7, Algorithms 3 and 4).

Each pin takes a ``magnet(P, T, E, mode) -> (vector_str, count)`` callable so the
same checks run against the oracle and against copies of it with a planted
mistake.
"""
import os
import random

from _pins import GOLDEN, read_kv

LOCAL = 1


def magnet_readings_cases():
    cases = []
    with open(os.path.join(GOLDEN, "magnet_readings.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            name, P, T, E, V, ones = line.split()
            cases.append((name, P, T, int(E), V, int(ones)))
    return cases


def pin_fig6ab_counts(magnet):
    """Fig. 6(a),(b): the printed MAGNET vectors hold 4 ones each.  The printed
    vectors lost characters in extraction; for (a) the gaps between its first
    two and its last two ones (2 and 4) survived."""
    ok = True
    for fig in ("fig6a.txt", "fig6b.txt"):
        g = read_kv(fig)
        V, c = magnet(g["P"], g["T"], int(g["E"]), 0)
        ok &= c == 4
        if fig == "fig6a.txt":
            ones = [i for i, x in enumerate(V) if x == "1"]
            ok &= len(ones) == 4 and ones[1] - ones[0] == 2 and ones[3] - ones[2] == 4
    return ok


def pin_hand_cases(magnet):
    """Tiny pairs traced by hand, one per reading."""
    return all(magnet(P, T, E, 0) == (V, ones)
               for _, P, T, E, V, ones in magnet_readings_cases())


def pin_identical_and_disjoint(magnet):
    """Identical sequences: one run covers everything, zero edits.  Sequences over
    disjoint alphabets: no zero anywhere, so the first extraction finds nothing and
    the vector stays all ones."""
    rng = random.Random(31)
    for m in (1, 7, 64, 100, 250):
        for E in (0, 2, 5):
            P = "".join(rng.choice("ACGT") for _ in range(m))
            if magnet(P, P, E, 0)[1] != 0:
                return False
            A = "".join(rng.choice("AC") for _ in range(m))
            B = "".join(rng.choice("GT") for _ in range(m))
            if magnet(A, B, E, 0)[1] != m:
                return False
    return True


def pin_E0_identity(magnet):
    """E = 0: one extraction on the main diagonal, and the bound ceil(m/1) = m
    rejects all but a full-length run, so the pair passes iff P == T."""
    rng = random.Random(32)
    for _ in range(200):
        m = rng.randint(1, 30)
        P = "".join(rng.choice("ACGT") for _ in range(m))
        T = P if rng.random() < 0.3 else "".join(rng.choice("ACGT") for _ in range(m))
        if (magnet(P, T, 0, 0)[1] <= 0) != (P == T):
            return False
    return True


def pin_shift_and_substitution(magnet):
    """P over {A, C}; T adds G, a base P lacks.  T = G^d + P[:m-d]: the only long
    run is [d, m-1] on upper diagonal d, so V = 1^d 0^(m-d).  T = P with one
    substitution by G at x: the two runs of the main diagonal are extracted with
    the encapsulation bit x between them, so V has a single one, at x."""
    rng = random.Random(33)
    m = 100
    for E in (3, 5):
        for d in range(1, E + 1):
            P = "".join(rng.choice("AC") for _ in range(m))
            if magnet(P, "G" * d + P[: m - d], E, 0) != ("1" * d + "0" * (m - d), d):
                return False
        for x in (30, 50, 70):
            P = "".join(rng.choice("AC") for _ in range(m))
            T = P[:x] + "G" + P[x + 1:]
            if magnet(P, T, E, 0) != ("0" * x + "1" + "0" * (m - x - 1), 1):
                return False
    return True


def pin_local_count(magnet):
    """Local counting drops the leading and trailing ones: T = G^d + P[:m-d]
    has only leading ones, so its local count is 0."""
    rng = random.Random(35)
    P = "".join(rng.choice("AC") for _ in range(100))
    return magnet(P, "GGG" + P[:97], 4, LOCAL)[1] == 0


ALL_MAGNET_PINS = [pin_fig6ab_counts, pin_hand_cases, pin_identical_and_disjoint,
                   pin_E0_identity, pin_shift_and_substitution, pin_local_count]
