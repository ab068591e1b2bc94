"""MAGNET oracle (Supplementary Sec. 7, Algorithms 3-4): its pins, a check that
every zero it reports is a match, and planted mistakes that the pins catch."""
import ctypes
import os
import random
import subprocess

import numpy as np
import pytest

import oracle
from _magnet_pins import ALL_MAGNET_PINS, magnet_readings_cases
from _pins import read_kv

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "shouji_oracle.c")


def _oracle_magnet(P, T, E, mode):
    V, c = oracle.magnet(P, T, E, mode)
    return "".join(map(str, V)), c


@pytest.mark.parametrize("pin", ALL_MAGNET_PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    assert pin(_oracle_magnet)


@pytest.mark.parametrize("case", magnet_readings_cases(), ids=lambda c: c[0])
def test_hand_case(case):
    name, P, T, E, V, ones = case
    assert _oracle_magnet(P, T, E, 0) == (V, ones)


def test_fig6c_local_parity_unpinned():
    """Fig. 6(c): the figure labels MAGNET's local result as 4 edits; the readings
    taken here give 5 (the Shouji count of the same example is also one above
    its label).  Kept as a regression value, not a pin."""
    g = read_kv("fig6c.txt")
    assert oracle.magnet(g["P"], g["T"], int(g["E"]), oracle.LOCAL)[1] == 5


def test_vector_zeros_are_matches():
    """Every zero of the MAGNET vector is a matching cell of some diagonal in the
    band (checked by comparing characters), and the count is the number of ones."""
    rng = random.Random(34)
    for _ in range(300):
        m = rng.randint(1, 40)
        E = rng.randint(0, 4)
        P = "".join(rng.choice("ACGT") for _ in range(m))
        T = "".join(rng.choice("ACGT") for _ in range(m))
        V, c = oracle.magnet(P, T, E)
        assert c == int(V.sum())
        for col in range(m):
            if V[col] == 0:
                assert any(0 <= col - d < m and P[col - d] == T[col]
                           for d in range(-E, E + 1))


def test_N_matches_nothing():
    """An N on either side is a mismatch on every diagonal."""
    assert oracle.magnet("N" * 20, "N" * 20, 3)[1] == 20
    P = "ACGT" * 5
    assert oracle.magnet(P, P[:10] + "N" + P[11:], 3) [1] == 1


MUTANTS = {
    "lower_wins_pair_tie": [("int L = X > Y ? X : Y;\n        int ls = X > Y ? s1 : s2, le = X > Y ? e1 : e2;",
                             "int L = X >= Y ? X : Y;\n        int ls = X >= Y ? s1 : s2, le = X >= Y ? e1 : e2;")],
    "last_j_wins": [("if (L > len) {", "if (L >= len) {")],
    "main_wins_ties": [("if (X > len) {", "if (X >= len) {")],
    "main_dropped": [("if (X > len) {", "if (0) {")],
    "ccz_rightmost": [("if (run > best) {", "if (run >= best) {")],
    "no_encapsulation": [("EXEN(st, e + 2, EI, calls + 1)", "EXEN(st, e + 1, EI, calls + 1)"),
                         ("EXEN(st, SI, s - 2, calls + 1)", "EXEN(st, SI, s - 1, calls + 1)")],
    "left_first": [("calls = EXEN(st, e + 2, EI, calls + 1);       /* right subproblem */\n"
                    "    calls = EXEN(st, SI, s - 2, calls + 1);       /* left subproblem */",
                    "calls = EXEN(st, SI, s - 2, calls + 1);\n"
                    "    calls = EXEN(st, e + 2, EI, calls + 1);")],
    "floor_bound": [("len < (st->m - E + E) / (E + 1)", "len < (st->m - E) / (E + 1)")],
    "no_early_reject": [("if (calls == 1 && len <", "if (0 && len <")],
    "early_reject_every_call": [("if (calls == 1 && len <", "if (len <")],
    "E_plus_2_extractions": [("calls <= E + 1))", "calls <= E + 2))")],
    "E_extractions": [("calls <= E + 1))", "calls <= E))")],
    "empty_range_counts": [("    if (len == 0)\n        return calls - 1;",
                            "    if (len == 0)\n        return calls;")],
    "P_and_T_exchanged": [("build_map(P, mp, T, m, E, map);\n    for (int c = 0; c < m; ++c)\n        vec[c] = 1;",
                           "build_map(T, mp, P, m, E, map);\n    for (int c = 0; c < m; ++c)\n        vec[c] = 1;")],
}


def _build(name, subs, tmp_path):
    src = open(SRC).read()
    for a, b in subs:
        assert src.count(a) == 1, "mutation anchor for %s not unique: %r" % (name, a)
        src = src.replace(a, b)
    c = tmp_path / ("%s.c" % name)
    so = tmp_path / ("%s.so" % name)
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-o", str(so), str(c)])
    lib = ctypes.CDLL(str(so))
    lib.oracle_magnet_mode.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_char_p,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p]
    lib.oracle_magnet_mode.restype = ctypes.c_int

    def magnet(P, T, E, mode):
        V = np.zeros(len(T), np.uint8)
        c = lib.oracle_magnet_mode(P.encode(), len(P), T.encode(), len(T), E, mode,
                                   V.ctypes.data)
        return "".join(map(str, V)), c
    return magnet


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    magnet = _build(name, MUTANTS[name], tmp_path)
    failed = [p.__name__ for p in ALL_MAGNET_PINS if not p(magnet)]
    assert failed, "planted mistake %s passes every MAGNET pin" % name


def test_batch_matches_single_calls():
    """The threaded batch entry gives, pair by pair, the single-pair results."""
    rng = np.random.default_rng(21)
    n, m, E = 300, 60, 4
    reads = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=(n, m))
    refs = reads.copy()
    mut = rng.random((n, m)) < 0.06
    refs[mut] = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=int(mut.sum()))
    acc, cnt = oracle.shouji_batch(reads, refs, E, threads=3, magnet=True)
    for i in range(n):
        _, c = oracle.magnet(reads[i].tobytes(), refs[i].tobytes(), E)
        assert cnt[i] == c and acc[i] == (c <= E)
