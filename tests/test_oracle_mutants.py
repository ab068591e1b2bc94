"""The pins have teeth: each plausible mistake, planted in a temporary copy of
the oracle source (never in the oracle itself), fails at least one pin."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from _pins import ALL_PINS

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "shouji_oracle.c")

MUTANTS = {
    "orientation_swapped": [("int i = c - d;", "int i = c + d;")],
    "out_of_band_is_match": [("cell = 1;                /* R3", "cell = 0;                /* R3")],
    "m_minus_3_windows": [("for (int c = 0; c < m; ++c) {            /* m search",
                           "for (int c = 0; c < m - 3; ++c) {            /* m search")],
    "no_leading_zero_tie_rule": [("|| (zc == zz && Z[0] == 1 && cand[0] == 0)", "")],
    "tie_takes_last": [("if (zc > zz ||", "if (zc >= zz ||")],
    "update_on_tie": [("if (CZ(Z, 4) > CZ(cur, 4))", "if (CZ(Z, 4) >= CZ(cur, 4))")],
    "main_wins_ties": [("if (CZ(cand, 4) > CZ(Z, 4))\n                memcpy",
                        "if (CZ(cand, 4) >= CZ(Z, 4))\n                memcpy")],
    "upper_before_lower": [("int d = (side == 0) ? -j : +j;", "int d = (side == 0) ? +j : -j;")],
    "P_and_T_exchanged": [("build_map(P, mp, T, m, E, map);",
                           "build_map(T, mp, P, m, E, map);")],
    "main_diagonal_dropped": [("if (CZ(cand, 4) > CZ(Z, 4))\n                memcpy(Z, cand, 4);\n        }",
                               "if (0)\n                memcpy(Z, cand, 4);\n        }")],
    "past_end_segment_is_match": [("seg[k] = (c + k < m) ? map[(size_t)(d + E) * m + c + k] : 1;",
                                   "seg[k] = (c + k < m) ? map[(size_t)(d + E) * m + c + k] : 0;")],
    "past_end_vector_is_match": [("cur[k] = (c + k < m) ? shouji[c + k] : 1;",
                                  "cur[k] = (c + k < m) ? shouji[c + k] : 0;")],
    "N_matches_N": [("static int is_unknown_base(char x) { return x == 'N'; }",
                     "static int is_unknown_base(char x) { (void)x; return 0; }")],
    "last_column_dropped": [("int ones = m - CZ(shouji, m);", "int ones = (m - 1) - CZ(shouji, m - 1);")],
    "selection_not_reset_per_window": [
        ("            segment(map, m, E, -1, c, Z);    /* lower_1 is examined first */\n",
         "            if (c == 0) segment(map, m, E, -1, c, Z);\n")],
}


def _build(name, subs, tmp_path):
    src = open(SRC).read()
    for a, b in subs:
        assert a in src, "mutation anchor missing for %s: %r" % (name, a)
        src = src.replace(a, b)
    c = tmp_path / ("%s.c" % name)
    so = tmp_path / ("%s.so" % name)
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-o", str(so), str(c)])
    lib = ctypes.CDLL(str(so))
    lib.oracle_shouji.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_void_p]
    lib.oracle_shouji.restype = ctypes.c_int

    def shouji(P, T, E):
        S = np.zeros(len(P), np.uint8)
        ones = lib.oracle_shouji(P.encode(), T.encode(), len(P), E, S.ctypes.data)
        return "".join(map(str, S)), ones
    return shouji


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    shouji = _build(name, MUTANTS[name], tmp_path)
    failed = [p.__name__ for p in ALL_PINS if not p(shouji)]
    assert failed, "planted mistake %s passes every pin" % name
