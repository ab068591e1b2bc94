"""The integer-pipe probe that sets the ALU roofline: every instruction kind
reports a plausible issue rate, and the call checks its arguments on the
host."""
import ctypes

import pytest

import paper_1809_07858_gb300 as sj


def test_probe_rejects_bad_arguments():
    lib = sj.load_library()
    out = ctypes.c_double(0.0)
    assert lib.shouji_alu_probe(0, None) == 1
    assert lib.shouji_alu_probe(-1, ctypes.byref(out)) == 1
    assert lib.shouji_alu_probe(7, ctypes.byref(out)) == 1


@pytest.mark.gpu
def test_probe_rates(cuda_device):
    rates = {op: sj.shouji_alu_probe(op) for op in sj.PROBE_OPS}
    print("lane-ops per SM clock:", {k: round(v, 2) for k, v in rates.items()})
    # An SM issues at most 4 warp instructions per clock (128 lanes); the
    # narrowest integer pipe (population count) still does several lanes.
    for op, r in rates.items():
        assert 4.0 <= r <= 128.5, (op, r)
    # The logic pipe must sustain at least the rate the filter's roofline uses.
    assert rates["lop3"] >= 60.0
    # Two kinds on different pipes issue together at least as fast as one alone.
    assert rates["lop3+imad"] >= 0.95 * max(rates["lop3"], rates["imad"])
