"""False accepts / false rejects of the filter against exact global edit
distance (the paper's accuracy measure, Sec. 3.2), on the synthetic workloads.

The paper reports zero false rejects on its real datasets; that is an empirical
result and it does not hold on these synthetic pairs, so the counts are printed
(run with -s) and only the exact case E = 0 is asserted.
"""
import numpy as np

import oracle
from paper_1809_07858_gb300 import synth


def fa_fr(reads, refs, E):
    acc, _ = oracle.shouji_batch(reads, refs, E, threads=8)
    ed = np.array([oracle.edit_distance(a.tobytes(), b.tobytes()) for a, b in zip(reads, refs)])
    sim = ed <= E
    return int((acc & ~sim).sum()), int((~acc & sim).sum()), int(sim.sum()), int((~sim).sum())


def test_report(capsys):
    rows = []
    r, t = synth.workload("small")
    rows.append(("small m=100", 5) + fa_fr(r, t, 5))
    for E in (0, 2, 5, 10):
        r, t = synth.workload("sweep", 20_000, E=E)
        rows.append(("sweep m=100", E) + fa_fr(r, t, E))
    for m, E in ((150, 7), (250, 15)):
        r, t = synth.workload("long", 5_000, m=m, E=E)
        rows.append(("long m=%d" % m, E) + fa_fr(r, t, E))
    with capsys.disabled():
        for name, E, fa, fr, sim, dis in rows:
            print("%-12s E=%2d similar=%5d dissimilar=%5d  FA=%5d (%.4f)  FR=%3d (%.4f)"
                  % (name, E, sim, dis, fa, fa / max(1, dis), fr, fr / max(1, sim)))
    for name, E, fa, fr, sim, dis in rows:
        if E == 0:
            assert fa == 0 and fr == 0   # E = 0 is the exact Hamming test
