"""The mixed path's real-space cutoff, erfc(alpha r_c) = 1e-10, against the
definition's 1e-16 (paper Sec. 6.1 re-expresses hard-wired tolerances in
terms of the working precision; Eq. (3) is the sum being truncated).

The images the mixed path leaves out change the oracle's energy by far less
than the mixed path's 1e-6 accuracy gate, on every workload shape, including
random electron-gas walkers whose E is a small difference of large parts.
"""
import numpy as np
import pytest

import oracle
from paper_2507_02888_gb300 import inputs as I

MIXED_REAL_TOL = 1e-10


def _all(w, k):
    p, q = w["pos"][k], w["q"]
    if len(w["fixed_q"]):
        p = np.concatenate([p, w["fixed_pos"]])
        q = np.concatenate([q, w["fixed_q"]])
    return p, q


@pytest.mark.parametrize("name,walkers", [("heg3d_sc_n54", 4), ("heg2d_hex_n338", 2),
                                          ("diamond_3x3x3", 1), ("heg3d_fcc_n1024", 1)])
def test_mixed_real_cutoff_truncation_is_far_below_the_gate(name, walkers):
    w = I.workload(name, walkers)
    rc16, gc = oracle.cutoffs(w["dim"], w["alpha"])
    rc10, _ = oracle.cutoffs(w["dim"], w["alpha"], MIXED_REAL_TOL)
    assert rc10 < rc16
    for k in range(walkers):
        p, q = _all(w, k)
        e16, c16 = oracle.energy(w["dim"], w["lattice"], p, q, w["alpha"], rc16, gc)
        e10, c10 = oracle.energy(w["dim"], w["lattice"], p, q, w["alpha"], rc10, gc)
        floor = max(abs(e16), 1e-2 * (abs(c16[0]) + abs(c16[2]) + abs(c16[1] + c16[3]) + abs(c16[4])))
        # only the real-space parts (pair sum and Madelung self-images) change
        assert np.array_equal(c10[2:], c16[2:])
        assert abs(e10 - e16) <= 2e-8 * floor, (name, k, (e10 - e16) / floor)
