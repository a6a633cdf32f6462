"""The double-float erfc of the tiered FP64 form's head terms
(csrc/erfc_df_coeffs.h): 32 pieces of width 1/8 on [0, 4], 14 Taylor
coefficients each stored as float pairs.  The committed header must be what
its generator writes, and the coefficients as stored (hi + lo) must give
erfc to a few 1e-15 relative against mpmath's erfc at 40 digits."""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2507_02888_gb300", "csrc")


def test_header_is_generator_output():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "gen_erfc_df.py")], capture_output=True, text=True,
                         check=True).stdout
    assert out == open(os.path.join(CSRC, "erfc_df_coeffs.h")).read()


def test_stored_coefficients_give_erfc():
    text = open(os.path.join(CSRC, "erfc_df_coeffs.h")).read()
    rows = re.findall(r"\{(\{[^{}]*\}(?:, \{[^{}]*\})*)\},", text)
    assert len(rows) == 32
    # the C float literals denote the nearest float32
    coef = [[tuple(float(np.float32(float(v.strip().rstrip("f")))) for v in pair.split(","))
             for pair in re.findall(r"\{([^{}]*)\}", row)] for row in rows]
    assert all(len(r) == 14 for r in coef)
    mp.mp.dps = 40
    worst = mp.mpf(0)
    for m in range(32):
        c = (m + mp.mpf(1) / 2) / 8
        a = [mp.mpf(h) + mp.mpf(l) for h, l in coef[m]]
        for j in range(9):
            s = (-mp.mpf(1) / 2 + mp.mpf(j) / 8) / 8
            p = mp.fsum(a[k] * s ** k for k in range(14))
            worst = max(worst, abs(p / mp.erfc(c + s) - 1))
    assert worst < 5e-15, worst
