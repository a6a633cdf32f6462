"""The FP32 pair term's polynomial coefficients (csrc/erfc_coeffs.h).

erfcx(x) is a degree-11 polynomial in w = p x / (1 + p x) and exp(r) a
degree-7 polynomial on |r| <= ln2/2 (the FP32 erfc of the mixed path, paper
Sec. 6).  The committed header must be what its generator writes, and the
float coefficients, as stored, must meet the fit's bounds against SciPy's
double-precision erfcx and exp.
"""
import math
import os
import re
import subprocess
import sys

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2507_02888_gb300", "csrc")


def _coeffs(text, name):
    body = re.search(name + r"\[\d+\] = \{([^}]*)\}", text).group(1)
    return np.array([float(v.strip().rstrip("f")) for v in body.split(",")], dtype=np.float32).astype(np.float64)


def test_header_is_generator_output():
    gen = subprocess.run([sys.executable, os.path.join(CSRC, "gen_erfc_coeffs.py")], capture_output=True,
                         text=True, check=True).stdout
    assert gen == open(os.path.join(CSRC, "erfc_coeffs.h")).read()


def test_float_coefficients_meet_the_fit_bounds():
    text = open(os.path.join(CSRC, "erfc_coeffs.h")).read()
    p = float(re.search(r"kErfcP = ([0-9.e+-]+)f", text).group(1))
    cw, ce = _coeffs(text, "kErfcxP"), _coeffs(text, "kExpP")
    x = np.linspace(0.0, 7.0, 200001)
    w = p * x / (1 + p * x)
    rel = np.polyval(cw[::-1], w) / scipy_special.erfcx(x) - 1
    assert np.max(np.abs(rel)) < 5e-10
    r = np.linspace(-math.log(2) / 2, math.log(2) / 2, 100001)
    assert np.max(np.abs(np.polyval(ce[::-1], r) / np.exp(r) - 1)) < 2e-10
    # erfc(x) = exp(-x^2) erfcx(x) at a few points, to the fit's accuracy
    for xv in (0.0, 0.3, 1.0, 2.5, 4.5):
        wv = p * xv / (1 + p * xv)
        assert abs(math.exp(-xv * xv) * np.polyval(cw[::-1], wv) / math.erfc(xv) - 1) < 5e-10
