"""Generate erfc_coeffs.h: polynomial coefficients of the FP32 erfc used by
the mixed-precision kernels.

erfc(x) = exp(-x^2) * erfcx(x), with erfcx approximated by a polynomial of
degree 11 in w = 1 - t = p x t, t = 1/(1 + p x), p = 0.3125 (t is the change
of variable of the Hastings-type approximations in Abramowitz & Stegun
7.1.26; the fit is our own, of higher degree), and exp(r) on |r| <= ln2/2 by
a degree-7 polynomial after Cody & Waite range reduction.  The polynomial is
written in w rather than t because the kernels compute w = (p x) t with an
error proportional to w: near x = 0, where the pair terms are largest, erfcx
is then evaluated from an argument whose rounding vanishes with x (in t, one
rounding of 1 + p x is amplified about 3.6 times into erfcx).  Both are fitted here in relative error
(least squares driven towards minimax by Lawson reweighting) against SciPy's
double-precision erfcx and exp.  The coefficients are rounded to float32 one
at a time and the remaining ones refitted, so that the rounded polynomial
itself stays within a few 1e-10 of the target: the kernels' errors are then
the (unbiased) roundings of FP32 arithmetic, not a systematic offset.

Usage: python gen_erfc_coeffs.py > erfc_coeffs.h
"""
import math

import numpy as np
from scipy.special import erfcx

P = 0.3125          # exactly representable
XMAX = 7.0          # erfc(7) ~ 4e-23, beyond any cutoff in use
DEG_P, DEG_E = 11, 7


def seq_fit(nodes, target, deg):
    V = np.vander(nodes, deg + 1, increasing=True)
    fixed = []
    for k in range(deg + 1):
        resid = target - (V[:, :k] @ np.array(fixed) if k else 0.0)
        A = V[:, k:] / target[:, None]
        b = resid / target
        wgt = np.ones_like(target)
        for _ in range(25):
            c, *_ = np.linalg.lstsq(A * np.sqrt(wgt)[:, None], b * np.sqrt(wgt), rcond=None)
            e = np.abs(A @ c - b)
            wgt *= e / e.max() + 1e-3
            wgt /= wgt.sum()
        fixed.append(float(np.float32(c[0])))
    return np.array(fixed)


def main():
    tlo = 1.0 / (1.0 + P * XMAX)
    k = np.arange(8000)
    tn = 0.5 * (1 + tlo) + 0.5 * (1 - tlo) * np.cos(np.pi * (k + 0.5) / len(k))
    cp = seq_fit(1 - tn, erfcx((1 / tn - 1) / P), DEG_P)
    h = math.log(2) / 2
    rn = np.cos(np.pi * (np.arange(4000) + 0.5) / 4000) * h
    ce = seq_fit(rn, np.exp(rn), DEG_E)
    tt = np.linspace(tlo, 1, 400001)
    ep = np.max(np.abs(np.polyval(cp[::-1], 1 - tt) / erfcx((1 / tt - 1) / P) - 1))
    rr = np.linspace(-h, h, 200001)
    ee = np.max(np.abs(np.polyval(ce[::-1], rr) / np.exp(rr) - 1))
    print("// Generated by gen_erfc_coeffs.py; do not edit.")
    print("// erfcx(x) ~ sum_k kErfcxP[k] w^k, w = p x / (1 + p x), p = %.4f, x in [0, %g]: max rel err %.2e"
          % (P, XMAX, ep))
    print("// exp(r) ~ sum_k kExpP[k] r^k, |r| <= ln2/2: max rel err %.2e" % ee)
    print("#pragma once")
    print("namespace ewald {")
    print("constexpr float kErfcP = %.9ef;" % P)
    print("constexpr int kErfcxDeg = %d, kExpDeg = %d;" % (DEG_P, DEG_E))
    print("__device__ constexpr float kErfcxP[%d] = {%s};" % (DEG_P + 1, ", ".join("%.9ef" % v for v in cp)))
    print("__device__ constexpr float kExpP[%d] = {%s};" % (DEG_E + 1, ", ".join("%.9ef" % v for v in ce)))
    print("}  // namespace ewald")


if __name__ == "__main__":
    main()
