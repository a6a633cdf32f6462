"""Generate erfc_df_coeffs.h: piecewise Taylor coefficients of erfc(x) on
[0, 4] for the double-float evaluation of the tiered FP64 form's head terms.

The interval [0, 4] is cut into 32 pieces of width 1/8; on piece m,
erfc(c_m + s) = sum_{k=0}^{13} a_k s^k with c_m = (m + 1/2)/8, |s| <= 1/16,
a_k = erfc^(k)(c_m) / k! from the derivatives of the definition
(d/dx erfc = -2/sqrt(pi) e^{-x^2}, then Hermite-type recurrences, all done
by mpmath at 40 digits).  The truncation error is below 1.1e-17 relative on
every piece (the Taylor terms fall like (2 x s)^k / k!); each coefficient is
stored as a pair of floats hi + lo (48 bits).

Usage: python gen_erfc_df.py > erfc_df_coeffs.h   (needs mpmath)
"""
import mpmath as mp
import numpy as np

PIECES, WIDTH, DEG = 32, 0.125, 13


def main():
    mp.mp.dps = 40
    worst = mp.mpf(0)
    rows = []
    for m in range(PIECES):
        c = (m + mp.mpf(1) / 2) * WIDTH
        a = [mp.diff(mp.erfc, c, k) / mp.factorial(k) for k in range(DEG + 1)]
        for j in range(17):
            s = (-mp.mpf(1) / 2 + mp.mpf(j) / 16) * WIDTH
            p = mp.fsum(a[k] * s ** k for k in range(DEG + 1))
            worst = max(worst, abs(p / mp.erfc(c + s) - 1))
        pairs = []
        for v in a:
            hi32 = float(np.float32(float(v)))
            lo32 = float(np.float32(float(v - mp.mpf(hi32))))
            pairs.append((hi32, lo32))
        rows.append(pairs)
    print("// Generated by gen_erfc_df.py; do not edit.")
    print("// erfc(c_m + s) ~ sum_k kErfcDf[m][k] s^k, c_m = (m + 1/2) / 8, |s| <= 1/16, m < %d:" % PIECES)
    print("// truncation below %s relative; coefficients as float pairs (hi, lo)." % mp.nstr(worst, 3))
    print("#pragma once")
    print("namespace ewald {")
    print("constexpr int kErfcDfPieces = %d, kErfcDfDeg = %d;" % (PIECES, DEG))
    print("constexpr float kErfcDfWidthInv = %.1ff;" % (1 / WIDTH))
    print("__device__ const float2 kErfcDf[%d][%d] = {" % (PIECES, DEG + 1))
    for pairs in rows:
        print("    {%s}," % ", ".join("{%.9ef, %.9ef}" % p for p in pairs))
    print("};")
    print("}  // namespace ewald")


if __name__ == "__main__":
    main()
