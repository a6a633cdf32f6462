// Generated by gen_erfc_coeffs.py; do not edit.
// erfcx(x) ~ sum_k kErfcxP[k] w^k, w = p x / (1 + p x), p = 0.3125, x in [0, 7]: max rel err 3.61e-10
// exp(r) ~ sum_k kExpP[k] r^k, |r| <= ln2/2: max rel err 9.75e-11
#pragma once
namespace ewald {
constexpr float kErfcP = 3.125000000e-01f;
constexpr int kErfcxDeg = 11, kExpDeg = 7;
__device__ constexpr float kErfcxP[12] = {1.000000000e+00f, -3.610813379e+00f, 6.629189968e+00f, -7.780716419e+00f, 5.589600086e+00f, -1.808152556e+00f, -4.549140930e-01f, 4.032078087e-01f, 3.148303926e-01f, -4.375574291e-01f, 1.813006699e-01f, -2.595391311e-02f};
__device__ constexpr float kExpP[8] = {1.000000000e+00f, 1.000000000e+00f, 5.000000000e-01f, 1.666666567e-01f, 4.166646302e-02f, 8.333570324e-03f, 1.393507700e-03f, 1.974022452e-04f};
}  // namespace ewald
