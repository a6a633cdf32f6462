// Generated by gen_erfc_coeffs.py; do not edit.
// erfcx(x) ~ sum_k kErfcxP[k] t^k, t = 1/(1 + 0.3125 x), x in [0, 7]: max rel err 3.77e-10
// exp(r) ~ sum_k kExpP[k] r^k, |r| <= ln2/2: max rel err 9.75e-11
#pragma once
namespace ewald {
constexpr float kErfcP = 3.125000000e-01f;
constexpr int kErfcxDeg = 11, kExpDeg = 7;
__device__ constexpr float kErfcxP[12] = {4.256363172e-05f, 1.754120886e-01f, 1.847466528e-01f, 1.210958883e-01f, 3.176951706e-01f, -2.798867822e-01f, 7.653132081e-01f, -6.559600830e-01f, 4.879517555e-01f, -7.091723382e-02f, -6.618145853e-02f, 2.068823017e-02f};
__device__ constexpr float kExpP[8] = {1.000000000e+00f, 1.000000000e+00f, 5.000000000e-01f, 1.666666567e-01f, 4.166646302e-02f, 8.333570324e-03f, 1.393507700e-03f, 1.974022452e-04f};
}  // namespace ewald
