// Diagnostic entry points: the real-space term erfc(alpha r)/r (paper Eq.
// (3), second term) as the kernels evaluate it - the mixed form's FP32
// function, scalar and paired (two terms per lane), and the tiered form's
// double-float head-term arithmetic - for the tests that pin their accuracy
// against FP64 and the two FP32 forms against each other.
#include <cmath>

#include "../../include/ewald.h"
#include "device_common.cuh"

using namespace ewald;

namespace {

__global__ void k_pair_terms(int n, const float *__restrict__ r2, TermK32 k, float *__restrict__ s_out,
                             float *__restrict__ p_out) {
    const int a = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (a >= n) return;
    const bool two = a + 1 < n;
    const float ra = r2[a], rb = two ? r2[a + 1] : ra;
    const float2 p = erfc_over_r_f32x2(make_float2(ra, rb), k);
    s_out[a] = erfc_over_r_f32(ra, k);
    p_out[a] = p.x;
    if (two) {
        s_out[a + 1] = erfc_over_r_f32(rb, k);
        p_out[a + 1] = p.y;
    }
}

// The tiered form's head-term arithmetic on r^2 alone: erfc(alpha r)/r in
// double-float (df_rsqrt, df_erfc; df_math.cuh), returned in FP64.
__global__ void k_pair_terms_df(int n, const double *__restrict__ r2, float a_hi, float a_lo,
                                double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DF q = df_from(r2[i]);
    const DF rinv = df_rsqrt(q);
    const DF x = df_mul(DF{a_hi, a_lo}, df_mul(q, rinv));
    out[i] = df_to(df_mul(df_erfc(x), rinv));
}

}  // namespace

extern "C" int ewald_pair_terms_df(int n, const double *r2, double alpha, double *out) {
    if (n < 0 || (n > 0 && (!r2 || !out)) || !(alpha > 0) || !std::isfinite(alpha)) return EWALD_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!(r2[i] > 0) || !std::isfinite(r2[i])) return EWALD_ERR_ARG;
    if (n == 0) return EWALD_OK;
    const float a_hi = (float)alpha, a_lo = (float)(alpha - (double)a_hi);
    double *d = nullptr;
    const size_t bytes = sizeof(double) * (size_t)n;
    cudaError_t e = cudaMalloc((void **)&d, 2 * bytes);
    if (e) return e == cudaErrorMemoryAllocation ? EWALD_ERR_OOM : EWALD_ERR_CUDA;
    e = cudaMemcpy(d, r2, bytes, cudaMemcpyHostToDevice);
    if (!e) {
        k_pair_terms_df<<<(n + 255) / 256, 256>>>(n, d, a_hi, a_lo, d + n);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpy(out, d + n, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e ? EWALD_ERR_CUDA : EWALD_OK;
}

extern "C" int ewald_pair_terms(int n, const float *r2, double alpha, float *scalar_out, float *paired_out) {
    if (n < 0 || (n > 0 && (!r2 || !scalar_out || !paired_out)) || !(alpha > 0) || !std::isfinite(alpha))
        return EWALD_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!(r2[i] > 0) || !std::isfinite(r2[i])) return EWALD_ERR_ARG;
    if (n == 0) return EWALD_OK;
    TermK32 k;
    k.a_hi = (float)alpha;
    k.a_lo = (float)(alpha - (double)k.a_hi);
    k.a2_hi = (float)(alpha * alpha);
    k.a2_lo = (float)(alpha * alpha - (double)k.a2_hi);
    float *d = nullptr;
    const size_t bytes = sizeof(float) * (size_t)n;
    cudaError_t e = cudaMalloc((void **)&d, 3 * bytes);
    if (e) return e == cudaErrorMemoryAllocation ? EWALD_ERR_OOM : EWALD_ERR_CUDA;
    e = cudaMemcpy(d, r2, bytes, cudaMemcpyHostToDevice);
    if (!e) {
        const int pairs = (n + 1) / 2, threads = 256;
        k_pair_terms<<<(pairs + threads - 1) / threads, threads>>>(n, d, k, d + n, d + 2 * (size_t)n);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpy(scalar_out, d + n, bytes, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(paired_out, d + 2 * (size_t)n, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e ? EWALD_ERR_CUDA : EWALD_OK;
}
