// Splitting parameter by measurement.  alpha moves work between the real-
// space pair sum (terms inside r_c ~ 1/alpha: cost ~ alpha^-3 in 3D) and
// the reciprocal sum (G inside g_c ~ alpha: cost ~ alpha^3); the total is
// alpha-independent up to the cutoff tolerances (paper Eq. (2): v_E does
// not depend on gamma).  The best balance depends on the precision (GB300's
// FP64 pipe is ~70x slower than its FP32 pipe, and the two sums use them in
// different proportions), on N and on the cell, so it is measured: the
// full energy of sample configurations on trial contexts.
#include <algorithm>
#include <cmath>
#include <vector>

#include "capi_internal.h"

using namespace ewald;
using namespace ewald_capi;

namespace {

// Fastest of three timed full energies (after one untimed) of the sample on
// a context with splitting parameter alpha; < 0 if the context or a call
// fails (cutoffs the cell cannot take, memory).
double time_alpha(const ewald_desc &base, double alpha, void *stream, int W, const double *pos, double *e_dev) {
    ewald_desc d = base;
    d.gamma = alpha;
    ewald_ctx *c = nullptr;
    if (ewald_create(&d, stream, &c) != EWALD_OK) return -1.0;
    ewald_batch *b = nullptr;
    double best = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ewald_batch_create(c, W, &b) == EWALD_OK && ewald_batch_set_positions(b, pos, 0) == EWALD_OK &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        bool ok = ewald_energy(b, e_dev, 1) == EWALD_OK;
        for (int rep = 0; ok && rep < 3; ++rep) {
            ok = cudaEventRecord(e0, c->stream) == cudaSuccess && ewald_energy(b, e_dev, 1) == EWALD_OK &&
                 cudaEventRecord(e1, c->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0;
            if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && (best < 0 || ms < best)) best = ms;
        }
        if (ok && ewald_batch_sync(b) != EWALD_OK) best = -1.0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (b) ewald_batch_destroy(b);
    ewald_destroy(c);
    return best;
}

}  // namespace

extern "C" int ewald_tune_alpha(const ewald_desc *desc, void *cuda_stream, int n_walkers, const double *pos,
                                double *alpha_out, double *us_per_walker) {
    EWALD_NVTX("ewald_tune_alpha");
    if (!desc || !pos || !alpha_out || n_walkers < 1) return EWALD_ERR_ARG;
    if (desc->r_cutoff > 0 || desc->g_cutoff > 0) return EWALD_ERR_ARG;  // cutoffs follow alpha
    // starting point: the desc's alpha, else the library's balanced default
    ewald_ctx *c0 = nullptr;
    int st = ewald_create(desc, cuda_stream, &c0);
    if (st) return st;
    const double a0 = c0->t.alpha;
    ewald_destroy(c0);
    double *e_dev = nullptr;
    if (cudaMalloc((void **)&e_dev, sizeof(double) * (size_t)n_walkers) != cudaSuccess) return EWALD_ERR_OOM;
    double best_a = a0, best_t = time_alpha(*desc, a0, cuda_stream, n_walkers, pos, e_dev);
    if (best_t < 0) {
        cudaFree(e_dev);
        return EWALD_ERR_CUDA;
    }
    const double grid[] = {0.6, 0.75, 0.9, 1.15, 1.3, 1.5, 1.75, 2.0, 2.4, 3.0};
    for (double m : grid) {
        const double t = time_alpha(*desc, a0 * m, cuda_stream, n_walkers, pos, e_dev);
        if (t >= 0 && t < best_t) best_t = t, best_a = a0 * m;
    }
    // one refinement step around the best grid point
    for (double m : {0.93, 1.07}) {
        const double t = time_alpha(*desc, best_a * m, cuda_stream, n_walkers, pos, e_dev);
        if (t >= 0 && t < best_t) best_t = t, best_a = best_a * m;
    }
    cudaFree(e_dev);
    *alpha_out = best_a;
    if (us_per_walker) *us_per_walker = 1e3 * best_t / n_walkers;
    return EWALD_OK;
}
