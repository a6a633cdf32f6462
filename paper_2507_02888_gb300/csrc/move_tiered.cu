// Proposed single-particle moves of the tiered FP64 form (EWALD_FP64_TIERED):
// one CTA per walker, the work in tiered_delta_e (move_tiered.cuh).
// Accepting a move is the FP64 form's k_accept (rho(G) stays FP64).
#include "move_tiered.cuh"
#include "move_tiered.h"

namespace ewald {

namespace {

template <int DIM>
__global__ void __launch_bounds__(kMoveThreads)
    k_propose_tiered(SysDev s, BatchDev b, const int *__restrict__ kk, const double *__restrict__ r_new,
                     double *__restrict__ de) {
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ int sk;
    __shared__ unsigned long long su_old[3], su_new[3];
    TieredMoveSmem m;
    m.carve_split(smem, smem + TieredMoveSmem::img_bytes(s), s, DIM);
    const int w = blockIdx.x, tid = threadIdx.x;
    if (tid == 0) {
        const int k = kk[w];
        unsigned long long un[3] = {0, 0, 0};
        bool ok = k >= 0 && k < s.n_mob;
        ok = cart_to_fixed<DIM>(s, r_new + (size_t)w * DIM, un) && ok;
        if (!ok) {
            atomicOr(b.status, ST_BAD_INDEX);
            b.pend_k[w] = -1;
            sk = -1;
        } else {
            b.pend_k[w] = k;
            for (int d = 0; d < 3; ++d) {
                b.pend_u[(size_t)w * 3 + d] = un[d];
                su_new[d] = un[d];
                su_old[d] = d < DIM ? b.u[((size_t)w * DIM + d) * s.mob_stride + k] : 0;
            }
            sk = k;
        }
    }
    __syncthreads();
    const int k = sk;
    if (k < 0) {
        if (tid == 0) de[w] = __longlong_as_double(0x7ff8000000000000LL);  // NaN
        return;
    }
    m.stage(s, DIM);
    const unsigned long long uo[3] = {su_old[0], su_old[1], su_old[2]}, un[3] = {su_new[0], su_new[1], su_new[2]};
    Part<float> pold, pnew;
    tiered_move_parts<DIM>(s, k, uo, un, pold, pnew);
    build_move_tables<double, DIM>(s, uo, un, m.tab);
    __syncthreads();
    const double tot = tiered_delta_e<DIM>(s, b, w, k, pold, pnew, m);
    if (tid == 0) de[w] = tot;
}

}  // namespace

int launch_propose_tiered(const SysDev &s, const BatchDev &b, const int *k, const double *r_new, double *de,
                          cudaStream_t st) {
    const size_t smem = TieredMoveSmem::bytes(s);
    cudaError_t e;
    if (s.dim == 3) {
        if ((e = allow_max_smem(k_propose_tiered<3>, smem))) return e;
        k_propose_tiered<3><<<b.W, kMoveThreads, smem, st>>>(s, b, k, r_new, de);
    } else {
        if ((e = allow_max_smem(k_propose_tiered<2>, smem))) return e;
        k_propose_tiered<2><<<b.W, kMoveThreads, smem, st>>>(s, b, k, r_new, de);
    }
    return cudaGetLastError();
}

}  // namespace ewald
