// The mixed path's real-space kernel (pair loop in real_mixed.cuh):
// persistent CTAs over (walker, tile pair) items, one instantiation per
// candidate-list length and charge pattern, chosen on the host so that
// each is compiled with the registers of its own loop.
#include "real_mixed.cuh"

namespace ewald {

// DIRECT: the system's mixed_direct, as a compile-time choice (the first
// two images of each pair evaluated without the lane rings, CM = 4 ... 8)
template <int DIM, int CM, bool QW, bool DIRECT = false>
__global__ void __launch_bounds__(kRealMixedThreads, kRealMinBlocksMixed) k_real_mixed(SysDev s, BatchDev b) {
    extern __shared__ __align__(32) unsigned char smem[];
    MixedImageSmem ims;
    ims.carve(smem, s, DIM);
    ims.stage(s, DIM);
    unsigned char *work = smem + MixedImageSmem::bytes(s, DIM);
    const long long total = (long long)b.W * s.n_items;
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        const int w = (int)(item / s.n_items), p = (int)(item - (long long)w * s.n_items);
        // units of 32 x 8 pairs (16 warps) or 32 x 16 (8 warps): a 256 x 256
        // item splits evenly over the CTA's warps
        real_item_mixed_cm<DIM, CM, QW, DIRECT ? kDirectAlways : kDirectNever>(s, b, w, p, ims, work,
                                                                             s.real_warps / 4);
    }
}

using RealFn = void (*)(SysDev, BatchDev);

template <int DIM, bool QW>
static RealFn pick_cm(int cm, bool direct) {
    switch (cm) {
        case 2: return k_real_mixed<DIM, 2, QW>;
        case 4: return direct ? k_real_mixed<DIM, 4, QW, true> : k_real_mixed<DIM, 4, QW>;
        case 6: return direct ? k_real_mixed<DIM, 6, QW, true> : k_real_mixed<DIM, 6, QW>;
        case 8: return direct ? k_real_mixed<DIM, 8, QW, true> : k_real_mixed<DIM, 8, QW>;
        default: return k_real_mixed<DIM, 0, QW>;
    }
}

static RealFn real_mixed_fn(const SysDev &s) {
    const int cm = mixed_cm(s.cand_max);
    const bool d = s.mixed_direct != 0;
    if (s.dim == 3) return s.q_uniform ? pick_cm<3, false>(cm, d) : pick_cm<3, true>(cm, d);
    return s.q_uniform ? pick_cm<2, false>(cm, d) : pick_cm<2, true>(cm, d);
}

int configure_real_mixed(const SysDev &s, size_t smem, int *blocks_per_sm) {
    const RealFn f = real_mixed_fn(s);
    cudaError_t e = allow_max_smem(f, smem);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, 32 * s.real_warps, smem);
    return e;
}

int launch_real_mixed(const SysDev &s, const BatchDev &b, int grid, size_t smem, cudaStream_t st) {
    real_mixed_fn(s)<<<grid, 32 * s.real_warps, smem, st>>>(s, b);
    return cudaGetLastError();
}

}  // namespace ewald
