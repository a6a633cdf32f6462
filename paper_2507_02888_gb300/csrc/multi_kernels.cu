// Persistent multi-system kernels: walkers of several systems (different N,
// cell, dimension and charges, one precision) in one launch.
//
// k_multi_energy: a host-built list of work items (walker x G-run chunk and
// walker x pair tile) ordered longest first; CTAs take the next item from an
// atomic counter; after each item the CTA bumps its walker's completion
// counter, and the CTA that completes a walker's last item adds up that
// walker's partial sums (in a fixed order, so results do not depend on the
// schedule or on the other systems in the launch).  No CTA ever waits for
// another one.
#include <type_traits>

#include "energy_items.cuh"
#include "multi.h"
#include "real_mixed.cuh"

namespace ewald {

// Copy a POD struct from global to shared memory with the whole CTA.
template <typename T>
__device__ inline void cta_copy(T *dst, const T *src) {
    static_assert(sizeof(T) % 4 == 0, "word copy");
    const int *s = (const int *)src;
    int *d = (int *)dst;
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
}

// j slices per 32 x 32 sub-tile of a pair item, so that the item has at
// least as many work units as the CTA has warps (FP32: four times as many,
// so that diagonal items split evenly too; a property of the system alone:
// results do not depend on the other systems of the launch)
template <typename R>
__device__ inline int multi_jsplit(const SysDev &s) {
    const int S = s.tile / 32, per = S * S, want = (kMultiThreadsOf<R> / 32) * (sizeof(R) == 4 ? 4 : 1);
    int js = 1;
    while (per * js < want && js < 32) js *= 2;
    return js;
}

template <typename R>
__global__ void __launch_bounds__(kMultiThreadsOf<R>, sizeof(R) == 4 ? kMultiMinBlocks32 : kMultiMinBlocks64)
    k_multi_energy(MultiDev m) {
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ SysDev ss;
    __shared__ BatchDev sb;
    __shared__ int s_item, s_last, s_img_sys, s_bat;
    // candidate tables: the FP64 loop's (ImageSmem) or the mixed loop's
    using Ims = typename std::conditional<sizeof(R) == 4, MixedImageSmem, ImageSmem<R>>::type;
    Ims ims;
    unsigned char *work = smem + m.img_bytes;
    if (threadIdx.x == 0) s_img_sys = s_bat = -1;
    for (;;) {
        __syncthreads();  // the previous item is finished with shared memory
        if (threadIdx.x == 0) s_item = atomicAdd(m.next, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= m.n_items) break;
        const int4 d = m.items[it];  // (kind, batch, walker, sub)
        const int sys = m.bat_sys[d.y];
        if (d.y != s_bat) {  // uniform over the CTA; items come grouped by batch
            cta_copy(&ss, m.sys + sys);
            cta_copy(&sb, m.bat + d.y);
            __syncthreads();
            if (threadIdx.x == 0) s_bat = d.y;
        }
        __syncthreads();
        if (d.x == kItemReal && s_img_sys != sys) {  // uniform over the CTA
            ims.carve(smem, ss, ss.dim);
            ims.stage(ss, ss.dim);
            __syncthreads();
            if (threadIdx.x == 0) s_img_sys = sys;
        }
        ims.carve(smem, ss, ss.dim);
        if (d.x == kItemSfac) {
            if (ss.dim == 3) sfac_item<R, 3>(ss, sb, d.z, d.w, ss.sfac_te, true, work);
            else sfac_item<R, 2>(ss, sb, d.z, d.w, ss.sfac_te, true, work);
        } else {
            const int js = multi_jsplit<R>(ss);
            if constexpr (sizeof(R) == 4) {
                if (ss.dim == 3) real_item_mixed<3>(ss, sb, d.z, d.w, ims, work, js);
                else real_item_mixed<2>(ss, sb, d.z, d.w, ims, work, js);
            } else {
                if (ss.dim == 3) real_item<R, 3>(ss, sb, d.z, d.w, ims, work, js);
                else real_item<R, 2>(ss, sb, d.z, d.w, ims, work, js);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();  // this item's partial sum is visible before the count
            const int c = atomicAdd(m.done + m.wbase[d.y] + d.z, 1);
            s_last = c == ss.n_items + ss.n_gchunks - 1;
        }
        __syncthreads();
        if (s_last && threadIdx.x == 0) {
            __threadfence();  // read the other CTAs' partial sums after their counts
            m.e_all[m.wbase[d.y] + d.z] = combine_walker(ss, sb, d.z);
        }
    }
}

size_t multi_energy_smem(const std::vector<SysDev> &sys, int precision, size_t *img_bytes) {
    size_t img = 0, work = 0;
    for (const SysDev &s : sys) {
        size_t ib = precision == EWALD_FP64 ? ImageSmem<double>::bytes(s, s.dim) : MixedImageSmem::bytes(s, s.dim);
        img = std::max(img, ib);
        const int threads = precision == EWALD_FP64 ? kMultiThreads64 : kMultiThreads32;
        work = std::max(work, sfac_bytes(s, precision, s.sfac_te, threads));
        work = std::max(work, precision == EWALD_FP64 ? real_work_bytes(s, precision, threads / 32)
                                                      : mixed_real_work_bytes(s, threads / 32));
    }
    *img_bytes = img;
    return img + work;
}

int configure_multi(int precision, size_t smem, int *grid) {
    int dev, sms, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) return e;
    if (precision == EWALD_FP64) {
        if ((e = allow_max_smem(k_multi_energy<double>, smem))) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_multi_energy<double>, kMultiThreads64, smem);
    } else {
        if ((e = allow_max_smem(k_multi_energy<float>, smem))) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_multi_energy<float>, kMultiThreads32, smem);
    }
    if (e) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    *grid = sms * occ;
    return cudaSuccess;
}

int launch_multi_energy(const MultiDev &m, int precision, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(m.next, 0, sizeof(int), st);
    if (!e) e = cudaMemsetAsync(m.done, 0, sizeof(int) * (size_t)m.n_walkers, st);
    if (e) return e;
    const int g = std::min(grid, std::max(m.n_items, 1));
    if (precision == EWALD_FP64) k_multi_energy<double><<<g, kMultiThreads64, smem, st>>>(m);
    else k_multi_energy<float><<<g, kMultiThreads32, smem, st>>>(m);
    return cudaGetLastError();
}

}  // namespace ewald
