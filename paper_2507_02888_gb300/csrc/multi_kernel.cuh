// The persistent multi-system energy kernel (multi_kernels.cu): its body as
// a template, compiled in general form and, for the common compositions of
// a launch, specialized (multi_spec.cu).
//
// k_multi_energy_t<R, DIMX, CMA, CMB, QWX>: DIMX = 2 or 3 when every
// system has that dimension (0: any); CMA, CMB >= 0 when every system's
// FP32 pair loop has one of these candidate slot counts (mixed_cm), -1:
// any; QWX = false when every system has uniform charges.  A specialized
// kernel carries only the code paths its systems take, so its registers
// serve those paths alone.
#pragma once
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

// Add one to a walker's completion counter, with release order for this
// thread's earlier writes (the item's partial sum) and acquire order for the
// combine that may follow; the count before the addition is returned.
__device__ inline int count_done(int *p) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

// A specialized kernel's FP32 pair item: the system's mixed_direct as a
// compile-time choice per item (uniform over the CTA), as in the
// single-system kernel's instantiations
template <int DIM, int CM>
__device__ __forceinline__ void multi_real_cm(const SysDev &ss, const BatchDev &sb, int w, int p,
                                              const MixedImageSmem &ims, unsigned char *work, int js) {
    if constexpr (CM >= 4) {
        if (ss.mixed_direct) {
            real_item_mixed_cm<DIM, CM, false, kDirectAlways>(ss, sb, w, p, ims, work, js);
            return;
        }
    }
    real_item_mixed_cm<DIM, CM, false, kDirectNever>(ss, sb, w, p, ims, work, js);
}

template <typename R, int DIMX, int CMA, int CMB, bool QWX>
__device__ __forceinline__ void multi_real(const SysDev &ss, const BatchDev &sb, int w, int p,
                                           const typename std::conditional<sizeof(R) == 4, MixedImageSmem,
                                                                           ImageSmem<R>>::type &ims,
                                           unsigned char *work, int js) {
    if constexpr (sizeof(R) == 8) {
        if (ss.dim == 3) real_item<R, 3>(ss, sb, w, p, ims, work, js);
        else real_item<R, 2>(ss, sb, w, p, ims, work, js);
    } else if constexpr (CMA < 0 || DIMX == 0 || QWX) {
        if (ss.dim == 3) real_item_mixed<3>(ss, sb, w, p, ims, work, js);
        else real_item_mixed<2>(ss, sb, w, p, ims, work, js);
    } else {
        if (mixed_cm(ss.cand_max) == CMA) multi_real_cm<DIMX, CMA>(ss, sb, w, p, ims, work, js);
        else multi_real_cm<DIMX, (CMB < 0 ? CMA : CMB)>(ss, sb, w, p, ims, work, js);
    }
}

template <typename R, int DIMX, int CMA, int CMB, bool QWX>
__global__ void __launch_bounds__(kMultiThreadsOf<R>, sizeof(R) == 4 ? kMultiMinBlocks32 : kMultiMinBlocks64)
    k_multi_energy_t(MultiDev m) {
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ SysDev ss;
    __shared__ BatchDev sb;
    __shared__ int s_next, s_img_sys, s_bat;
    // candidate tables: the FP64 loop's (ImageSmem) or the mixed loop's
    using Ims = typename std::conditional<sizeof(R) == 4, MixedImageSmem, ImageSmem<R>>::type;
    Ims ims;
    unsigned char *work = smem + m.img_bytes;
    // thread 0: the completion count of the previous item, examined one item
    // later (its latency then overlaps the next item); the last item of a
    // walker combines the walker's partial sums
    int pend_c = -1, pend_b = -1, pend_w = 0;
    auto finish_prev = [&]() {
        if (pend_b < 0) return;
        const SysDev &sp = m.sys[m.bat_sys[pend_b]];
        if (pend_c == sp.n_items + sp.n_gchunks - 1)
            m.e_all[m.wbase[pend_b] + pend_w] = combine_walker(sp, m.bat[pend_b], pend_w);
    };
    if (threadIdx.x == 0) {
        s_img_sys = s_bat = -1;
        s_next = atomicAdd(m.next, 1);
    }
    for (;;) {
        __syncthreads();  // the previous item is finished with shared memory
        const int it = s_next;
        if (it >= m.n_items) break;
        __syncthreads();  // every thread has read s_next
        if (threadIdx.x == 0) s_next = atomicAdd(m.next, 1);  // the item after this one
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
            if (DIMX == 3 || (DIMX == 0 && ss.dim == 3)) sfac_item<R, 3>(ss, sb, d.z, d.w, ss.sfac_te, true, work);
            else sfac_item<R, 2>(ss, sb, d.z, d.w, ss.sfac_te, true, work);
        } else {
            multi_real<R, DIMX, CMA, CMB, QWX>(ss, sb, d.z, d.w, ims, work, multi_jsplit<R>(ss));
        }
        if (threadIdx.x == 0) {  // thread 0 wrote the item's partial sum
            finish_prev();
            pend_c = count_done(m.done + m.wbase[d.y] + d.z);
            pend_b = d.y;
            pend_w = d.z;
        }
    }
    if (threadIdx.x == 0) finish_prev();
}


}  // namespace ewald
