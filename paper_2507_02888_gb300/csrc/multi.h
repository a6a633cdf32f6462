// Device-side description of a multi-system launch (multi_kernels.cu).
#pragma once
#include <vector>

#include "ewald_internal.h"

namespace ewald {

// threads per CTA: the FP32 kernel takes the mixed real-space loop's 16
// warps (real_mixed.cuh), the FP64 one 8
constexpr int kMultiThreads32 = 512, kMultiThreads64 = 256;
template <typename R>
constexpr int kMultiThreadsOf = sizeof(R) == 4 ? kMultiThreads32 : kMultiThreads64;
// resident CTAs per SM the register budget is sized for (FP32, FP64 path)
constexpr int kMultiMinBlocks32 = 2, kMultiMinBlocks64 = 2;
enum : int { kItemSfac = 0, kItemReal = 1 };

struct MultiDev {
    const SysDev *sys;     // [n_sys]
    const BatchDev *bat;   // [n_bat]
    const int *bat_sys;    // [n_bat] system of each batch
    const int *wbase;      // [n_bat] first walker of each batch in the concatenation
    const int4 *items;     // [n_items] (kind, batch, walker, sub), longest first
    int n_items, n_walkers;
    size_t img_bytes;      // shared memory reserved for the image table
    int *next;             // work counter
    int *done;             // [n_walkers] items completed per walker
    double *e_all;         // [n_walkers] energies
};

using MultiFn = void (*)(MultiDev);
size_t multi_energy_smem(const std::vector<SysDev> &sys, int precision, size_t *img_bytes);
MultiFn multi_kernel(int precision, const std::vector<SysDev> &sys);
// multi_spec.cu: the FP32 kernel specialized for systems of one dimension
// with uniform charges and candidate slot counts cma, cmb; null if none is
// compiled for that composition
MultiFn multi_kernel_spec(int dim, int cma, int cmb);
int configure_multi(MultiFn f, int precision, size_t smem, int *grid);
int launch_multi_energy(MultiFn f, const MultiDev &m, int precision, int grid, size_t smem, cudaStream_t st);

}  // namespace ewald
