// Persistent multi-system kernels: walkers of several systems (different N,
// cell, dimension and charges, one precision) in one launch.
//
// k_multi_energy_t (multi_kernel.cuh): a host-built list of work items
// (walker x G-run chunk and walker x pair tile) grouped by batch, longest
// first; CTAs take the next item from an atomic counter; after each item the
// CTA bumps its walker's completion counter, and the CTA that completes a
// walker's last item adds up that walker's partial sums (in a fixed order,
// so results do not depend on the schedule or on the other systems in the
// launch).  No CTA ever waits for another one.  This file holds the general
// kernels and the host side; multi_spec.cu the specializations.
#include "multi_kernel.cuh"

namespace ewald {

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

// The kernel for a launch: a specialization for the systems' composition if
// one is compiled (multi_spec.cu), else the general kernel of the precision.
MultiFn multi_kernel(int precision, const std::vector<SysDev> &sys) {
    if (precision == EWALD_FP64) return k_multi_energy_t<double, 0, -1, -1, true>;
    int dim = sys.empty() ? 0 : sys[0].dim, cma = -1, cmb = -1;
    bool uniform = true, two = true;
    for (const SysDev &s : sys) {
        if (s.dim != dim) dim = 0;
        uniform = uniform && s.q_uniform;
        const int cm = mixed_cm(s.cand_max);
        if (cma < 0 || cm == cma) cma = cm;
        else if (cmb < 0 || cm == cmb) cmb = cm;
        else two = false;
    }
    if (dim && uniform && two) {
        if (MultiFn f = multi_kernel_spec(dim, cma, cmb < 0 ? cma : cmb)) return f;
    }
    return k_multi_energy_t<float, 0, -1, -1, true>;
}

int configure_multi(MultiFn f, int precision, size_t smem, int *grid) {
    int dev, sms, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) return e;
    const int threads = precision == EWALD_FP64 ? kMultiThreads64 : kMultiThreads32;
    if ((e = allow_max_smem(f, smem))) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, threads, smem);
    if (e) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    *grid = sms * occ;
    return cudaSuccess;
}

int launch_multi_energy(MultiFn f, const MultiDev &m, int precision, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(m.next, 0, sizeof(int), st);
    if (!e) e = cudaMemsetAsync(m.done, 0, sizeof(int) * (size_t)m.n_walkers, st);
    if (e) return e;
    const int g = std::min(grid, std::max(m.n_items, 1));
    f<<<g, precision == EWALD_FP64 ? kMultiThreads64 : kMultiThreads32, smem, st>>>(m);
    return cudaGetLastError();
}

}  // namespace ewald
