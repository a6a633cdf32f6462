// Full-energy kernels: position ingest, structure factor with the
// reciprocal energy, real-space pair sum, and the per-walker combine.
//
// The split into an independent reciprocal loop, an independent real-space
// loop and a final combine follows the paper (Sec. 5.1); the kernels
// themselves are designed for sm_103a: many walkers per launch, G rows owned
// by threads with power recurrences (Sec. 2.3, Eq. (10)), pair tiles staged
// in shared memory, per-warp compaction of the images inside the cutoff,
// and deterministic per-walker reductions in FP64.
#include <math.h>

#include <algorithm>

#include "energy_items.cuh"
#include "real_mixed.cuh"

namespace ewald {

// ------------------------------------------------------------------ ingest
// Cartesian FP64 -> fractional f = B r / 2pi, wrapped to [0, 1) and stored
// as a 64-bit fixed-point fraction (one lattice period = 2^64).
template <int DIM>
__global__ void k_ingest(SysDev s, BatchDev b, const double *__restrict__ pos) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)b.W * s.n_mob) return;
    int w = (int)(t / s.n_mob), i = (int)(t - (long long)w * s.n_mob);
    const double *r = pos + t * DIM;
    double rr[DIM];
#pragma unroll
    for (int x = 0; x < DIM; ++x) rr[x] = r[x];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        double f = 0;
#pragma unroll
        for (int x = 0; x < DIM; ++x) f += s.Binv[k][x] * rr[x];
        if (!isfinite(f)) {
            atomicOr(b.status, ST_NONFINITE);
            f = 0;
        }
        f -= floor(f);
        if (f >= 1.0) f = 0.0;
        b.u[((size_t)w * DIM + k) * s.mob_stride + i] = __double2ull_rz(f * 0x1p64);
    }
}

template <int DIM>
__global__ void k_positions_out(SysDev s, BatchDev b, double *__restrict__ pos) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)b.W * s.n_mob) return;
    int w = (int)(t / s.n_mob), i = (int)(t - (long long)w * s.n_mob);
    double f[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k)
        f[k] = __ull2double_rn(b.u[((size_t)w * DIM + k) * s.mob_stride + i]) * 0x1p-64;
#pragma unroll
    for (int x = 0; x < DIM; ++x) {
        double v = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) v += f[k] * s.A[k][x];
        pos[t * DIM + x] = v;
    }
}

// ------------------------------------------------------- structure factor
// One CTA of s.sfac_threads threads per (walker, chunk of that many G runs);
// see sfac_item.  With
// `only`, walkers whose flag is 0 are skipped (re-sum after accepted moves).
template <typename R, int DIM>
__global__ void __launch_bounds__(kSfacThreads, sizeof(R) == 4 ? kSfacMinBlocks32 : kSfacMinBlocks64)
    k_sfac(SysDev s, BatchDev b, const unsigned char *__restrict__ only, int te, int write_energy) {
    extern __shared__ __align__(32) unsigned char smem[];
    const int w = blockIdx.x / s.n_gchunks, chunk = blockIdx.x - w * s.n_gchunks;
    if (only && !only[w]) return;  // uniform over the CTA
    sfac_item<R, DIM>(s, b, w, chunk, te, write_energy != 0, smem);
}

// The structure factor of the walkers listed in b.resum_list (a count,
// then walker indices), rho only: persistent CTAs over (listed walker,
// chunk) items, so that a re-sum after accepted moves costs in proportion
// to the walkers due, not to the batch.
template <typename R, int DIM>
__global__ void __launch_bounds__(kSfacThreads, sizeof(R) == 4 ? kSfacMinBlocks32 : kSfacMinBlocks64)
    k_sfac_listed(SysDev s, BatchDev b, int te) {
    extern __shared__ __align__(32) unsigned char smem[];
    const int n = b.resum_list[0] * s.n_gchunks;
    for (int it = blockIdx.x; it < n; it += gridDim.x) {
        const int w = b.resum_list[1 + it / s.n_gchunks], chunk = it % s.n_gchunks;
        sfac_item<R, DIM>(s, b, w, chunk, te, false, smem);
    }
}

// -------------------------------------------------------------- real space
// Persistent CTAs walk the (walker, tile pair) items; see real_item.
template <typename R, int DIM>
__global__ void __launch_bounds__(kRealThreads, sizeof(R) == 4 ? kRealMinBlocks32 : kRealMinBlocks64) k_real(SysDev s, BatchDev b) {
    extern __shared__ __align__(32) unsigned char smem[];
    ImageSmem<R> ims;
    ims.carve(smem, s, DIM);
    ims.stage(s, DIM);
    unsigned char *work = smem + ImageSmem<R>::bytes(s, DIM);
    const long long total = (long long)b.W * s.n_items;
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        const int w = (int)(item / s.n_items), p = (int)(item - (long long)w * s.n_items);
        real_item<R, DIM>(s, b, w, p, ims, work);
    }
}

// Tiered FP64 form: FP32 tiles and image tests, head terms in FP64.
template <int DIM>
__global__ void __launch_bounds__(kRealThreads, kRealMinBlocks64) k_real_tiered(SysDev s, BatchDev b) {
    extern __shared__ __align__(32) unsigned char smem[];
    ImageSmem<float> ims;
    ims.carve(smem, s, DIM);
    ims.stage(s, DIM);
    float4 *img_lo = (float4 *)(smem + ImageSmem<float>::bytes(s, DIM));
    for (int i = threadIdx.x; i <= s.n_img; i += blockDim.x) img_lo[i] = s.img_lo_f[i];
    unsigned char *work = smem + ImageSmem<float>::bytes(s, DIM) + align16((s.n_img + 1) * sizeof(float4));
    const long long total = (long long)b.W * s.n_items;
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        const int w = (int)(item / s.n_items), p = (int)(item - (long long)w * s.n_items);
        real_item<float, DIM, true>(s, b, w, p, ims, work, 1, img_lo);
    }
}

// ----------------------------------------------------------------- combine
__global__ void k_combine(SysDev s, BatchDev b) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < b.W) combine_walker(s, b, w);
}

template <typename R>
__global__ void k_rho_out(SysDev s, BatchDev b, const int *__restrict__ g2slot, double *__restrict__ out) {
    // out[W][n_layers][n_gh]: t = (w * n_layers + L) * n_gh + g
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)b.W * s.n_layers * s.n_gh) return;
    const long long wl = t / s.n_gh;
    const int g = (int)(t - wl * s.n_gh);
    const double2 v = RhoIO<R>::get(b.rho, (size_t)wl * s.n_runs * s.run_len + g2slot[g]);
    out[2 * t] = v.x;
    out[2 * t + 1] = v.y;
}

// ---------------------------------------------------------------- launchers
static size_t sfac_smem(const SysDev &s, int precision, int te) { return sfac_bytes(s, precision, te, kSfacThreads); }

static size_t real_smem(const SysDev &s, int precision) {
    if (s.tier2_f > 0)
        return ImageSmem<float>::bytes(s, s.dim) + align16((s.n_img + 1) * sizeof(float4)) +
               real_work_bytes(s, precision, kRealWarps, true);
    if (precision != EWALD_FP64) return MixedImageSmem::bytes(s, s.dim) + mixed_real_work_bytes(s, s.real_warps);
    return ImageSmem<double>::bytes(s, s.dim) + real_work_bytes(s, precision, kRealWarps);
}

template <typename F>
static cudaError_t allow_smem(F *f, size_t bytes) {
    return allow_max_smem(f, bytes);
}

size_t move_smem_bytes(const SysDev &s, int precision);  // move_kernels.cu
int configure_move(const SysDev &s, int precision, size_t smem);

int configure_launch(SysDev &s, int precision, LaunchCfg *cfg) {
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    e = cudaDeviceGetAttribute(&cfg->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e) return e;
    // structure factor: the largest electron tile (<= 64) whose tables fit in 96 KB
    int te = 64;
    while (te > 8 && sfac_smem(s, precision, te) > 96 * 1024) te /= 2;
    cfg->sfac_te = te;
    s.sfac_te = te;
    cfg->sfac_smem = sfac_smem(s, precision, te);
    cfg->real_smem = real_smem(s, precision);
    {   // the listed structure factor: persistent CTAs, as many as fit
        int so = 0;
        if (precision == EWALD_FP64) {
            e = s.dim == 3 ? allow_smem(k_sfac_listed<double, 3>, cfg->sfac_smem) : allow_smem(k_sfac_listed<double, 2>, cfg->sfac_smem);
            if (!e) e = s.dim == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&so, k_sfac_listed<double, 3>, s.sfac_threads, cfg->sfac_smem)
                                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&so, k_sfac_listed<double, 2>, s.sfac_threads, cfg->sfac_smem);
        } else {
            e = s.dim == 3 ? allow_smem(k_sfac_listed<float, 3>, cfg->sfac_smem) : allow_smem(k_sfac_listed<float, 2>, cfg->sfac_smem);
            if (!e) e = s.dim == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&so, k_sfac_listed<float, 3>, s.sfac_threads, cfg->sfac_smem)
                                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&so, k_sfac_listed<float, 2>, s.sfac_threads, cfg->sfac_smem);
        }
        if (e) return e;
        cfg->sfac_grid = cfg->sm_count * std::max(so, 1);
    }
    int occ = 0;
    if (s.tier2_f > 0) {  // tiered FP64: FP64 structure factor, tiered real space
        if (s.dim == 3) {
            if ((e = allow_smem(k_sfac<double, 3>, cfg->sfac_smem))) return e;
            if ((e = allow_smem(k_real_tiered<3>, cfg->real_smem))) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_real_tiered<3>, kRealThreads, cfg->real_smem);
        } else {
            if ((e = allow_smem(k_sfac<double, 2>, cfg->sfac_smem))) return e;
            if ((e = allow_smem(k_real_tiered<2>, cfg->real_smem))) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_real_tiered<2>, kRealThreads, cfg->real_smem);
        }
    } else if (precision == EWALD_FP64) {
        if (s.dim == 3) {
            if ((e = allow_smem(k_sfac<double, 3>, cfg->sfac_smem))) return e;
            if ((e = allow_smem(k_real<double, 3>, cfg->real_smem))) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_real<double, 3>, kRealThreads, cfg->real_smem);
        } else {
            if ((e = allow_smem(k_sfac<double, 2>, cfg->sfac_smem))) return e;
            if ((e = allow_smem(k_real<double, 2>, cfg->real_smem))) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_real<double, 2>, kRealThreads, cfg->real_smem);
        }
    } else {
        if (s.dim == 3) {
            if ((e = allow_smem(k_sfac<float, 3>, cfg->sfac_smem))) return e;
        } else {
            if ((e = allow_smem(k_sfac<float, 2>, cfg->sfac_smem))) return e;
        }
        e = (cudaError_t)configure_real_mixed(s, cfg->real_smem, &occ);
    }
    if (e) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    cfg->real_grid = cfg->sm_count * occ;
    cfg->propose_grid = 0;
    if (precision == EWALD_MIXED && (e = (cudaError_t)configure_propose_mixed(s, cfg->sm_count, &cfg->propose_grid)))
        return e;
    cfg->move_smem = move_smem_bytes(s, precision);
    return configure_move(s, precision, cfg->move_smem);
}

int launch_ingest(const SysDev &s, const BatchDev &b, const double *pos, cudaStream_t st) {
    long long n = (long long)b.W * s.n_mob;
    int grid = (int)((n + 255) / 256);
    if (s.dim == 3) k_ingest<3><<<grid, 256, 0, st>>>(s, b, pos);
    else k_ingest<2><<<grid, 256, 0, st>>>(s, b, pos);
    return cudaGetLastError();
}

int launch_positions_out(const SysDev &s, const BatchDev &b, double *pos, cudaStream_t st) {
    long long n = (long long)b.W * s.n_mob;
    int grid = (int)((n + 255) / 256);
    if (s.dim == 3) k_positions_out<3><<<grid, 256, 0, st>>>(s, b, pos);
    else k_positions_out<2><<<grid, 256, 0, st>>>(s, b, pos);
    return cudaGetLastError();
}

int launch_sfac(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg,
                const unsigned char *only, cudaStream_t st) {
    int grid = b.W * s.n_gchunks;
    int we = only ? 0 : 1;
    if (precision == EWALD_FP64) {
        if (s.dim == 3) k_sfac<double, 3><<<grid, s.sfac_threads, cfg.sfac_smem, st>>>(s, b, only, cfg.sfac_te, we);
        else k_sfac<double, 2><<<grid, s.sfac_threads, cfg.sfac_smem, st>>>(s, b, only, cfg.sfac_te, we);
    } else {
        if (s.dim == 3) k_sfac<float, 3><<<grid, s.sfac_threads, cfg.sfac_smem, st>>>(s, b, only, cfg.sfac_te, we);
        else k_sfac<float, 2><<<grid, s.sfac_threads, cfg.sfac_smem, st>>>(s, b, only, cfg.sfac_te, we);
    }
    return cudaGetLastError();
}

int launch_sfac_listed(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg, cudaStream_t st) {
    if (precision == EWALD_FP64) {
        if (s.dim == 3) k_sfac_listed<double, 3><<<cfg.sfac_grid, s.sfac_threads, cfg.sfac_smem, st>>>(s, b, cfg.sfac_te);
        else k_sfac_listed<double, 2><<<cfg.sfac_grid, s.sfac_threads, cfg.sfac_smem, st>>>(s, b, cfg.sfac_te);
    } else {
        if (s.dim == 3) k_sfac_listed<float, 3><<<cfg.sfac_grid, s.sfac_threads, cfg.sfac_smem, st>>>(s, b, cfg.sfac_te);
        else k_sfac_listed<float, 2><<<cfg.sfac_grid, s.sfac_threads, cfg.sfac_smem, st>>>(s, b, cfg.sfac_te);
    }
    return cudaGetLastError();
}

int launch_real(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg, cudaStream_t st) {
    long long total = (long long)b.W * s.n_items;
    int grid = (int)std::min<long long>(total, cfg.real_grid);
    if (s.tier2_f > 0) {
        if (s.dim == 3) k_real_tiered<3><<<grid, kRealThreads, cfg.real_smem, st>>>(s, b);
        else k_real_tiered<2><<<grid, kRealThreads, cfg.real_smem, st>>>(s, b);
    } else if (precision == EWALD_FP64) {
        if (s.dim == 3) k_real<double, 3><<<grid, kRealThreads, cfg.real_smem, st>>>(s, b);
        else k_real<double, 2><<<grid, kRealThreads, cfg.real_smem, st>>>(s, b);
    } else {
        return launch_real_mixed(s, b, grid, cfg.real_smem, st);
    }
    return cudaGetLastError();
}

int launch_combine(const SysDev &s, const BatchDev &b, cudaStream_t st) {
    k_combine<<<(b.W + 127) / 128, 128, 0, st>>>(s, b);
    return cudaGetLastError();
}

int launch_rho_out(const SysDev &s, const BatchDev &b, int precision, const int *g2slot, double *out,
                   cudaStream_t st) {
    long long n = (long long)b.W * s.n_layers * s.n_gh;
    if (precision == EWALD_FP64) k_rho_out<double><<<(int)((n + 255) / 256), 256, 0, st>>>(s, b, g2slot, out);
    else k_rho_out<float><<<(int)((n + 255) / 256), 256, 0, st>>>(s, b, g2slot, out);
    return cudaGetLastError();
}

}  // namespace ewald
