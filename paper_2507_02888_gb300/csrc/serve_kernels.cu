// Serving kernel: one launch advances every walker of every active request
// by one single-particle move (propose + accept fused), whatever system the
// request belongs to.  Work items (request slot, walker) are taken from an
// atomic counter; each walker's computation depends only on its own state
// and its request's move stream, so a request's results are the same alone
// and mixed with others.
//
// Moves come from a counter-based generator: draw c of a request is output
// c of a SplitMix64 stream (Steele, Lea & Flood, OOPSLA 2014) seeded with the
// request's seed, c = ((step << 32) + walker) * 8 + j.  j = 0 picks the
// particle, j = 1..4 give two Box-Muller pairs for the displacement, j = 5
// decides acceptance (no wave function here).
#include "energy_items.cuh"
#include "move_items.cuh"
#include "move_tiered.cuh"
#include "serve.h"

namespace ewald {

__device__ inline unsigned long long splitmix_out(unsigned long long seed, unsigned long long c) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (c + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ inline double uniform53(unsigned long long x) { return (double)(x >> 11) * 0x1p-53; }

template <typename T>
__device__ inline void cta_copy_words(T *dst, const T *src) {
    const int *s = (const int *)src;
    int *d = (int *)dst;
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
}

// TIER (R = double): the tiered FP64 form, dE by tiered_delta_e.
template <typename R, bool TIER>
__global__ void __launch_bounds__(kMoveThreads, kServeMinBlocks) k_serve_step(ServeDev sv) {
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ SysDev ss;
    __shared__ SlotDev sl;
    __shared__ int s_item, s_img_sys, s_slot, s_k, s_acc, s_resum;
    __shared__ unsigned long long s_uold[3], s_unew[3], s_x[6];
    __shared__ double s_g[4];
    if (threadIdx.x == 0) s_img_sys = s_slot = -1;
    const int n_items = *sv.n_items;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(sv.next, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int2 d = sv.items[it];  // (slot, walker)
        if (d.x != s_slot) {          // uniform over the CTA; items come slot by slot
            cta_copy_words(&sl, sv.slots + d.x);
            __syncthreads();
            cta_copy_words(&ss, sv.sys + sl.sys);
            __syncthreads();
            if (threadIdx.x == 0) s_slot = d.x;
        }
        const int w = d.y, dim = ss.dim;
        MoveSmem<R> m;
        TieredMoveSmem tm;
        if constexpr (TIER) tm.carve_split(smem, smem + sv.img_bytes, ss, dim);
        else m.carve_split(smem, smem + sv.img_bytes, ss, dim);
        if (s_img_sys != sl.sys) {  // uniform over the CTA
            if constexpr (TIER) tm.stage(ss, dim);
            else m.ims.stage(ss, dim);
            __syncthreads();
            if (threadIdx.x == 0) s_img_sys = sl.sys;
        }
        // the walker's six draws of this step, one per thread, then the two
        // Box-Muller pairs on two threads
        const unsigned long long c0 = (((unsigned long long)sl.step << 32) + (unsigned long long)w) * 8ull;
        if (threadIdx.x < 6) s_x[threadIdx.x] = splitmix_out(sl.seed, c0 + threadIdx.x);
        __syncthreads();
        if (threadIdx.x < 2) {
            const int p = threadIdx.x;
            const double u1 = uniform53(s_x[1 + 2 * p]), u2 = uniform53(s_x[2 + 2 * p]);
            const double rad = sqrt(-2.0 * log(1.0 - u1));
            double sn, cs;
            sincospi(2.0 * u2, &sn, &cs);
            s_g[2 * p] = rad * cs;
            s_g[2 * p + 1] = rad * sn;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int k = (int)(((s_x[0] >> 32) * (unsigned long long)ss.n_mob) >> 32);
            const double ua = uniform53(s_x[5]);
            // current Cartesian position of particle k, displaced
            double f[3] = {0, 0, 0}, r[3] = {0, 0, 0};
            for (int q = 0; q < dim; ++q) {
                s_uold[q] = sl.b.u[((size_t)w * dim + q) * ss.mob_stride + k];
                f[q] = __ull2double_rn(s_uold[q]) * 0x1p-64;
            }
            for (int x = 0; x < dim; ++x) {
                for (int q = 0; q < dim; ++q) r[x] += f[q] * ss.A[q][x];
                r[x] += sl.sigma * s_g[x];
            }
            unsigned long long un[3] = {0, 0, 0};
            for (int q = 0; q < dim; ++q) {
                double fr = 0;
                for (int x = 0; x < dim; ++x) fr += ss.Binv[q][x] * r[x];
                fr -= floor(fr);
                if (fr >= 1.0) fr = 0.0;
                un[q] = __double2ull_rz(fr * 0x1p64);
            }
            for (int q = 0; q < 3; ++q) {
                s_unew[q] = un[q];
                if (q >= dim) s_uold[q] = 0;
            }
            s_k = k;
            s_acc = ua < sl.accept_p ? 1 : 0;
        }
        __syncthreads();
        const int k = s_k;
        const R qk = FP<R>::q_mob(ss, k);
        double de;
        if constexpr (TIER) {
            const unsigned long long uo[3] = {s_uold[0], s_uold[1], s_uold[2]};
            const unsigned long long un[3] = {s_unew[0], s_unew[1], s_unew[2]};
            Part<float> po, pn;
            if (dim == 3) {
                tiered_move_parts<3>(ss, k, uo, un, po, pn);
                build_move_tables<double, 3>(ss, uo, un, tm.tab);
            } else {
                tiered_move_parts<2>(ss, k, uo, un, po, pn);
                build_move_tables<double, 2>(ss, uo, un, tm.tab);
            }
            __syncthreads();
            de = dim == 3 ? tiered_delta_e<3>(ss, sl.b, w, k, po, pn, tm) : tiered_delta_e<2>(ss, sl.b, w, k, po, pn, tm);
        } else {
            Part<R> pold, pnew;
            for (int q = 0; q < 3; ++q) {
                pold.u[q] = FP<R>::from64(s_uold[q]);
                pnew.u[q] = FP<R>::from64(s_unew[q]);
                set_lo<R>(pold, q, s_uold[q]);
                set_lo<R>(pnew, q, s_unew[q]);
            }
            pold.q = pnew.q = qk;
            if (dim == 2) {  // after the coordinates: the FP64 height shares the third word
                const R z = ss.n_layers > 1 ? FP<R>::z_mob(ss, k) : R(0);
                set_part_z(pold, z);
                set_part_z(pnew, z);
            }
            if (dim == 3) build_move_tables<R, 3>(ss, pold.u, pnew.u, m.tab);
            else build_move_tables<R, 2>(ss, pold.u, pnew.u, m.tab);
            __syncthreads();
            de = dim == 3 ? move_delta_e<R, 3>(ss, sl.b, w, k, pold, pnew, m)
                          : move_delta_e<R, 2>(ss, sl.b, w, k, pold, pnew, m);
        }
        if (s_acc) {  // uniform over the CTA
            const MoveTables<R> *tab;
            if constexpr (TIER) tab = &tm.tab;
            else tab = &m.tab;
            if (dim == 3) move_apply_rho<R, 3>(ss, sl.b, w, k, qk, *tab);
            else move_apply_rho<R, 2>(ss, sl.b, w, k, qk, *tab);
            __syncthreads();
            if (threadIdx.x < dim) sl.b.u[((size_t)w * dim + threadIdx.x) * ss.mob_stride + k] = s_unew[threadIdx.x];
            if (threadIdx.x == 0) {
                sl.b.e[w] += de;
                sv.n_acc[sl.walker_base + w] += 1;
                const int c = sl.b.acc_count[w] + 1;
                s_resum = c >= sl.resum_every;
                sl.b.acc_count[w] = s_resum ? 0 : c;
            }
            __syncthreads();
            if (s_resum) {  // rebuild this walker's rho(G) from its positions, in this CTA
                for (int chunk = 0; chunk < ss.n_gchunks; ++chunk) {
                    if (dim == 3) sfac_item<R, 3>(ss, sl.b, w, chunk, ss.sfac_te, false, smem + sv.img_bytes);
                    else sfac_item<R, 2>(ss, sl.b, w, chunk, ss.sfac_te, false, smem + sv.img_bytes);
                    __syncthreads();
                }
            }
        }
    }
}

// precision: EWALD_FP64, EWALD_MIXED or EWALD_FP64_TIERED (the tiered
// kernel; its in-kernel re-sums are the FP64 structure factor's)
size_t serve_smem(const std::vector<SysDev> &sys, int precision, size_t *img_bytes) {
    size_t img = 0, work = 0;
    for (const SysDev &s : sys) {
        if (precision == EWALD_FP64_TIERED) {
            img = std::max(img, TieredMoveSmem::img_bytes(s));
            work = std::max(work, TieredMoveSmem::work_bytes(s));
        } else if (precision == EWALD_FP64) {
            img = std::max(img, ImageSmem<double>::bytes(s, s.dim));
            work = std::max(work, MoveSmem<double>::bytes(s) - ImageSmem<double>::bytes(s, s.dim));
        } else {
            img = std::max(img, ImageSmem<float>::bytes(s, s.dim));
            work = std::max(work, MoveSmem<float>::bytes(s) - ImageSmem<float>::bytes(s, s.dim));
        }
        const int sp = precision == EWALD_MIXED ? EWALD_MIXED : EWALD_FP64;
        work = std::max(work, sfac_bytes(s, sp, s.sfac_te, kMoveThreads));
    }
    *img_bytes = img;
    return img + work;
}

template <typename R, bool TIER>
static cudaError_t configure_one(size_t smem, int *occ) {
    cudaError_t e = allow_max_smem(k_serve_step<R, TIER>, smem);
    if (e) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_serve_step<R, TIER>, kMoveThreads, smem);
}

int configure_serve(int precision, size_t smem, int *grid) {
    int dev, sms, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) return e;
    if (precision == EWALD_FP64_TIERED) e = configure_one<double, true>(smem, &occ);
    else if (precision == EWALD_FP64) e = configure_one<double, false>(smem, &occ);
    else e = configure_one<float, false>(smem, &occ);
    if (e) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    *grid = sms * occ;
    return cudaSuccess;
}

int launch_serve_step(const ServeDev &d, int precision, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d.next, 0, sizeof(int), st);
    if (e) return e;
    if (precision == EWALD_FP64_TIERED) k_serve_step<double, true><<<grid, kMoveThreads, smem, st>>>(d);
    else if (precision == EWALD_FP64) k_serve_step<double, false><<<grid, kMoveThreads, smem, st>>>(d);
    else k_serve_step<float, false><<<grid, kMoveThreads, smem, st>>>(d);
    return cudaGetLastError();
}

}  // namespace ewald
