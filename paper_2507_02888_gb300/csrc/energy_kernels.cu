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

#include "device_common.cuh"

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
// One CTA per (walker, chunk of kSfacThreads G runs).  Each thread owns one
// run of <= kRunLen consecutive n1 in a row (n2, n3).  Electrons are staged
// in tiles of te; for each electron of the tile the CTA buffers the powers
// e^{2 pi i n f_k}, n = -n_max..n_max, built by repeated multiplication from
// the base phase (paper Eq. (10)).  A thread then starts its run from the
// product of three buffered powers and steps along n1 by one complex
// multiplication per G.  Tile sums are in R and are added into FP64.
template <typename R, int DIM>
__global__ void __launch_bounds__(kSfacThreads)
    k_sfac(SysDev s, BatchDev b, const unsigned char *__restrict__ only, int te, int write_energy) {
    using C = Cx<R>;
    extern __shared__ __align__(32) unsigned char smem[];
    const int W1 = 2 * s.n1max + 1, W2 = 2 * s.n2max + 1, W3 = DIM == 3 ? s.n3max + 1 : 0;
    Part<R> *tp = (Part<R> *)smem;
    C *P1 = (C *)(smem + align16(te * sizeof(Part<R>)));
    C *P2 = P1 + (size_t)te * W1;
    C *P3 = P2 + (size_t)te * W2;
    double *red = (double *)(smem + align16(te * sizeof(Part<R>)) +
                             align16((size_t)te * (W1 + W2 + W3) * sizeof(C)));

    const int w = blockIdx.x / s.n_gchunks, chunk = blockIdx.x - w * s.n_gchunks;
    if (only && !only[w]) return;  // uniform over the CTA
    const int tid = threadIdx.x;
    const int run = chunk * blockDim.x + tid;
    const bool has = run < s.n_runs;
    const int4 rn = has ? s.runs[run] : make_int4(0, 0, 0, 0);
    double ax[kRunLen], ay[kRunLen];
#pragma unroll
    for (int r = 0; r < kRunLen; ++r) ax[r] = ay[r] = 0;

    for (int e0 = 0; e0 < s.n_mob; e0 += te) {
        const int ne = min(te, s.n_mob - e0);
        for (int t = tid; t < ne; t += blockDim.x) tp[t] = load_mobile<R>(s, b, w, e0 + t, DIM);
        __syncthreads();
        for (int t = tid; t < ne * DIM; t += blockDim.x) {
            const int e = t / DIM, k = t - e * DIM;
            R sn, cs;
            FP<R>::sincospi2(FP<R>::frac(tp[e].u[k]), &sn, &cs);
            const C base = {cs, sn};
            C p = {R(1), R(0)};
            if (k < 2) {
                const int nm = k == 0 ? s.n1max : s.n2max;
                C *P = k == 0 ? P1 + (size_t)e * W1 : P2 + (size_t)e * W2;
                P[nm] = p;
                for (int n = 1; n <= nm; ++n) {
                    p = cmul(p, base);
                    P[nm + n] = p;
                    P[nm - n] = {p.x, -p.y};
                }
            } else {
                C *P = P3 + (size_t)e * W3;
                P[0] = p;
                for (int n = 1; n < W3; ++n) {
                    p = cmul(p, base);
                    P[n] = p;
                }
            }
        }
        __syncthreads();
        R tx[kRunLen], ty[kRunLen];
#pragma unroll
        for (int r = 0; r < kRunLen; ++r) tx[r] = ty[r] = 0;
        if (has) {
            for (int e = 0; e < ne; ++e) {
                const R q = tp[e].q;
                C z = cmul(P1[(size_t)e * W1 + rn.x + s.n1max], P2[(size_t)e * W2 + rn.y + s.n2max]);
                if (DIM == 3) z = cmul(z, P3[(size_t)e * W3 + rn.z]);
                const C step = P1[(size_t)e * W1 + s.n1max + 1];
#pragma unroll
                for (int r = 0; r < kRunLen; ++r) {
                    if (r < rn.w) {
                        tx[r] += q * z.x;
                        ty[r] += q * z.y;
                        z = cmul(z, step);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kRunLen; ++r) {
            ax[r] += (double)tx[r];
            ay[r] += (double)ty[r];
        }
        __syncthreads();
    }

    const int slots = s.n_runs * s.run_len;
    double epart = 0;
    if (has) {
        double2 *rho = b.rho + (size_t)w * slots;
#pragma unroll
        for (int r = 0; r < kRunLen; ++r) {
            if (r < s.run_len) {
                const int slot = r * s.n_runs + run;
                double2 v = make_double2(0.0, 0.0);
                if (r < rn.w) {
                    v.x = ax[r];
                    v.y = ay[r];
                    if (s.rho_fix) {
                        v.x += s.rho_fix[slot].x;
                        v.y += s.rho_fix[slot].y;
                    }
                    epart += s.gw_d[slot] * (v.x * v.x + v.y * v.y);
                }
                rho[slot] = v;
            }
        }
    }
    if (write_energy) {
        double tot = block_sum(epart, red);
        if (tid == 0) b.part_recip[(size_t)w * s.n_gchunks + chunk] = tot;
    }
}

// -------------------------------------------------------------- real space
// Persistent CTAs walk the (walker, tile pair) items.  A tile pair stages
// tile*tile particles; each warp takes 32 x 32 sub-tiles (lane = i, loop over
// j), diagonal tiles only their upper triangle.  Images inside the cutoff
// go through the warp queue; partial sums per item are written in FP64.
template <typename R, int DIM>
__global__ void __launch_bounds__(kRealThreads) k_real(SysDev s, BatchDev b) {
    extern __shared__ __align__(32) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    ImageSmem<R> ims;
    ims.carve(smem, s, DIM);
    size_t off = ImageSmem<R>::bytes(s, DIM);
    Part<R> *ti = (Part<R> *)(smem + off);
    off += align16(s.tile * sizeof(Part<R>));
    Part<R> *tj = (Part<R> *)(smem + off);
    off += align16(s.tile * sizeof(Part<R>));
    QE<R> *qbase = (QE<R> *)(smem + off);
    off += align16(kRealWarps * kQueueCap * sizeof(QE<R>));
    double *red = (double *)(smem + off);

    ims.stage(s, DIM);
    const int S = s.tile / 32;
    const long long total = (long long)b.W * s.n_items;
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        const int w = (int)(item / s.n_items), p = (int)(item - (long long)w * s.n_items);
        const int2 tt = s.items[p];
        const bool fixedj = tt.y >= s.n_mob_tiles;
        const int i0 = tt.x * s.tile;
        const int j0 = (fixedj ? tt.y - s.n_mob_tiles : tt.y) * s.tile;
        const int nj = fixedj ? s.n_fix : s.n_mob;
        __syncthreads();  // previous item's tiles are no longer read
        for (int t = tid; t < s.tile; t += blockDim.x) {
            ti[t] = load_mobile<R>(s, b, w, i0 + t, DIM);
            tj[t] = fixedj ? load_fixed<R>(s, j0 + t, DIM) : load_mobile<R>(s, b, w, j0 + t, DIM);
        }
        __syncthreads();
        WarpQueue<R> wq{qbase + warp * kQueueCap, 0};
        Acc<R> acc;
        const bool diag = !fixedj && tt.x == tt.y;
        const int nst = diag ? S * (S + 1) / 2 : S * S;
        for (int st = warp; st < nst; st += kRealWarps) {
            int a, c;
            if (diag) {
                a = 0;
                int rem = st;
                while (rem >= S - a) {
                    rem -= S - a;
                    ++a;
                }
                c = a + rem;
            } else {
                a = st / S;
                c = st - a * S;
            }
            const Part<R> pi = ti[a * 32 + lane];
            const bool vi = i0 + a * 32 + lane < s.n_mob;
            for (int jj = 0; jj < 32; ++jj) {
                const int lj = c * 32 + jj;
                const bool v = vi && (j0 + lj < nj) && (!(diag && a == c) || lane < jj);
                pair_images<R, DIM>(s, pi, tj[lj], v, R(1), ims.img, ims.cand, ims.cand_len, wq, acc,
                                    lane, b.status);
            }
        }
        wq.drain(acc, FP<R>::term_consts(s), lane);
        double v = warp_sum(acc.get());
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0;
            for (int k = 0; k < kRealWarps; ++k) t += red[k];
            b.part_real[item] = t;
        }
    }
}

// ----------------------------------------------------------------- combine
// E = E_real + E_madR + E_recip + E_self + E_bg (paper Eq. (2)); partial sums
// are added in a fixed order so a walker's result does not depend on how
// the items were scheduled.
__global__ void k_combine(SysDev s, BatchDev b) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= b.W) return;
    double er = 0;
    for (int p = 0; p < s.n_items; ++p) er += b.part_real[(size_t)w * s.n_items + p];
    er += s.e_II;
    double ek = 0;
    for (int c = 0; c < s.n_gchunks; ++c) ek += b.part_recip[(size_t)w * s.n_gchunks + c];
    double *cp = b.comp + (size_t)w * 5;
    cp[0] = er;
    cp[1] = s.e_madR;
    cp[2] = ek;
    cp[3] = s.e_self;
    cp[4] = s.e_bg;
    b.e[w] = er + s.e_madR + ek + s.e_self + s.e_bg;
    b.acc_count[w] = 0;
    b.pend_k[w] = -1;
}

__global__ void k_rho_out(SysDev s, BatchDev b, const int *__restrict__ g2slot, double *__restrict__ out) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)b.W * s.n_gh) return;
    int w = (int)(t / s.n_gh), g = (int)(t - (long long)w * s.n_gh);
    double2 v = b.rho[(size_t)w * s.n_runs * s.run_len + g2slot[g]];
    out[2 * t] = v.x;
    out[2 * t + 1] = v.y;
}

// ---------------------------------------------------------------- launchers
static size_t sfac_smem(const SysDev &s, int precision, int te) {
    size_t part = precision == EWALD_FP64 ? sizeof(Part<double>) : sizeof(Part<float>);
    size_t cx = precision == EWALD_FP64 ? sizeof(Cx<double>) : sizeof(Cx<float>);
    int W = (2 * s.n1max + 1) + (2 * s.n2max + 1) + (s.dim == 3 ? s.n3max + 1 : 0);
    return align16(te * part) + align16((size_t)te * W * cx) + (kSfacThreads / 32) * sizeof(double);
}

static size_t real_smem(const SysDev &s, int precision) {
    if (precision == EWALD_FP64)
        return ImageSmem<double>::bytes(s, s.dim) + 2 * align16(s.tile * sizeof(Part<double>)) +
               align16(kRealWarps * kQueueCap * sizeof(QE<double>)) + kRealWarps * sizeof(double);
    return ImageSmem<float>::bytes(s, s.dim) + 2 * align16(s.tile * sizeof(Part<float>)) +
           align16(kRealWarps * kQueueCap * sizeof(QE<float>)) + kRealWarps * sizeof(double);
}

template <typename F>
static cudaError_t allow_smem(F *f, size_t bytes) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

size_t move_smem_bytes(const SysDev &s, int precision);  // move_kernels.cu
int configure_move(const SysDev &s, int precision, size_t smem);

int configure_launch(const SysDev &s, int precision, LaunchCfg *cfg) {
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    e = cudaDeviceGetAttribute(&cfg->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e) return e;
    // structure factor: the largest electron tile (<= 64) whose tables fit in 96 KB
    int te = 64;
    while (te > 8 && sfac_smem(s, precision, te) > 96 * 1024) te /= 2;
    cfg->sfac_te = te;
    cfg->sfac_smem = sfac_smem(s, precision, te);
    cfg->real_smem = real_smem(s, precision);
    int occ = 0;
    if (precision == EWALD_FP64) {
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
            if ((e = allow_smem(k_real<float, 3>, cfg->real_smem))) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_real<float, 3>, kRealThreads, cfg->real_smem);
        } else {
            if ((e = allow_smem(k_sfac<float, 2>, cfg->sfac_smem))) return e;
            if ((e = allow_smem(k_real<float, 2>, cfg->real_smem))) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_real<float, 2>, kRealThreads, cfg->real_smem);
        }
    }
    if (e) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    cfg->real_grid = cfg->sm_count * occ;
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
        if (s.dim == 3) k_sfac<double, 3><<<grid, kSfacThreads, cfg.sfac_smem, st>>>(s, b, only, cfg.sfac_te, we);
        else k_sfac<double, 2><<<grid, kSfacThreads, cfg.sfac_smem, st>>>(s, b, only, cfg.sfac_te, we);
    } else {
        if (s.dim == 3) k_sfac<float, 3><<<grid, kSfacThreads, cfg.sfac_smem, st>>>(s, b, only, cfg.sfac_te, we);
        else k_sfac<float, 2><<<grid, kSfacThreads, cfg.sfac_smem, st>>>(s, b, only, cfg.sfac_te, we);
    }
    return cudaGetLastError();
}

int launch_real(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg, cudaStream_t st) {
    long long total = (long long)b.W * s.n_items;
    int grid = (int)std::min<long long>(total, cfg.real_grid);
    if (precision == EWALD_FP64) {
        if (s.dim == 3) k_real<double, 3><<<grid, kRealThreads, cfg.real_smem, st>>>(s, b);
        else k_real<double, 2><<<grid, kRealThreads, cfg.real_smem, st>>>(s, b);
    } else {
        if (s.dim == 3) k_real<float, 3><<<grid, kRealThreads, cfg.real_smem, st>>>(s, b);
        else k_real<float, 2><<<grid, kRealThreads, cfg.real_smem, st>>>(s, b);
    }
    return cudaGetLastError();
}

int launch_combine(const SysDev &s, const BatchDev &b, cudaStream_t st) {
    k_combine<<<(b.W + 127) / 128, 128, 0, st>>>(s, b);
    return cudaGetLastError();
}

int launch_rho_out(const SysDev &s, const BatchDev &b, const int *g2slot, double *out, cudaStream_t st) {
    long long n = (long long)b.W * s.n_gh;
    k_rho_out<<<(int)((n + 255) / 256), 256, 0, st>>>(s, b, g2slot, out);
    return cudaGetLastError();
}

}  // namespace ewald
