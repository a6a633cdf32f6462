// Single-particle move kernels: propose (energy change) and accept
// (rho(G) += delta(G), position update).  Paper Sec. 2.1: VMC and DMC propose
// one-particle moves and need the change of the potential energy; with the
// walker's rho(G) resident on the device the change costs O(N + N_G):
//
//   dE = q_k sum_{j != k} q_j sum_R [phi(r' - r_j + R) - phi(r - r_j + R)]
//      + sum_{G half} 2 C f(G) (2 Re(conj(rho) delta) + |delta|^2),
//   delta(G) = q_k (e^{iG.r'} - e^{iG.r}),  phi(x) = erfc(alpha|x|)/|x|.
//
// One CTA per walker.  The powers e^{2 pi i n f_k} of the old and new
// position are computed from exact fixed-point phases (n u mod 2^bits), and
// each thread walks its G runs by one complex multiplication per G.
#include <math.h>

#include "device_common.cuh"

namespace ewald {

template <typename R>
struct MoveTables {
    Cx<R> *P[2][3];  // [old/new][direction]
};

template <typename R, int DIM>
__device__ inline void build_move_tables(const SysDev &s, const typename FP<R>::U *uo,
                                         const typename FP<R>::U *un, MoveTables<R> &t) {
    using U = typename FP<R>::U;
    const int W[3] = {2 * s.n1max + 1, 2 * s.n2max + 1, DIM == 3 ? s.n3max + 1 : 0};
    const int off[3] = {s.n1max, s.n2max, 0};
    const int per = W[0] + W[1] + W[2];
    for (int t2 = threadIdx.x; t2 < 2 * per; t2 += blockDim.x) {
        const int which = t2 / per;
        int rem = t2 - which * per, k = 0;
        while (rem >= W[k]) {
            rem -= W[k];
            ++k;
        }
        const int n = rem - off[k];
        const U u = which ? un[k] : uo[k];
        const U ph = (U)(long long)n * u;  // exact phase modulo one period
        R sn, cs;
        FP<R>::sincospi2(FP<R>::frac(ph), &sn, &cs);
        t.P[which][k][rem] = {cs, sn};
    }
}

// Walk this thread's G runs; for each G compute delta and call f(slot, delta).
template <typename R, int DIM, typename F>
__device__ inline void for_each_delta(const SysDev &s, const MoveTables<R> &t, R qk, F &&f) {
    for (int run = threadIdx.x; run < s.n_runs; run += blockDim.x) {
        const int4 rn = s.runs[run];
        const int dir = rn.w < 0 ? -1 : 1, len = rn.w * dir;
        Cx<R> zo = cmul(t.P[0][0][rn.x + s.n1max], t.P[0][1][rn.y + s.n2max]);
        Cx<R> zn = cmul(t.P[1][0][rn.x + s.n1max], t.P[1][1][rn.y + s.n2max]);
        if (DIM == 3) {
            zo = cmul(zo, t.P[0][2][rn.z]);
            zn = cmul(zn, t.P[1][2][rn.z]);
        }
        const Cx<R> so = t.P[0][0][s.n1max + dir], sn = t.P[1][0][s.n1max + dir];
        for (int r = 0; r < len; ++r) {
            const Cx<R> d = {qk * (zn.x - zo.x), qk * (zn.y - zo.y)};
            f(r * s.n_runs + run, d);
            zo = cmul(zo, so);
            zn = cmul(zn, sn);
        }
    }
}

template <typename R>
struct MoveSmem {
    ImageSmem<R> ims;
    QE<R> *queues;
    MoveTables<R> tab;
    double *red;
    __host__ __device__ static size_t table_bytes(const SysDev &s) {
        int per = (2 * s.n1max + 1) + (2 * s.n2max + 1) + (s.dim == 3 ? s.n3max + 1 : 0);
        return align16(2 * per * sizeof(Cx<R>));
    }
    __host__ __device__ static size_t bytes(const SysDev &s) {
        return ImageSmem<R>::bytes(s, s.dim) + align16((kMoveThreads / 32) * kQueueCap * sizeof(QE<R>)) +
               table_bytes(s) + (kMoveThreads / 32) * sizeof(double);
    }
    __device__ void carve(unsigned char *base, const SysDev &s, int dim) {
        ims.carve(base, s, dim);
        size_t off = ImageSmem<R>::bytes(s, dim);
        queues = (QE<R> *)(base + off);
        off += align16((kMoveThreads / 32) * kQueueCap * sizeof(QE<R>));
        Cx<R> *p = (Cx<R> *)(base + off);
        const int W[3] = {2 * s.n1max + 1, 2 * s.n2max + 1, dim == 3 ? s.n3max + 1 : 0};
        for (int which = 0; which < 2; ++which)
            for (int k = 0; k < 3; ++k) {
                tab.P[which][k] = p;
                p += W[k];
            }
        off += table_bytes(s);
        red = (double *)(base + off);
    }
};

// Fixed-point fractional coordinates of a Cartesian point (same convention
// as the ingest kernel).
template <int DIM>
__device__ inline bool cart_to_fixed(const SysDev &s, const double *r, unsigned long long *u) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        double f = 0;
#pragma unroll
        for (int x = 0; x < DIM; ++x) f += s.Binv[k][x] * r[x];
        if (!isfinite(f)) {
            ok = false;
            f = 0;
        }
        f -= floor(f);
        if (f >= 1.0) f = 0.0;
        u[k] = __double2ull_rz(f * 0x1p64);
    }
    return ok;
}

template <typename R, int DIM>
__global__ void __launch_bounds__(kMoveThreads)
    k_propose(SysDev s, BatchDev b, const int *__restrict__ kk, const double *__restrict__ r_new,
              double *__restrict__ de) {
    using U = typename FP<R>::U;
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ int sk;
    __shared__ unsigned long long su_old[3], su_new[3];
    MoveSmem<R> m;
    m.carve(smem, s, DIM);
    const int w = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        int k = kk[w];
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
    m.ims.stage(s, DIM);
    Part<R> pold, pnew;
    for (int d = 0; d < 3; ++d) {
        pold.u[d] = FP<R>::from64(su_old[d]);
        pnew.u[d] = FP<R>::from64(su_new[d]);
    }
    pold.q = pnew.q = FP<R>::q_mob(s, k);
    build_move_tables<R, DIM>(s, pold.u, pnew.u, m.tab);
    __syncthreads();

    // real space: slots (other particle j, old/new), j over mobile != k then fixed
    WarpQueue<R> wq{m.queues + warp * kQueueCap, 0, FP<R>::coin2(s), b.status};
    Acc<R> acc;
    const int n_other = s.n_mob - 1 + s.n_fix;
    const int total = 2 * n_other;
    for (int base = warp * 32; base < total; base += blockDim.x) {
        const int t = base + lane;
        const bool v = t < total;
        const int jj = t >> 1, which = t & 1;
        Part<R> pj;
        if (!v) pj = load_mobile<R>(s, b, w, s.n_mob, DIM);  // zero particle
        else if (jj < s.n_mob - 1) pj = load_mobile<R>(s, b, w, jj < k ? jj : jj + 1, DIM);
        else pj = load_fixed<R>(s, jj - (s.n_mob - 1), DIM);
        pair_images<R, DIM>(s, which ? pnew : pold, pj, v, which ? R(1) : R(-1), m.ims.img, m.ims.cand,
                            wq, acc, lane);
    }
    wq.drain(acc, FP<R>::term_consts(s), lane);
    double tot = acc.get();

    // reciprocal space
    const double2 *rho = b.rho + (size_t)w * s.n_runs * s.run_len;
    R part = 0;
    for_each_delta<R, DIM>(s, m.tab, pold.q, [&](int slot, Cx<R> d) {
        const double2 rv = rho[slot];
        const R rx = (R)rv.x, ry = (R)rv.y;
        part += FP<R>::gw(s, slot) * (R(2) * (rx * d.x + ry * d.y) + d.x * d.x + d.y * d.y);
    });
    tot += (double)part;
    tot = block_sum(tot, m.red);
    if (tid == 0) de[w] = tot;
}

template <typename R, int DIM>
__global__ void __launch_bounds__(kMoveThreads)
    k_accept(SysDev s, BatchDev b, const unsigned char *__restrict__ acc, int resum_every) {
    extern __shared__ __align__(32) unsigned char smem[];
    MoveSmem<R> m;
    m.carve(smem, s, DIM);
    const int w = blockIdx.x, tid = threadIdx.x;
    const int k = b.pend_k[w];
    if (k < 0 || !acc[w]) {
        __syncthreads();
        if (tid == 0) {
            b.pend_k[w] = -1;
            b.resum_flag[w] = 0;
        }
        return;
    }
    Part<R> pold, pnew;
    for (int d = 0; d < 3; ++d) {
        unsigned long long uo = d < DIM ? b.u[((size_t)w * DIM + d) * s.mob_stride + k] : 0;
        pold.u[d] = FP<R>::from64(uo);
        pnew.u[d] = FP<R>::from64(b.pend_u[(size_t)w * 3 + d]);
    }
    pold.q = FP<R>::q_mob(s, k);
    build_move_tables<R, DIM>(s, pold.u, pnew.u, m.tab);
    __syncthreads();
    double2 *rho = b.rho + (size_t)w * s.n_runs * s.run_len;
    for_each_delta<R, DIM>(s, m.tab, pold.q, [&](int slot, Cx<R> d) {
        double2 rv = rho[slot];
        rv.x += (double)d.x;
        rv.y += (double)d.y;
        rho[slot] = rv;
    });
    __syncthreads();
    if (tid < DIM) b.u[((size_t)w * DIM + tid) * s.mob_stride + k] = b.pend_u[(size_t)w * 3 + tid];
    if (tid == 0) {
        b.pend_k[w] = -1;
        const int c = b.acc_count[w] + 1;
        const bool f = c >= resum_every;
        b.acc_count[w] = f ? 0 : c;
        b.resum_flag[w] = f ? 1 : 0;
    }
}

size_t move_smem_bytes(const SysDev &s, int precision) {
    return precision == EWALD_FP64 ? MoveSmem<double>::bytes(s) : MoveSmem<float>::bytes(s);
}

int configure_move(const SysDev &s, int precision, size_t smem) {
    cudaError_t e;
    auto set = [&](const void *f) {
        return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    };
    if (precision == EWALD_FP64) {
        if (s.dim == 3) {
            if ((e = set((const void *)k_propose<double, 3>))) return e;
            e = set((const void *)k_accept<double, 3>);
        } else {
            if ((e = set((const void *)k_propose<double, 2>))) return e;
            e = set((const void *)k_accept<double, 2>);
        }
    } else {
        if (s.dim == 3) {
            if ((e = set((const void *)k_propose<float, 3>))) return e;
            e = set((const void *)k_accept<float, 3>);
        } else {
            if ((e = set((const void *)k_propose<float, 2>))) return e;
            e = set((const void *)k_accept<float, 2>);
        }
    }
    return e;
}

int launch_propose(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg, const int *k,
                   const double *r_new, double *de, cudaStream_t st) {
    if (precision == EWALD_FP64) {
        if (s.dim == 3) k_propose<double, 3><<<b.W, kMoveThreads, cfg.move_smem, st>>>(s, b, k, r_new, de);
        else k_propose<double, 2><<<b.W, kMoveThreads, cfg.move_smem, st>>>(s, b, k, r_new, de);
    } else {
        if (s.dim == 3) k_propose<float, 3><<<b.W, kMoveThreads, cfg.move_smem, st>>>(s, b, k, r_new, de);
        else k_propose<float, 2><<<b.W, kMoveThreads, cfg.move_smem, st>>>(s, b, k, r_new, de);
    }
    return cudaGetLastError();
}

int launch_accept(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg,
                  const unsigned char *acc, int resum_every, cudaStream_t st) {
    if (precision == EWALD_FP64) {
        if (s.dim == 3) k_accept<double, 3><<<b.W, kMoveThreads, cfg.move_smem, st>>>(s, b, acc, resum_every);
        else k_accept<double, 2><<<b.W, kMoveThreads, cfg.move_smem, st>>>(s, b, acc, resum_every);
    } else {
        if (s.dim == 3) k_accept<float, 3><<<b.W, kMoveThreads, cfg.move_smem, st>>>(s, b, acc, resum_every);
        else k_accept<float, 2><<<b.W, kMoveThreads, cfg.move_smem, st>>>(s, b, acc, resum_every);
    }
    return cudaGetLastError();
}

}  // namespace ewald
