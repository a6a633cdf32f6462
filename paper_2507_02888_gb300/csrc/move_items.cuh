// Single-particle move work as device functions, shared by the per-batch
// propose/accept kernels (move_kernels.cu) and the serving kernel
// (serve_kernels.cu).  Paper Sec. 2.1: VMC and DMC propose one-particle
// moves and need the change of the potential energy:
//
//   dE = q_k sum_{j != k} q_j sum_R [phi(r' - r_j + R) - phi(r - r_j + R)]
//      + sum_{G half} 2 C f(G) (2 Re(conj(rho) delta) + |delta|^2),
//   delta(G) = q_k (e^{iG.r'} - e^{iG.r}),  phi(x) = erfc(alpha|x|)/|x|.
//
// Layered 2D cells (particle k in layer K, weights W_{LL'}(G) of
// Re(rho_L conj(rho_L'))): the reciprocal part is
//   sum_{G half} [2 sum_L' W_{KL'} Re(conj(rho_L') delta) + W_KK |delta|^2].
#pragma once
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
        return ImageSmem<R>::bytes(s, s.dim) + align16((kMoveThreads / 32) * kQueueCapOf<R> * sizeof(QE<R>)) +
               table_bytes(s) + align16((kMoveThreads / 32) * sizeof(double));
    }
    __device__ void carve(unsigned char *base, const SysDev &s, int dim) {
        carve_split(base, base + ImageSmem<R>::bytes(s, dim), s, dim);
    }
    // images at img_base, everything else at work (the serving kernel keeps
    // the images of the last system in place across items)
    __device__ void carve_split(unsigned char *img_base, unsigned char *work, const SysDev &s, int dim) {
        ims.carve(img_base, s, dim);
        unsigned char *base = work;
        size_t off = 0;
        queues = (QE<R> *)(base + off);
        off += align16((kMoveThreads / 32) * kQueueCapOf<R> * sizeof(QE<R>));
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

// This thread's share of the reciprocal dE in a layered cell (particle k of
// layer K), out of line like the layered structure factor.
template <typename R, int DIM>
__device__ __noinline__ R layered_recip_delta(const SysDev &s, const BatchDev &b, int w, int k, R qk,
                                              const MoveTables<R> &tab) {
    const int slots = s.n_runs * s.run_len, nl = s.n_layers, K = s.mob_layer[k];
    const double2 *rho = b.rho + (size_t)w * nl * slots;
    R part = 0;
    for_each_delta<R, DIM>(s, tab, qk, [&](int slot, Cx<R> d) {
        R t = FP<R>::gwl(s, ((size_t)K * nl + K) * slots + slot) * (d.x * d.x + d.y * d.y);
        for (int L = 0; L < nl; ++L) {
            const Cx<R> rv = RhoIO<R>::lead(rho, (size_t)L * slots + slot);
            t += R(2) * FP<R>::gwl(s, ((size_t)K * nl + L) * slots + slot) * (rv.x * d.x + rv.y * d.y);
        }
        part += t;
    });
    return part;
}

// dE of moving particle k of walker w from pold to pnew (tables of m built
// and images staged).  All threads call it; the result is valid in thread 0.
template <typename R, int DIM>
__device__ double move_delta_e(const SysDev &s, const BatchDev &b, int w, int k, const Part<R> &pold,
                               const Part<R> &pnew, MoveSmem<R> &m) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    WarpQueue<R> wq{m.queues + warp * kQueueCapOf<R>, 0, FP<R>::coin2(s), b.status};
    Acc<R> acc;
    // real space: slots (other particle j, old/new), j over mobile != k then fixed
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
        pair_images<R, DIM>(s, which ? pnew : pold, pj, v, which ? R(1) : R(-1), m.ims.img, m.ims.cand, wq, acc,
                            lane);
    }
    wq.drain(acc, FP<R>::term_consts(s), lane);
    double tot = acc.get();
    // reciprocal space
    R part = 0;
    if (DIM == 2 && s.n_layers > 1) {
        part = layered_recip_delta<R, DIM>(s, b, w, k, pold.q, m.tab);
    } else {
        const double2 *rho = b.rho + (size_t)w * s.n_runs * s.run_len;
        for_each_delta<R, DIM>(s, m.tab, pold.q, [&](int slot, Cx<R> d) {
            const Cx<R> rv = RhoIO<R>::lead(rho, slot);
            part += FP<R>::gw(s, slot) * (R(2) * (rv.x * d.x + rv.y * d.y) + d.x * d.x + d.y * d.y);
        });
    }
    tot += (double)part;
    return block_sum(tot, m.red);
}

// rho(G) += delta(G) of walker w's particle k (tables built): the FP64
// running sum (of k's layer in a layered cell).
template <typename R, int DIM>
__device__ void move_apply_rho(const SysDev &s, const BatchDev &b, int w, int k, R qk, const MoveTables<R> &tab) {
    const size_t slots = (size_t)s.n_runs * s.run_len;
    double2 *rho = b.rho + ((size_t)w * s.n_layers + (DIM == 2 && s.n_layers > 1 ? s.mob_layer[k] : 0)) * slots;
    for_each_delta<R, DIM>(s, tab, qk, [&](int slot, Cx<R> d) {
        RhoIO<R>::add(rho, slot, d);
    });
}

}  // namespace ewald
