// Single-particle move energy change of the tiered FP64 form
// (EWALD_FP64_TIERED), shared by the per-batch propose kernel
// (move_tiered.cu) and the serving kernel (serve_kernels.cu): dE of moving
// particle k of a walker (paper Sec. 2.1) to FP64 accuracy.  The real-space
// part is split by term size as in k_real_tiered: FP32 image tests; the
// images with erfc(alpha r) above the tier evaluated in double-float from
// the exact fixed-point geometry; the others in FP32 (the FP32 image
// rounding corrected inside the r^2 chain).  The reciprocal part is the
// FP64 form's: FP64 tables from exact phases and rho(G) in FP64, so
// accepting a move is the FP64 form's rho update.
#pragma once
#include "df_math.cuh"
#include "move_items.cuh"

namespace ewald {

// Shared memory of one walker's tiered move: the FP32 images with their
// rounding (img_lo), per-warp FP32 and head queues, FP64 phase tables and the
// block reduction.  Images at img_base, the rest at work, as MoveSmem.
struct TieredMoveSmem {
    ImageSmem<float> ims;
    float4 *img_lo;
    QE<float> *queues;
    uint2 *heads;
    MoveTables<double> tab;
    double *red;
    __host__ __device__ static size_t img_bytes(const SysDev &s) {
        return ImageSmem<float>::bytes(s, s.dim) + align16((size_t)(s.n_img + 1) * sizeof(float4));
    }
    __host__ __device__ static size_t work_bytes(const SysDev &s) {
        const size_t warps = kMoveThreads / 32;
        return align16(warps * kQueueCap32 * sizeof(QE<float>)) + align16(warps * kHeadCap * sizeof(uint2)) +
               MoveSmem<double>::table_bytes(s) + align16(warps * sizeof(double));
    }
    __host__ __device__ static size_t bytes(const SysDev &s) { return img_bytes(s) + work_bytes(s); }
    __device__ void carve_split(unsigned char *img_base, unsigned char *work, const SysDev &s, int dim) {
        ims.carve(img_base, s, dim);
        img_lo = (float4 *)(img_base + ImageSmem<float>::bytes(s, dim));
        const size_t warps = kMoveThreads / 32;
        size_t off = 0;
        queues = (QE<float> *)(work + off);
        off += align16(warps * kQueueCap32 * sizeof(QE<float>));
        heads = (uint2 *)(work + off);
        off += align16(warps * kHeadCap * sizeof(uint2));
        Cx<double> *p = (Cx<double> *)(work + off);
        const int W[3] = {2 * s.n1max + 1, 2 * s.n2max + 1, dim == 3 ? s.n3max + 1 : 0};
        for (int which = 0; which < 2; ++which)
            for (int k = 0; k < 3; ++k) {
                tab.P[which][k] = p;
                p += W[k];
            }
        off += MoveSmem<double>::table_bytes(s);
        red = (double *)(work + off);
    }
    __device__ void stage(const SysDev &s, int dim) {
        ims.stage(s, dim);
        for (int i = threadIdx.x; i <= s.n_img; i += blockDim.x) img_lo[i] = s.img_lo_f[i];
    }
};

// The double-float term of a head image between particle a (mobile index ka,
// the moving one) and particle b (mobile index jb, or fixed if bfixed)
template <int DIM>
__device__ inline DF head_pair_df(const SysDev &s, const Part<float> &a, const Part<float> &b, int ka, int jb,
                                  bool bfixed, const float4 &Rh, const float4 &Rl, int *status) {
    DF y[3] = {{Rh.x, Rl.x}, {Rh.y, Rl.y}, {Rh.z, Rl.z}};
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const unsigned long long ua = ((unsigned long long)a.u[k] << 32) | a.lo[k];
        const unsigned long long ub = ((unsigned long long)b.u[k] << 32) | b.lo[k];
        const DF f = df_from_fixed((long long)(ua - ub));
#pragma unroll
        for (int x = 0; x < DIM; ++x) y[x] = df_fma(f, DF{s.A32[k][x], s.A32lo[k][x]}, y[x]);
    }
    DF r2 = {0.0f, 0.0f};
    if (DIM == 2 && s.n_layers > 1) {
        const double dz = s.z_mob[ka] - (bfixed ? s.z_fix[jb] : s.z_mob[jb]);
        r2 = df_from(dz * dz);
    }
#pragma unroll
    for (int x = 0; x < DIM; ++x) r2 = df_fma(y[x], y[x], r2);
    if (r2.h < s.coin2_f) {
        atomicOr(status, ST_COINCIDENT);
        return DF{0.0f, 0.0f};
    }
    const DF rinv = df_rsqrt(r2);
    const DF xa = df_mul(DF{s.alpha_f, s.alpha_lo_f}, df_mul(r2, rinv));
    const float2 qa = s.q_mob_df[ka], qb = bfixed ? s.q_fix_df[jb] : s.q_mob_df[jb];
    const DF w = df_mul(DF{qa.x, qa.y}, DF{qb.x, qb.y});
    return df_mul(df_mul(w, df_erfc(xa)), rinv);
}

// The other particle of real-space slot t = 2 jj + which (jj over the mobile
// particles but k, then the fixed ones): its FP32 record and global index.
template <int DIM>
__device__ inline Part<float> slot_particle(const SysDev &s, const BatchDev &b, int w, int k, int jj, int *g,
                                            bool *fixedp) {
    if (jj < s.n_mob - 1) {
        *g = jj < k ? jj : jj + 1;
        *fixedp = false;
        return load_mobile<float>(s, b, w, *g, DIM);
    }
    *g = jj - (s.n_mob - 1);
    *fixedp = true;
    return load_fixed<float>(s, *g, DIM);
}

// The FP32 records of particle k at its old and new fixed-point positions.
template <int DIM>
__device__ inline void tiered_move_parts(const SysDev &s, int k, const unsigned long long *uo,
                                         const unsigned long long *un, Part<float> &pold, Part<float> &pnew) {
    for (int d = 0; d < 3; ++d) {
        pold.u[d] = FP<float>::from64(uo[d]);
        pnew.u[d] = FP<float>::from64(un[d]);
        set_lo<float>(pold, d, uo[d]);
        set_lo<float>(pnew, d, un[d]);
    }
    pold.q = pnew.q = FP<float>::q_mob(s, k);
    pold.z = pnew.z = DIM == 2 && s.n_layers > 1 ? FP<float>::z_mob(s, k) : 0.0f;
}

// dE of moving particle k of walker w from pold to pnew (tables of m built
// and images staged).  All threads call it; the result is valid in thread 0.
template <int DIM>
__device__ double tiered_delta_e(const SysDev &s, const BatchDev &b, int w, int k, const Part<float> &pold,
                                 const Part<float> &pnew, TieredMoveSmem &m) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // real space: slots t = 2 jj + which, old terms with weight -1
    WarpQueue<float> wq{m.queues + warp * kQueueCap32, 0, FP<float>::coin2(s), b.status};
    HeadQueue hq{m.heads + warp * kHeadCap, 0};
    Acc<float> acc;
    DF hacc = {0.0f, 0.0f};
    const TermK32 tk = FP<float>::term_consts(s);
    const unsigned lt = (1u << lane) - 1u;
    auto head_flush = [&](uint2 e) {
        const int t = (int)e.x, jj = t >> 1, which = t & 1;
        int g;
        bool fixedp;
        const Part<float> pj = slot_particle<DIM>(s, b, w, k, jj, &g, &fixedp);
        const DF v = head_pair_df<DIM>(s, which ? pnew : pold, pj, k, g, fixedp, m.ims.img[e.y], m.img_lo[e.y],
                                       b.status);
        hacc = df_add(hacc, which ? v : DF{-v.h, -v.l});
    };
    const int total = 2 * (s.n_mob - 1 + s.n_fix);
    for (int base = warp * 32; base < total; base += blockDim.x) {
        const int t = base + lane;
        const bool v = t < total;
        const int which = t & 1;
        int g = 0;
        bool fixedp = false;
        const Part<float> pj = v ? slot_particle<DIM>(s, b, w, k, t >> 1, &g, &fixedp)
                                 : load_mobile<float>(s, b, w, s.n_mob, DIM);  // a zero particle
        const Part<float> &pa = which ? pnew : pold;
        const PairGeom<float, DIM> geo = pair_geom<float, DIM>(s, pa, pj);
        const float wgt = (which ? 1.0f : -1.0f) * pa.q * pj.q;
        const float rc2 = v ? s.rc2_f : 0.0f;
        const unsigned short *lst = m.ims.cand + geo.sc * s.cand_max;
        for (int c = 0; c < s.cand_max; ++c) {
            const int ic = lst[c];
            const float4 Rv = m.ims.img[ic], Rl = m.img_lo[ic];
            const float y0 = __fadd_rn(geo.x[0], Rv.x), y1 = __fadd_rn(geo.x[1], Rv.y);
            const float y2 = DIM == 3 ? __fadd_rn(geo.x[DIM - 1], Rv.z) : 0.0f;
            float cr = __fmaf_rn(y1, Rl.y, __fmul_rn(y0, Rl.x));
            if (DIM == 3) cr = __fmaf_rn(y2, Rl.z, cr);
            float r2 = __fmaf_rn(y1, y1, __fmaf_rn(y0, y0, __fmaf_rn(2.0f, cr, geo.z2)));
            if (DIM == 3) r2 = __fmaf_rn(y2, y2, r2);
            const bool pass = r2 < rc2;
            const bool head = pass && r2 < s.tier2_f;
            const unsigned hb = __ballot_sync(0xffffffffu, head);
            if (head) hq.q[hq.n + __popc(hb & lt)] = make_uint2((unsigned)t, (unsigned)ic);
            hq.n += __popc(hb);
            if (hq.n >= 32) {
                __syncwarp();
                head_flush(hq.q[hq.n - 32 + lane]);
                hq.n -= 32;
                __syncwarp();
            }
            wq.push(pass && !head, r2, wgt, acc, tk, lane);
        }
    }
    wq.drain(acc, tk, lane);
    __syncwarp();
    if (lane < hq.n) head_flush(hq.q[lane]);
    __syncwarp();
    double tot = acc.get() + df_to(hacc);

    // reciprocal space, FP64
    double part = 0;
    const double qk = FP<double>::q_mob(s, k);
    if (DIM == 2 && s.n_layers > 1) {
        part = layered_recip_delta<double, DIM>(s, b, w, k, qk, m.tab);
    } else {
        const double2 *rho = b.rho + (size_t)w * s.n_runs * s.run_len;
        for_each_delta<double, DIM>(s, m.tab, qk, [&](int slot, Cx<double> d) {
            const double2 rv = rho[slot];
            part += s.gw_d[slot] * (2.0 * (rv.x * d.x + rv.y * d.y) + d.x * d.x + d.y * d.y);
        });
    }
    tot += part;
    return block_sum(tot, m.red);
}

}  // namespace ewald
