// Proposed single-particle moves of the tiered FP64 form (EWALD_FP64_TIERED):
// dE of moving particle k of every walker (paper Sec. 2.1) to FP64 accuracy.
// The real-space part is split by term size as in k_real_tiered: FP32
// image tests; the images with erfc(alpha r) above the tier evaluated in
// double-float from the exact fixed-point geometry; the others in FP32 (the
// FP32 image rounding corrected inside the r^2 chain).  The reciprocal part
// is the FP64 form's: FP64 tables from exact phases and rho(G) in FP64.
// Accepting a move is the FP64 form's k_accept.
#include "df_math.cuh"
#include "move_items.cuh"
#include "move_tiered.h"

namespace ewald {

namespace {

struct TieredMoveLayout {
    size_t img_lo, queues, heads, tables, red, total;
};

__host__ __device__ inline TieredMoveLayout tiered_move_layout(const SysDev &s) {
    const int warps = kMoveThreads / 32;
    TieredMoveLayout l;
    size_t off = ImageSmem<float>::bytes(s, s.dim);
    l.img_lo = off;
    off += align16((size_t)(s.n_img + 1) * sizeof(float4));
    l.queues = off;
    off += align16((size_t)warps * kQueueCap * sizeof(QE<float>));
    l.heads = off;
    off += align16((size_t)warps * kHeadCap * sizeof(uint2));
    l.tables = off;
    off += MoveSmem<double>::table_bytes(s);
    l.red = off;
    off += align16((size_t)warps * sizeof(double));
    l.total = off;
    return l;
}

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

template <int DIM>
__global__ void __launch_bounds__(kMoveThreads)
    k_propose_tiered(SysDev s, BatchDev b, const int *__restrict__ kk, const double *__restrict__ r_new,
                     double *__restrict__ de) {
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ int sk;
    __shared__ unsigned long long su_old[3], su_new[3];
    const TieredMoveLayout lay = tiered_move_layout(s);
    ImageSmem<float> ims;
    ims.carve(smem, s, DIM);
    float4 *img_lo = (float4 *)(smem + lay.img_lo);
    QE<float> *queues = (QE<float> *)(smem + lay.queues);
    uint2 *heads = (uint2 *)(smem + lay.heads);
    double *red = (double *)(smem + lay.red);
    MoveTables<double> tab;
    {
        Cx<double> *p = (Cx<double> *)(smem + lay.tables);
        const int W[3] = {2 * s.n1max + 1, 2 * s.n2max + 1, DIM == 3 ? s.n3max + 1 : 0};
        for (int which = 0; which < 2; ++which)
            for (int k = 0; k < 3; ++k) {
                tab.P[which][k] = p;
                p += W[k];
            }
    }
    const int w = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        const int k = kk[w];
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
    ims.stage(s, DIM);
    for (int i = tid; i <= s.n_img; i += blockDim.x) img_lo[i] = s.img_lo_f[i];
    Part<float> pold, pnew;
    for (int d = 0; d < 3; ++d) {
        pold.u[d] = FP<float>::from64(su_old[d]);
        pnew.u[d] = FP<float>::from64(su_new[d]);
        set_lo<float>(pold, d, su_old[d]);
        set_lo<float>(pnew, d, su_new[d]);
    }
    pold.q = pnew.q = FP<float>::q_mob(s, k);
    pold.z = pnew.z = DIM == 2 && s.n_layers > 1 ? FP<float>::z_mob(s, k) : 0.0f;
    {
        const unsigned long long uo[3] = {su_old[0], su_old[1], su_old[2]}, un[3] = {su_new[0], su_new[1], su_new[2]};
        build_move_tables<double, DIM>(s, uo, un, tab);
    }
    __syncthreads();

    // real space: slots t = 2 jj + which, old terms with weight -1
    WarpQueue<float> wq{queues + warp * kQueueCap, 0, FP<float>::coin2(s), b.status};
    HeadQueue hq{heads + warp * kHeadCap, 0};
    Acc<float> acc;
    DF hacc = {0.0f, 0.0f};
    const TermK32 tk = FP<float>::term_consts(s);
    const unsigned lt = (1u << lane) - 1u;
    auto head_flush = [&](uint2 e) {
        const int t = (int)e.x, jj = t >> 1, which = t & 1;
        int g;
        bool fixedp;
        const Part<float> pj = slot_particle<DIM>(s, b, w, k, jj, &g, &fixedp);
        const DF v = head_pair_df<DIM>(s, which ? pnew : pold, pj, k, g, fixedp, ims.img[e.y], img_lo[e.y], b.status);
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
        const unsigned short *lst = ims.cand + geo.sc * s.cand_max;
        for (int c = 0; c < s.cand_max; ++c) {
            const int ic = lst[c];
            const float4 Rv = ims.img[ic], Rl = img_lo[ic];
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
        part = layered_recip_delta<double, DIM>(s, b, w, k, qk, tab);
    } else {
        const double2 *rho = b.rho + (size_t)w * s.n_runs * s.run_len;
        for_each_delta<double, DIM>(s, tab, qk, [&](int slot, Cx<double> d) {
            const double2 rv = rho[slot];
            part += s.gw_d[slot] * (2.0 * (rv.x * d.x + rv.y * d.y) + d.x * d.x + d.y * d.y);
        });
    }
    tot += part;
    tot = block_sum(tot, red);
    if (tid == 0) de[w] = tot;
}

}  // namespace

int launch_propose_tiered(const SysDev &s, const BatchDev &b, const int *k, const double *r_new, double *de,
                          cudaStream_t st) {
    const size_t smem = tiered_move_layout(s).total;
    cudaError_t e;
    if (s.dim == 3) {
        if ((e = allow_max_smem(k_propose_tiered<3>, smem))) return e;
        k_propose_tiered<3><<<b.W, kMoveThreads, smem, st>>>(s, b, k, r_new, de);
    } else {
        if ((e = allow_max_smem(k_propose_tiered<2>, smem))) return e;
        k_propose_tiered<2><<<b.W, kMoveThreads, smem, st>>>(s, b, k, r_new, de);
    }
    return cudaGetLastError();
}

}  // namespace ewald
