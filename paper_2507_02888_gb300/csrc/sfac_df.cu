// Structure factor of the tiered FP64 form (EWALD_FP64_TIERED) in double-
// float arithmetic: rho(G) = sum_i q_i e^{iG.r_i} and the reciprocal energy
// (paper Eq. (3) / Eq. (5), powers of e^{i b_k.r} buffered as in Eq. (10)),
// to FP64 accuracy on GB300's FP32 pipe.
//
// A double-float is an unevaluated pair hi + lo of floats (48 significant
// bits).  Products use the exact FMA residual of hi * hi plus the cross
// terms, sums Knuth's two-sum, each result renormalised by a fast two-sum
// (Dekker 1971; the standard double-float arithmetic).  A complex
// multiply-and-walk step costs ~40 FP32 operations against 4 FP64 ones,
// which GB300 runs ~70x slower than FP32 ones.
//
// The power tables start from one FP64 sincospi of the exact fixed-point
// phase per electron and axis and are built in double-float by binary
// splitting; each thread then starts its run from the product of three
// table entries and walks up to kRunLen G by double-float complex
// multiplication, two electrons side by side, with double-float slot sums.
// Errors: ~2^-46 per operation, chains of at most ~20 operations, so rho(G)
// carries ~1e-13 of relative error, inside the FP64 form's 1e-12 bound.
#include <algorithm>

#include "df_math.cuh"
#include "energy_items.cuh"
#include "sfac_df.h"

namespace ewald {

struct SfacTileDF {
    const Part<double> *tp;
    const CDF *P1, *P2, *P3;
    int W1, W2, W3, n1max, n2max, ne;
};

template <int DIM, int L>
__device__ __forceinline__ void sfac_runs_df(const SfacTileDF &t, int4 rn, int dir, DF *ax, DF *ay) {
    auto start = [&](int e, CDF &z, CDF &step) {
        z = cdf_mul(t.P1[(size_t)e * t.W1 + rn.x + t.n1max], t.P2[(size_t)e * t.W2 + rn.y + t.n2max]);
        if (DIM == 3) z = cdf_mul(z, t.P3[(size_t)e * t.W3 + rn.z]);
        const double qb = t.tp[e].q;  // the charge as a double-float, stored in the slot of q
        const DF q = {__int_as_float(__double2hiint(qb)), __int_as_float(__double2loint(qb))};
        z = {df_mul(z.x, q), df_mul(z.y, q)};
        step = t.P1[(size_t)e * t.W1 + t.n1max + dir];
    };
    int e = 0;
    for (; e + 1 < t.ne; e += 2) {
        CDF za, sa, zb, sb;
        start(e, za, sa);
        start(e + 1, zb, sb);
#pragma unroll
        for (int r = 0; r < L; ++r) {
            if (r < rn.w) {
                ax[r] = df_add(ax[r], df_add(za.x, zb.x));
                ay[r] = df_add(ay[r], df_add(za.y, zb.y));
                if (r + 1 < L) {
                    za = cdf_mul(za, sa);
                    zb = cdf_mul(zb, sb);
                }
            }
        }
    }
    if (e < t.ne) {
        CDF z, st;
        start(e, z, st);
#pragma unroll
        for (int r = 0; r < L; ++r) {
            if (r < rn.w) {
                ax[r] = df_add(ax[r], z.x);
                ay[r] = df_add(ay[r], z.y);
                if (r + 1 < L) z = cdf_mul(z, st);
            }
        }
    }
}

// One CTA per (walker, chunk of runs), as k_sfac; layers one pass each.
// Registers sized for 4 CTAs per SM (a few spilled values, which cost less
// than the fewer warps: measured 52.6 ms at 3 CTAs, 42.6 ms at 4, per 4096
// fcc walkers) and electron tiles of kDfTile, so that enough warps are
// resident to hide the latency of the double-float chains.
constexpr int kDfTile = 32, kDfMinBlocks = 4;

template <int DIM>
__global__ void __launch_bounds__(kSfacThreads, kDfMinBlocks)
    k_sfac_df(SysDev s, BatchDev b, const unsigned char *__restrict__ only, int te, int write_energy) {
    extern __shared__ __align__(32) unsigned char smem[];
    const int w = blockIdx.x / s.n_gchunks, chunk = blockIdx.x - w * s.n_gchunks;
    if (only && !only[w]) return;  // uniform over the CTA
    const int W1 = 2 * s.n1max + 1, W2 = 2 * s.n2max + 1, W3 = DIM == 3 ? s.n3max + 1 : 0;
    Part<double> *tp = (Part<double> *)smem;
    CDF *P1 = (CDF *)(smem + align16(te * sizeof(Part<double>)));
    CDF *P2 = P1 + (size_t)te * W1;
    CDF *P3 = P2 + (size_t)te * W2;
    double *red = (double *)(smem + align16(te * sizeof(Part<double>)) + align16((size_t)te * (W1 + W2 + W3) * sizeof(CDF)));

    const int tid = threadIdx.x;
    const int run = chunk * s.sfac_threads + tid;
    const bool has = tid < s.sfac_threads && run < s.n_runs;
    const int4 rn0 = has ? s.runs[run] : make_int4(0, 0, 0, 0);
    const int dir = rn0.w < 0 ? -1 : 1;
    const int4 rn = make_int4(rn0.x, rn0.y, rn0.z, rn0.w * dir);
    const int wmax = __shfl_sync(0xffffffffu, rn.w, 0);  // runs are stored longest first
    const int slots = s.n_runs * s.run_len;
    const int nl = DIM == 2 ? s.n_layers : 1;
    double epart = 0;
    for (int L = 0; L < nl; ++L) {
        DF ax[kRunLen], ay[kRunLen];
#pragma unroll
        for (int r = 0; r < kRunLen; ++r) ax[r] = ay[r] = DF{0.f, 0.f};
        const int e_lo = nl > 1 ? s.lay_start[L] : 0, e_hi = nl > 1 ? s.lay_start[L + 1] : s.n_mob;
        for (int e0 = e_lo; e0 < e_hi; e0 += te) {
            const int ne = min(te, e_hi - e0);
            __syncthreads();  // the previous tile's tables are no longer read
            for (int t = tid; t < ne; t += blockDim.x) {
                Part<double> pt = load_mobile<double>(s, b, w, nl > 1 ? s.lay_idx[e0 + t] : e0 + t, DIM);
                const DF q = df_from(pt.q);  // converted once per electron, kept in q's 8 bytes
                pt.q = __hiloint2double(__float_as_int(q.h), __float_as_int(q.l));
                tp[t] = pt;
            }
            __syncthreads();
            // powers e^{2 pi i n f_k}: the base phase by one FP64 sincospi of
            // the exact fraction, the powers in double-float by binary
            // splitting (P^(2m) = (P^m)^2, P^(2m+1) = P^(2m) P), so that no
            // power is more than ~2 log2(n) multiplications from the base
            for (int t = tid; t < ne * DIM; t += blockDim.x) {
                const int e = t / DIM, k = t - e * DIM;
                double sn, cs;
                sincospi(2.0 * FP<double>::frac(tp[e].u[k]), &sn, &cs);
                const CDF base = {df_from(cs), df_from(sn)};
                const int nm = k == 0 ? s.n1max : (k == 1 ? s.n2max : W3 - 1);
                CDF *P = k == 0 ? P1 + (size_t)e * W1 + s.n1max
                                : (k == 1 ? P2 + (size_t)e * W2 + s.n2max : P3 + (size_t)e * W3);
                P[0] = {df_from(1.0), df_from(0.0)};
                for (int n = 1; n <= nm; ++n) {
                    const CDF p = n == 1 ? base : ((n & 1) ? cdf_mul(P[n - 1], base) : cdf_mul(P[n >> 1], P[n >> 1]));
                    P[n] = p;
                    if (k < 2) P[-n] = {p.x, DF{-p.y.h, -p.y.l}};
                }
            }
            __syncthreads();
            const SfacTileDF tl{tp, P1, P2, P3, W1, W2, W3, s.n1max, s.n2max, ne};
            switch (wmax) {  // uniform over the warp
                case 8: sfac_runs_df<DIM, 8>(tl, rn, dir, ax, ay); break;
                case 7: sfac_runs_df<DIM, 7>(tl, rn, dir, ax, ay); break;
                case 6: sfac_runs_df<DIM, 6>(tl, rn, dir, ax, ay); break;
                case 5: sfac_runs_df<DIM, 5>(tl, rn, dir, ax, ay); break;
                case 4: sfac_runs_df<DIM, 4>(tl, rn, dir, ax, ay); break;
                case 3: sfac_runs_df<DIM, 3>(tl, rn, dir, ax, ay); break;
                case 2: sfac_runs_df<DIM, 2>(tl, rn, dir, ax, ay); break;
                case 1: sfac_runs_df<DIM, 1>(tl, rn, dir, ax, ay); break;
                default: break;
            }
        }
        if (has) {
            double2 *rho = b.rho + ((size_t)w * nl + L) * slots;
            const double2 *rfix = s.rho_fix ? s.rho_fix + (size_t)L * slots : nullptr;
#pragma unroll
            for (int r = 0; r < kRunLen; ++r) {
                if (r < s.run_len) {
                    const int slot = r * s.n_runs + run;
                    double2 v = make_double2(0.0, 0.0);
                    if (r < rn.w) {
                        v.x = df_to(ax[r]);
                        v.y = df_to(ay[r]);
                        if (rfix) {
                            v.x += rfix[slot].x;
                            v.y += rfix[slot].y;
                        }
                        if (nl == 1) epart += s.gw_d[slot] * (v.x * v.x + v.y * v.y);
                    }
                    rho[slot] = v;
                }
            }
        }
    }
    if (nl > 1 && has) {  // layered: sum_{L,L'} W_{LL'} Re(rho_L conj(rho_L')) over this thread's slots
        const double2 *rho = b.rho + (size_t)w * nl * slots;
        for (int r = 0; r < s.run_len && r < rn.w; ++r) {
            const int slot = r * s.n_runs + run;
            for (int L = 0; L < nl; ++L) {
                const double2 a = rho[(size_t)L * slots + slot];
                epart += s.gwl_d[((size_t)L * nl + L) * slots + slot] * (a.x * a.x + a.y * a.y);
                for (int M = L + 1; M < nl; ++M) {
                    const double2 c = rho[(size_t)M * slots + slot];
                    epart += 2.0 * s.gwl_d[((size_t)L * nl + M) * slots + slot] * (a.x * c.x + a.y * c.y);
                }
            }
        }
    }
    if (write_energy) {
        const double tot = block_sum(epart, red);
        if (tid == 0) b.part_recip[(size_t)w * s.n_gchunks + chunk] = tot;
    }
}

int launch_sfac_df(const SysDev &s, const BatchDev &b, const LaunchCfg &cfg, const unsigned char *only,
                   cudaStream_t st) {
    const int grid = b.W * s.n_gchunks, we = only ? 0 : 1;
    // tables of 16 bytes an entry, as in the FP64 kernel, for at most kDfTile electrons
    const int te = std::min(cfg.sfac_te, kDfTile);
    const size_t smem = sfac_bytes(s, EWALD_FP64, te, kSfacThreads);
    cudaError_t e;
    if (s.dim == 3) {
        if ((e = allow_max_smem(k_sfac_df<3>, smem))) return e;
        k_sfac_df<3><<<grid, s.sfac_threads, smem, st>>>(s, b, only, te, we);
    } else {
        if ((e = allow_max_smem(k_sfac_df<2>, smem))) return e;
        k_sfac_df<2><<<grid, s.sfac_threads, smem, st>>>(s, b, only, te, we);
    }
    return cudaGetLastError();
}

}  // namespace ewald
