// Single-particle move kernels: propose (energy change) and accept
// (rho(G) += delta(G), position update); the work itself is in
// move_items.cuh.  With the walker's rho(G) resident on the device the
// change costs O(N + N_G).
//
// One CTA per walker.  The powers e^{2 pi i n f_k} of the old and new
// position are computed from exact fixed-point phases (n u mod 2^bits), and
// each thread walks its G runs by one complex multiplication per G.
#include <math.h>

#include "move_items.cuh"

namespace ewald {

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
    const int w = blockIdx.x, tid = threadIdx.x;
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
        set_lo<R>(pold, d, su_old[d]);
        set_lo<R>(pnew, d, su_new[d]);
    }
    pold.q = pnew.q = FP<R>::q_mob(s, k);
    if (DIM == 2) {  // after the coordinates: the FP64 height shares the third word
        const R z = s.n_layers > 1 ? FP<R>::z_mob(s, k) : R(0);
        set_part_z(pold, z);
        set_part_z(pnew, z);
    }
    build_move_tables<R, DIM>(s, pold.u, pnew.u, m.tab);
    __syncthreads();

    const double tot = move_delta_e<R, DIM>(s, b, w, k, pold, pnew, m);
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
        set_lo<R>(pold, d, uo);
        set_lo<R>(pnew, d, b.pend_u[(size_t)w * 3 + d]);
    }
    pold.q = FP<R>::q_mob(s, k);
    build_move_tables<R, DIM>(s, pold.u, pnew.u, m.tab);
    __syncthreads();
    move_apply_rho<R, DIM>(s, b, w, k, pold.q, m.tab);
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

// Mixed precision accept: one CTA per walker, as k_accept, with each
// thread's G run of rho(G) loaded before the recurrence updates it (the
// loads of a run are independent, so up to kRunLen are in flight per
// thread), the float-pair rho updated by two-sums, and walkers due for a
// re-sum listed in b.resum_list.  CTAs of four warps: each thread takes
// about three runs, and more walkers are in flight per SM (measured per
// round of 4096 fcc walkers: 64 threads 0.043 ms, 128 0.033, 256 0.044).
constexpr int kAcceptMixedThreads = 128;
template <int DIM>
__global__ void __launch_bounds__(kAcceptMixedThreads)
    k_accept_mixed(SysDev s, BatchDev b, const unsigned char *__restrict__ acc, int resum_every) {
    extern __shared__ __align__(32) unsigned char smem[];
    MoveSmem<float> m;
    m.carve(smem, s, DIM);
    const int w = blockIdx.x, tid = threadIdx.x;
    const int k = b.pend_k[w];
    if (k < 0 || !acc[w]) {
        if (tid == 0) {
            b.pend_k[w] = -1;
            b.resum_flag[w] = 0;
        }
        return;
    }
    unsigned uo[3], un[3];
    for (int d = 0; d < 3; ++d) {
        uo[d] = d < DIM ? (unsigned)(b.u[((size_t)w * DIM + d) * s.mob_stride + k] >> 32) : 0u;
        un[d] = (unsigned)(b.pend_u[(size_t)w * 3 + d] >> 32);
    }
    build_move_tables<float, DIM>(s, uo, un, m.tab);
    __syncthreads();
    const float qk = s.q_mob_f[k];
    const size_t slots = (size_t)s.n_runs * s.run_len;
    float4 *rho = (float4 *)(b.rho + ((size_t)w * s.n_layers + (DIM == 2 && s.n_layers > 1 ? s.mob_layer[k] : 0)) * slots);
    const MoveTables<float> &t = m.tab;
    for (int run = tid; run < s.n_runs; run += blockDim.x) {
        const int4 rn = s.runs[run];
        const int dir = rn.w < 0 ? -1 : 1, len = rn.w * dir;
        float4 v[kRunLen];
#pragma unroll
        for (int r = 0; r < kRunLen; ++r)
            if (r < len) v[r] = rho[(size_t)r * s.n_runs + run];
        Cx<float> zo = cmul(t.P[0][0][rn.x + s.n1max], t.P[0][1][rn.y + s.n2max]);
        Cx<float> zn = cmul(t.P[1][0][rn.x + s.n1max], t.P[1][1][rn.y + s.n2max]);
        if (DIM == 3) {
            zo = cmul(zo, t.P[0][2][rn.z]);
            zn = cmul(zn, t.P[1][2][rn.z]);
        }
        const Cx<float> so = t.P[0][0][s.n1max + dir], sn = t.P[1][0][s.n1max + dir];
#pragma unroll
        for (int r = 0; r < kRunLen; ++r) {
            if (r < len) {
                float hx = v[r].x, lx = v[r].z, hy = v[r].y, ly = v[r].w;
                RhoIO<float>::acc(hx, lx, qk * (zn.x - zo.x));
                RhoIO<float>::acc(hy, ly, qk * (zn.y - zo.y));
                rho[(size_t)r * s.n_runs + run] = make_float4(hx, hy, lx, ly);
                zo = cmul(zo, so);
                zn = cmul(zn, sn);
            }
        }
    }
    __syncthreads();  // every thread has read the old position
    if (tid < DIM) b.u[((size_t)w * DIM + tid) * s.mob_stride + k] = b.pend_u[(size_t)w * 3 + tid];
    if (tid == 0) {
        b.pend_k[w] = -1;
        const int c = b.acc_count[w] + 1;
        const bool f = c >= resum_every;
        b.acc_count[w] = f ? 0 : c;
        b.resum_flag[w] = f ? 1 : 0;
        if (f) b.resum_list[1 + atomicAdd(b.resum_list, 1)] = w;
    }
}

size_t move_smem_bytes(const SysDev &s, int precision) {
    return precision == EWALD_FP64 ? MoveSmem<double>::bytes(s) : MoveSmem<float>::bytes(s);
}

int configure_move(const SysDev &s, int precision, size_t smem) {
    cudaError_t e;
    auto set = [&](const void *f) { return allow_max_smem(f, smem); };
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
            if ((e = set((const void *)k_accept_mixed<3>))) return e;
            e = set((const void *)k_accept<float, 3>);
        } else {
            if ((e = set((const void *)k_propose<float, 2>))) return e;
            if ((e = set((const void *)k_accept_mixed<2>))) return e;
            e = set((const void *)k_accept<float, 2>);
        }
    }
    return e;
}

int launch_propose(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg, const int *k,
                   const double *r_new, double *de, cudaStream_t st) {
    if (precision == EWALD_MIXED && cfg.propose_grid > 0) return launch_propose_mixed(s, b, cfg.propose_grid, k, r_new, de, st);
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
    if (precision != EWALD_FP64 && b.resum_list) {
        cudaError_t e = cudaMemsetAsync(b.resum_list, 0, sizeof(int), st);
        if (e) return e;
        if (s.dim == 3) k_accept_mixed<3><<<b.W, kAcceptMixedThreads, cfg.move_smem, st>>>(s, b, acc, resum_every);
        else k_accept_mixed<2><<<b.W, kAcceptMixedThreads, cfg.move_smem, st>>>(s, b, acc, resum_every);
        return cudaGetLastError();
    }
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
