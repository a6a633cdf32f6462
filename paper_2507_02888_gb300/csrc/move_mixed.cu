// Proposed single-particle moves of the mixed-precision form (paper
// Sec. 2.1: dE of moving particle k of each walker from r to r'):
//
//   dE = q_k sum_{j != k} q_j sum_R [phi(r' - r_j + R) - phi(r - r_j + R)]
//      + sum_{G half} 2 C f(G) (2 Re(conj(rho) delta) + |delta|^2).
//
// Persistent CTAs over the walkers, so that the candidate tables of the
// pair loop (real_mixed.cuh: distinct candidate lists as image pairs) are
// staged once per CTA.  Real space: the lanes of the CTA take the other
// particles j; each pair (k at r', j) and (k at r, j) goes through the same
// displacement-cell candidate test as the full energy, the passing r^2 with
// their weights +-q_k q_j into per-lane rings, evaluated two per lane by the
// paired FP32 erfc(alpha r)/r.  A pair closer than the close radius is
// evaluated in FP64 from the exact fixed-point difference.  Reciprocal
// space: each thread walks its G runs with the old and new phases' powers
// (move_items.cuh), reading the float-pair rho(G)'s leading pair.
#include "move_items.cuh"
#include "real_mixed.cuh"

namespace ewald {

// four warps per CTA: more walkers in flight per SM (7 CTAs at the fcc
// workload's 31 KB of shared memory) hide the per-walker chain of
// dependent steps better than wider CTAs (measured per round of 4096 fcc
// walkers: 64 threads 0.207 ms, 96 0.182, 128 0.166, 256 0.176, 512 0.227)
constexpr int kProposeMixedThreads = 128;
// pending terms per lane: a walker's move gives each lane ~25 terms, so a
// short ring (with weights: +-q_k q_j) keeps the CTA small
constexpr int kMoveRing = 16;

struct ProposeMixedSmem {
    MixedImageSmem ims;
    float *rings;
    MoveTables<float> tab;
    double *red;
    __host__ __device__ static size_t ring_bytes() {
        return align16((size_t)(kProposeMixedThreads / 32) * kMoveRing * 32 * sizeof(float) * 2);
    }
    __host__ __device__ static size_t bytes(const SysDev &s) {
        return MixedImageSmem::bytes(s, s.dim, true) + ring_bytes() + MoveSmem<float>::table_bytes(s) +
               align16((kProposeMixedThreads / 32) * sizeof(double));
    }
    __device__ void carve(unsigned char *base, const SysDev &s, int dim) {
        ims.carve(base, s, dim, true);
        size_t off = MixedImageSmem::bytes(s, dim, true);
        rings = (float *)(base + off);
        off += ring_bytes();
        Cx<float> *p = (Cx<float> *)(base + off);
        const int W[3] = {2 * s.n1max + 1, 2 * s.n2max + 1, dim == 3 ? s.n3max + 1 : 0};
        for (int which = 0; which < 2; ++which)
            for (int k = 0; k < 3; ++k) {
                tab.P[which][k] = p;
                p += W[k];
            }
        off += MoveSmem<float>::table_bytes(s);
        red = (double *)(base + off);
    }
};

// The FP64 term of the moved particle (exact 64-bit coordinates uk, height
// zk) and particle j through image img: a pair within the close radius.
template <int DIM>
__device__ inline double close_term_moved(const SysDev &s, const BatchDev &b, int w, const unsigned long long *uk,
                                          double zk, int j, bool fixedj, int img, double wgt) {
    long long dd[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const unsigned long long uj = fixedj ? s.fix_u[(size_t)d * s.fix_stride + j]
                                             : b.u[((size_t)w * DIM + d) * s.mob_stride + j];
        dd[d] = (long long)(uk[d] - uj);
    }
    double z2 = 0.0;
    if (DIM == 2 && s.n_layers > 1) {
        const double dz = zk - (fixedj ? s.z_fix[j] : s.z_mob[j]);
        z2 = dz * dz;
    }
    return close_term<DIM>(s, dd, img, wgt, b.status, z2);
}

// The proposals checked and converted, one thread per walker: the moved
// particle's index, its new position as fixed-point fractions (pend_u) and
// a flag on a bad index or a non-finite position (pend_k = -1, dE = NaN).
template <int DIM>
__global__ void k_propose_prepare(SysDev s, BatchDev b, const int *__restrict__ kk, const double *__restrict__ r_new,
                                  double *__restrict__ de) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= b.W) return;
    const int k = kk[w];
    unsigned long long un[3] = {0, 0, 0};
    bool ok = k >= 0 && k < s.n_mob;
    ok = cart_to_fixed<DIM>(s, r_new + (size_t)w * DIM, un) && ok;
    if (!ok) {
        atomicOr(b.status, ST_BAD_INDEX);
        b.pend_k[w] = -1;
        de[w] = __longlong_as_double(0x7ff8000000000000LL);  // NaN
        return;
    }
    b.pend_k[w] = k;
    for (int d = 0; d < 3; ++d) b.pend_u[(size_t)w * 3 + d] = un[d];
}

template <int DIM, int CM>
__global__ void __launch_bounds__(kProposeMixedThreads)
    k_propose_mixed(SysDev s, BatchDev b, double *__restrict__ de) {
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ unsigned long long su[2][3];  // old, new: exact fixed-point coordinates
    ProposeMixedSmem m;
    m.carve(smem, s, DIM);
    m.ims.stage(s, DIM, true);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const TermK32 tk = FP<float>::term_consts(s);
    const int n_other = s.n_mob - 1 + s.n_fix;
    for (int w = blockIdx.x; w < b.W; w += gridDim.x) {
        __syncthreads();  // the previous walker is done with the shared state
        const int k = b.pend_k[w];
        if (k < 0) continue;  // a bad proposal (k_propose_prepare set dE = NaN)
        if (tid < 6) {
            const int which = tid / 3, d = tid % 3;
            su[which][d] = which ? b.pend_u[(size_t)w * 3 + d]
                                 : (d < DIM ? b.u[((size_t)w * DIM + d) * s.mob_stride + k] : 0ull);
        }
        __syncthreads();
        unsigned uo[3], un[3];
        for (int d = 0; d < 3; ++d) {
            uo[d] = (unsigned)(su[0][d] >> 32);
            un[d] = (unsigned)(su[1][d] >> 32);
        }
        build_move_tables<float, DIM>(s, uo, un, m.tab);
        __syncthreads();  // the tables are read by every thread's G runs below
        const float qk = s.q_mob_f[k];
        const bool layered = DIM == 2 && s.n_layers > 1;
        const float zk = layered ? s.z_mob_f[k] : 0.0f;
        const unsigned u2o = DIM == 2 ? (layered ? __float_as_uint(zk) : 0u) : uo[2];
        const unsigned u2n = DIM == 2 ? (layered ? __float_as_uint(zk) : 0u) : un[2];
        // real space: slot t = (other particle jj, old/new) over the CTA's lanes
        LaneRing<true, kMoveRing> ring{m.rings + (size_t)warp * kMoveRing * 32 * 2 + lane, 0u, 0u, b.status};
        Acc<float> acc;
        double acc64 = 0.0;
        // slot t: the other particle of index jj (mobile ones except k, then
        // the fixed ones) at the old (t even) or new (t odd) position of k;
        // each lane loads its next slot's particle while it works on this one
        auto other = [&](int t, int &j, bool &fixedj) {
            const int jj = t >> 1;
            fixedj = jj >= s.n_mob - 1;
            j = fixedj ? jj - (s.n_mob - 1) : (jj < k ? jj : jj + 1);
            Tile16 p = {{0u, 0u, 0u}, 0.0f};
            if (t < 2 * n_other &&
                EWALD_IN_RANGE(j >= 0 && (fixedj ? j < s.n_fix : j < s.n_mob && j != k), b.status))
                p = fixedj ? tile16_fixed<DIM>(s, j) : tile16_mobile<DIM>(s, b, w, j);
            return p;
        };
        int jn;
        bool fn;
        Tile16 pn = other(warp * 32 + lane, jn, fn);
        for (int base = warp * 32; base < 2 * n_other; base += blockDim.x) {
            const int t = base + lane;
            const bool v = t < 2 * n_other;
            const int which = t & 1;
            const Tile16 pj = pn;
            const int j = jn;
            const bool fixedj = fn;
            pn = other(base + blockDim.x + lane, jn, fn);
            const float wgt = (which ? 1.0f : -1.0f) * qk * pj.q;
            const Tile16 pkw = which ? Tile16{{un[0], un[1], u2n}, qk} : Tile16{{uo[0], uo[1], u2o}, qk};
            bool close = false;
            pair_ring<DIM, CM, true, kMoveRing>(s, m.ims, pkw, pj, v, wgt, ring, close, acc, tk);
            ring_service<CM, 1>(ring, acc, tk);
            if (__any_sync(0xffffffffu, close) && close) {  // rare: the FP64 term now
                float x[DIM], z2;
                const int sc = pair_cart<DIM>(s, pkw, pj, x, z2);
                acc64 += close_term_moved<DIM>(s, b, w, su[which], layered ? s.z_mob[k] : 0.0, j, fixedj,
                                               s.cand[sc * s.cand_max], (double)wgt);
            }
        }
        ring.drain(acc, tk);
        double tot = acc.get() + acc64;
        // reciprocal space
        float part = 0.0f;
        if (layered) {
            part = layered_recip_delta<float, DIM>(s, b, w, k, qk, m.tab);
        } else {
            const double2 *rho = b.rho + (size_t)w * s.n_runs * s.run_len;
            for_each_delta<float, DIM>(s, m.tab, qk, [&](int slot, Cx<float> d) {
                const Cx<float> rv = RhoIO<float>::lead(rho, slot);
                part += FP<float>::gw(s, slot) * (2.0f * (rv.x * d.x + rv.y * d.y) + d.x * d.x + d.y * d.y);
            });
        }
        tot += (double)part;
        tot = block_sum(tot, m.red);
        if (tid == 0) de[w] = tot;
    }
}

using ProposeFn = void (*)(SysDev, BatchDev, double *);

template <int DIM>
static ProposeFn propose_fn(int cm) {
    switch (cm) {
        case 2: return k_propose_mixed<DIM, 2>;
        case 4: return k_propose_mixed<DIM, 4>;
        case 6: return k_propose_mixed<DIM, 6>;
        case 8: return k_propose_mixed<DIM, 8>;
        default: return k_propose_mixed<DIM, 0>;
    }
}

static ProposeFn propose_mixed_fn(const SysDev &s) {
    const int cm = mixed_cm(s.cand_max);
    return s.dim == 3 ? propose_fn<3>(cm) : propose_fn<2>(cm);
}

size_t propose_mixed_smem(const SysDev &s) { return ProposeMixedSmem::bytes(s); }

int configure_propose_mixed(const SysDev &s, int sm_count, int *grid) {
    const ProposeFn f = propose_mixed_fn(s);
    const size_t smem = ProposeMixedSmem::bytes(s);
    int occ = 0;
    cudaError_t e = allow_max_smem(f, smem);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kProposeMixedThreads, smem);
    if (!e && occ < 1) e = cudaErrorInvalidConfiguration;
    *grid = sm_count * occ;
    return e;
}

int launch_propose_mixed(const SysDev &s, const BatchDev &b, int grid, const int *k, const double *r_new, double *de,
                         cudaStream_t st) {
    if (s.dim == 3) k_propose_prepare<3><<<(b.W + 127) / 128, 128, 0, st>>>(s, b, k, r_new, de);
    else k_propose_prepare<2><<<(b.W + 127) / 128, 128, 0, st>>>(s, b, k, r_new, de);
    propose_mixed_fn(s)<<<std::min(grid, b.W), kProposeMixedThreads, ProposeMixedSmem::bytes(s), st>>>(s, b, de);
    return cudaGetLastError();
}

}  // namespace ewald
