// Real-space pair sum of the mixed-precision path (paper Eq. (3), second
// term), one (walker, tile pair) item per call: the FP32 loop of the
// full-energy kernels (energy_kernels.cu, multi_kernels.cu).
//
// Each warp takes 32 x 32 sub-tiles, lane = particle i, loop over the j of
// the sub-tile (staged in shared memory, read as a broadcast).  For one pair
// a lane forms the exact fixed-point difference, its displacement cell and
// its Cartesian vector, then tests the cell's candidate images, a list of
// compile-time length CM stored as pairs of images in the operand layout of
// the paired FP32 instructions (one 16-byte and one 8-byte load and six
// paired operations per two images).
// Images inside r_c are not compacted across the warp: every lane appends
// the r^2 of its passing images to a ring of its own in shared
// memory (column `lane` of a [kLaneRing][32] array: no bank conflicts, no
// ballots), and the warp evaluates two pending terms per lane (the paired
// erfc_over_r_f32x2) as often as every lane has two waiting.  Lanes drift
// apart by a few entries (the number of images inside r_c differs from pair
// to pair); when one lane's ring would overflow, a forced evaluation lets
// the lanes with two pending evaluate while the others idle, and the rings
// are drained at the end of the item.  Compared with a warp-wide queue this
// removes the per-candidate ballot, population counts and ring addressing,
// which were a third of the loop's instructions.
// Where a system's lists hold 3 to 8 images and their second image (the
// second nearest to the cell's centre) is inside r_c for most displacements
// (SysDev::mixed_direct, decided at set-up), the first two images of every
// pair skip the ring: one paired evaluation with the images outside r_c
// masked to zero.
//
// Charges: when every mobile charge is equal and every fixed charge is
// equal (the electron gases and the ionic solids), an item's pairs share
// one weight q_i q_j and the rings hold r^2 alone, the item's sum of
// erfc(alpha r)/r being multiplied by the weight once; otherwise (QW) each
// entry carries its weight.
#pragma once
#include "device_common.cuh"

namespace ewald {

constexpr int kLaneRing = 32;  // pending terms per lane (a power of two)
// how the pair loop takes the first two images of a list (see pair_ring)
constexpr int kDirectNever = 0, kDirectFlag = 1, kDirectAlways = 2;

// A particle of the FP32 pair loop in shared memory: the top 32 bits of the
// fixed-point coordinates and the charge; in a 2D cell the third word holds
// the height (float bits) of a layered cell, 0 otherwise.
struct __align__(16) Tile16 {
    unsigned u[3];
    float q;
};

// Candidate tables of the FP32 pair loop in shared memory.  The candidate
// lists of the displacement cells are stored once per distinct list (many
// cells share a list), as pairs of images in the operand layout of the
// paired FP32 instructions: for pair p of list L, xy[L][p] = (X_a, X_b,
// Y_a, Y_b) and, in 3D, z[L][p] = (Z_a, Z_b) (lists padded with the far
// sentinel to cand_pairs pairs, stored cand_pstride pairs apart); clist[cell]
// is the cell's list.  moves: the move kernel's copy of the tables (lists in
// the order of the FP64 tables; the energy kernels' copy differs where the
// system takes the first two images directly, SysDev::mixed_direct).
struct MixedImageSmem {
    float4 *xy;
    float2 *z;
    unsigned short *clist;
    int n_lists;  // distinct lists staged
    __host__ __device__ static int lists(const SysDev &s, bool moves) { return moves ? s.n_lists_mv : s.n_lists; }
    __host__ __device__ static size_t bytes(const SysDev &s, int dim, bool moves = false) {
        const size_t n_sub = (size_t)1 << (s.sub_bits * dim), np = (size_t)lists(s, moves) * s.cand_pstride;
        return align16(np * sizeof(float4)) + (dim == 3 ? align16(np * sizeof(float2)) : 0) +
               align16(n_sub * sizeof(unsigned short));
    }
    __device__ void carve(unsigned char *base, const SysDev &s, int dim, bool moves = false) {
        n_lists = lists(s, moves);
        const size_t np = (size_t)n_lists * s.cand_pstride;
        xy = (float4 *)base;
        z = (float2 *)(base + align16(np * sizeof(float4)));
        clist = (unsigned short *)(base + align16(np * sizeof(float4)) + (dim == 3 ? align16(np * sizeof(float2)) : 0));
    }
    // after carve with the same moves
    __device__ void stage(const SysDev &s, int dim, bool moves = false) {
        const int n_sub = 1 << (s.sub_bits * dim), np = n_lists * s.cand_pstride;
        const float4 *gxy = moves ? s.cxy_mv : s.cxy;
        const float2 *gz = moves ? s.cz_mv : s.cz;
        const unsigned short *gl = moves ? s.clist_mv : s.clist;
        for (int i = threadIdx.x; i < np; i += blockDim.x) xy[i] = gxy[i];
        if (dim == 3)
            for (int i = threadIdx.x; i < np; i += blockDim.x) z[i] = gz[i];
        for (int i = threadIdx.x; i < n_sub; i += blockDim.x) clist[i] = gl[i];
    }
};

// Shared memory of one item (besides the candidate tables): two particle
// tiles, the warps' rings (with weights when the charges differ), the
// warps' close-pair lists and the per-warp sums.
__host__ __device__ inline size_t mixed_real_work_bytes(const SysDev &s, int warps) {
    const size_t ring = (size_t)kLaneRing * 32 * sizeof(float) * (s.q_uniform ? 1 : 2);
    return 2 * align16(s.tile * sizeof(Tile16)) + align16((size_t)warps * ring) +
           align16((size_t)warps * kCloseCap * sizeof(unsigned)) + align16((size_t)warps * sizeof(double));
}

template <int DIM>
__device__ inline Tile16 tile16_mobile(const SysDev &s, const BatchDev &b, int w, int i) {
    Tile16 p = {{0u, 0u, 0u}, 0.0f};
    if (i < s.n_mob) {
        const unsigned long long *u = b.u + (size_t)w * DIM * s.mob_stride + i;
#pragma unroll
        for (int k = 0; k < DIM; ++k) p.u[k] = (unsigned)(u[(size_t)k * s.mob_stride] >> 32);
        if (DIM == 2 && s.n_layers > 1) p.u[2] = __float_as_uint(s.z_mob_f[i]);
        p.q = s.q_mob_f[i];
    }
    return p;
}

template <int DIM>
__device__ inline Tile16 tile16_fixed(const SysDev &s, int i) {
    Tile16 p = {{0u, 0u, 0u}, 0.0f};
    if (i < s.n_fix) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) p.u[k] = (unsigned)(s.fix_u[(size_t)k * s.fix_stride + i] >> 32);
        if (DIM == 2 && s.n_layers > 1) p.u[2] = __float_as_uint(s.z_fix_f[i]);
        p.q = s.q_fix_f[i];
    }
    return p;
}

// The FP64 term of a close pair (global particle indices; j fixed if
// fixedj) through image img, from the exact 64-bit fixed-point difference.
template <int DIM>
__device__ inline double close_term_global(const SysDev &s, const BatchDev &b, int w, int gi, int gj, bool fixedj,
                                           int img, double wgt) {
    long long dd[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const unsigned long long ua = b.u[((size_t)w * DIM + k) * s.mob_stride + gi];
        const unsigned long long ub = fixedj ? s.fix_u[(size_t)k * s.fix_stride + gj]
                                             : b.u[((size_t)w * DIM + k) * s.mob_stride + gj];
        dd[k] = (long long)(ua - ub);
    }
    double z2 = 0.0;
    if (DIM == 2 && s.n_layers > 1) {
        const double dz = s.z_mob[gi] - (fixedj ? s.z_fix[gj] : s.z_mob[gj]);
        z2 = dz * dz;
    }
    return close_term<DIM>(s, dd, img, wgt, b.status, z2);
}

// One warp's pending terms: lane l's entries k live at r2[k * 32] (and, with
// weights, at r2[kLaneRing * 32 + k * 32]) of its column; cnt counts the
// entries pushed, hd those evaluated (even, except after the final drain).
template <bool QW, int CAP = kLaneRing>
struct LaneRing {
    float *col;      // this lane's column
    unsigned cnt, hd;
    int *status = nullptr;  // the batch's status word (checks of the debug build)
    __device__ float *at(unsigned k) const { return col + (k & (CAP - 1)) * 32; }
    __device__ void push(bool pass, float r2, float wgt) {
        float *e = at(cnt);
        if (pass && EWALD_IN_RANGE(cnt - hd < (unsigned)CAP, status)) {  // an entry not yet evaluated
            e[0] = r2;
            if (QW) e[CAP * 32] = wgt;
        }
        cnt += pass ? 1u : 0u;
    }
    // two entries, hd even: slots hd and hd + 1 of the ring are adjacent rows
    __device__ void eval_two(Acc<float> &acc, const TermK32 &tk) {
        const float *e = at(hd);
        float2 t = erfc_over_r_f32x2(make_float2(e[0], e[32]), tk);
        if (QW) t = mul2(t, make_float2(e[CAP * 32], e[CAP * 32 + 32]));
        acc.add2(t);
        hd += 2;
    }
    // lanes with two entries evaluate them; the others idle
    __device__ void eval_some(Acc<float> &acc, const TermK32 &tk) {
        const bool take = cnt - hd >= 2u;
        const float *e = at(hd);
        const float2 r2 = take ? make_float2(e[0], e[32]) : make_float2(1.0f, 1.0f);
        float2 t = erfc_over_r_f32x2(r2, tk);
        if (take) {
            if (QW) t = mul2(t, make_float2(e[CAP * 32], e[CAP * 32 + 32]));
            acc.add2(t);
            hd += 2;
        }
    }
    // after a pair (or a chunk of candidates): evaluate while every lane has
    // two waiting; then, if some lane could not take `room` more entries,
    // let the lanes with two waiting evaluate until it can
    template <int ROOM>
    __device__ void service(Acc<float> &acc, const TermK32 &tk) {
        // a lane above the threshold has at least two entries, so every
        // forced evaluation below shortens the longest ring: the loop ends
        static_assert(CAP - ROOM >= 2, "ring too short for the entries pushed between services");
        const unsigned pend = cnt - hd;
        const unsigned lo = __reduce_min_sync(0xffffffffu, pend);
        for (unsigned n = lo >> 1; n > 0; --n) eval_two(acc, tk);
        unsigned hi = __reduce_max_sync(0xffffffffu, cnt - hd);
        while (hi > (unsigned)(CAP - ROOM)) {
            eval_some(acc, tk);
            hi = __reduce_max_sync(0xffffffffu, cnt - hd);
        }
    }
    // everything left, one or two per lane at a time
    __device__ void drain(Acc<float> &acc, const TermK32 &tk) {
        while (__any_sync(0xffffffffu, cnt != hd)) {
            const unsigned n = min(cnt - hd, 2u);
            const float *e0 = at(hd), *e1 = at(hd + 1);
            float2 r2 = make_float2(n > 0 ? e0[0] : 1.0f, n > 1 ? e1[0] : 1.0f);
            float2 t = erfc_over_r_f32x2(r2, tk);
            if (QW) t = mul2(t, make_float2(n > 0 ? e0[CAP * 32] : 0.0f, n > 1 ? e1[CAP * 32] : 0.0f));
            if (n == 1) t.y = 0.0f;
            if (n > 0) acc.add2(t);
            hd += n;
        }
    }
};

// Cartesian FP32 displacement of a pair from the exact fixed-point
// difference, with the lattice as (hi, lo) (lo products first), and its
// displacement cell (the top sub_bits bits of each wrapped fraction).
template <int DIM>
__device__ __forceinline__ int pair_cart(const SysDev &s, const Tile16 &a, const Tile16 &b, float *x, float &z2) {
    int d[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) d[k] = (int)(a.u[k] - b.u[k]);
    int sc = 0;
    const int sh = 32 - s.sub_bits;
    if (s.sub_bits) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) sc |= (int)(((unsigned)d[k] ^ 0x80000000u) >> sh) << (k * s.sub_bits);
    }
#pragma unroll
    for (int y = 0; y < DIM; ++y) {
        float v = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) v = __fmaf_rn((float)d[k], s.A32lo[k][y], v);
#pragma unroll
        for (int k = 0; k < DIM; ++k) v = __fmaf_rn((float)d[k], s.A32[k][y], v);
        x[y] = v;
    }
    z2 = 0.0f;
    if (DIM == 2 && s.n_layers > 1) {
        const float dz = __uint_as_float(a.u[2]) - __uint_as_float(b.u[2]);
        z2 = dz * dz;
    }
    return sc;
}

__device__ __forceinline__ float4 lds128(const float4 *p) {
    float4 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

// Test NP (compile-time) candidate pairs of a list, two images per paired
// instruction (each component rounded as image_r2 rounds it), and push the
// r^2 that pass; FIRST: the pairs start with candidate 0, the only image
// through which a displacement of the cell can come within the close
// radius: a close pair is recorded for FP64 instead.
// DIRECT_OK and direct (the system's mixed_direct): the first pair of
// images, the two nearest to the cell's centre, is evaluated at once as one
// paired term (images outside r_c, or close, contribute exactly zero)
// instead of entering the ring.  Measured on the GB300 (fcc N = 1024, 4096
// walkers): k_real_mixed 21.98 -> 20.86 ms, diamond +6%.  In the move
// kernel, which services its rings after every pair, it did not pay
// (propose 0.173 ms per round against 0.166), and the reordered lists alone
// slowed it to 0.178 ms: the move kernel keeps every image in the ring and
// its own copy of the tables in the original order (0.167 ms).
template <int DIM, int NP, bool FIRST, bool QW, int CAP, bool DIRECT_OK = false>
__device__ __forceinline__ void test_pairs(const float4 *xy, const float2 *zz, const float *x, float z2, float rc2,
                                           float close2, float wgt, LaneRing<QW, CAP> &ring, bool &close,
                                           bool direct = false, Acc<float> *acc = nullptr,
                                           const TermK32 *tk = nullptr) {
    const float2 x0 = splat(x[0]), x1 = splat(x[1]), zs = splat(z2);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float4 XY = lds128(xy + p);
        const float2 y0 = add2(x0, make_float2(XY.x, XY.y)), y1 = add2(x1, make_float2(XY.z, XY.w));
        float2 r2 = fma2(y1, y1, fma2(y0, y0, zs));
        if (DIM == 3) {
            const float2 y2 = add2(splat(x[DIM - 1]), zz[p]);
            r2 = fma2(y2, y2, r2);
        }
        bool pa = r2.x < rc2;
        const bool pb = r2.y < rc2;
        if (FIRST && p == 0) {
            close = pa && r2.x < close2;
            pa = pa && !close;
        }
        if (FIRST && DIRECT_OK && p == 0 && direct) {  // uniform over the warp (one system)
            // masked entries take r^2 = 1 (a finite term) and then weigh zero
            float2 t = erfc_over_r_f32x2(make_float2(pa ? r2.x : 1.0f, pb ? r2.y : 1.0f), *tk);
            t = make_float2(pa ? t.x : 0.0f, pb ? t.y : 0.0f);
            if (QW) t = mul2(t, splat(wgt));
            acc->add2(t);
        } else {
            ring.push(pa, r2.x, wgt);
            ring.push(pb, r2.y, wgt);
        }
    }
}

// Candidate slots with a compiled pair loop (pairs of images); a list of
// another length runs the next longer one (padded with the sentinel),
// longer than 8 the chunked loop (slots = 0: chunks of 8 pairs).
__host__ __device__ inline int mixed_cm(int cand_max) {
    return cand_max <= 2 ? 2 : cand_max <= 4 ? 4 : cand_max <= 6 ? 6 : cand_max <= 8 ? 8 : 0;
}
__host__ __device__ inline int mixed_pairs(int cand_max) {
    const int cm = mixed_cm(cand_max);
    return cm ? cm / 2 : (cand_max + 15) / 16 * 8;
}
// pairs of images per chunk of a long list: 8, or 4 for rings too short to
// take 16 entries between services
template <int CAP>
constexpr int kChunkPairs = CAP >= 32 ? 8 : 4;
// Particle pairs between services of the rings in the energy kernels
// (kPairsPerService x CM entries at most come in between): fewer services
// mean fewer warp reductions per pair.  Measured on the GB300 against one
// pair per service for CM = 6 and 8 and four for CM = 2: fcc N = 1024
// 22.27 -> 21.95 ms, diamond 7.34 -> 7.26 ms, 2D gas 0.81 -> 0.80 ms.
// Long lists (CM = 0) are serviced after every pair: pair_ring services
// only between the chunks of one pair, so the last chunk of a pair and the
// first of the next must not meet in one ring.
template <int CM>
constexpr int kPairsPerService = CM == 0 ? 1 : CM == 2 ? 8 : 2;

// The images of one pair of particles: CM candidate slots (CM = 2 ... 8
// compile-time; the caller services the rings every kPairsPerService<CM>
// pairs) or, CM = 0, the list in chunks of 8 pairs (serviced here after
// every chunk but the last, which the caller's service follows).
// DIRECT: how the first two images of a list are taken (CM = 4 ... 8):
// kDirectNever (through the ring: the move kernel), kDirectFlag (without the
// ring where the system's mixed_direct is set: the multi-system kernels) or
// kDirectAlways (the single-system kernel's instantiation for such systems).
template <int DIM, int CM, bool QW, int CAP, int DIRECT = kDirectNever>
__device__ __forceinline__ void pair_ring(const SysDev &s, const MixedImageSmem &ims, const Tile16 &a,
                                          const Tile16 &b, bool valid, float wgt, LaneRing<QW, CAP> &ring,
                                          bool &close, Acc<float> &acc, const TermK32 &tk) {
    float x[DIM], z2;
    const int sc = pair_cart<DIM>(s, a, b, x, z2);
    const float rc2 = valid ? s.rc2_f : 0.0f;  // invalid lanes never pass
    const int sub = EWALD_IN_RANGE(sc < (1 << (s.sub_bits * DIM)), ring.status) ? sc : 0;
    const int lid = ims.clist[sub];
    const int base = (EWALD_IN_RANGE(lid < ims.n_lists, ring.status) ? lid : 0) * s.cand_pstride;
    const float4 *xy = ims.xy + base;
    const float2 *zz = ims.z + base;
    if (CM > 0) {
        constexpr bool ok = DIRECT != kDirectNever && CM >= 4;
        const bool direct = DIRECT == kDirectAlways || (DIRECT == kDirectFlag && s.mixed_direct != 0);
        test_pairs<DIM, CM / 2, true, QW, CAP, ok>(xy, zz, x, z2, rc2, s.close2_f, wgt, ring, close, direct, &acc,
                                                   &tk);
    } else {
        constexpr int CP = kChunkPairs<CAP>;
        test_pairs<DIM, CP, true, QW, CAP>(xy, zz, x, z2, rc2, s.close2_f, wgt, ring, close);
        for (int ch = CP; ch < s.cand_pairs; ch += CP) {
            ring.template service<2 * CP>(acc, tk);
            bool unused;
            test_pairs<DIM, CP, false, QW, CAP>(xy + ch, zz + ch, x, z2, rc2, s.close2_f, wgt, ring, unused);
        }
    }
}

// The rings' service after the PAIRS pairs of a step (the energy kernels:
// kPairsPerService; the move kernel services after every pair).  PUSHED:
// the images of a pair that may enter the ring (CM, or CM - 2 when the
// first two are always evaluated directly).
template <int CM, int PAIRS = kPairsPerService<CM>, int PUSHED = CM, bool QW, int CAP>
__device__ __forceinline__ void ring_service(LaneRing<QW, CAP> &ring, Acc<float> &acc, const TermK32 &tk) {
    constexpr int room = CM > 0 ? PUSHED * PAIRS : 2 * kChunkPairs<CAP>;
    ring.template service<room>(acc, tk);
}

// One (walker w, tile pair p) item: E_real partial sum of the item into
// b.part_real.  All threads of the CTA call it; ims holds this system's
// candidate tables; work is this item's scratch (mixed_real_work_bytes).
// Units are 32 x 32 sub-tiles (diagonal tiles: the upper triangle), or
// jsplit slices of one, taken by the warps in turn; each warp sums its
// units, and the item's sum adds the warps' sums in warp order.
template <int DIM, int CM, bool QW, int DIRECT = kDirectFlag>
__device__ void real_item_mixed_cm(const SysDev &s, const BatchDev &b, int w, int p, const MixedImageSmem &ims,
                                   unsigned char *work, int jsplit) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    size_t off = 0;
    Tile16 *ti = (Tile16 *)(work + off);
    off += align16(s.tile * sizeof(Tile16));
    Tile16 *tj = (Tile16 *)(work + off);
    off += align16(s.tile * sizeof(Tile16));
    float *rings = (float *)(work + off);
    off += align16((size_t)nw * kLaneRing * 32 * sizeof(float) * (QW ? 2 : 1));
    unsigned *cbase = (unsigned *)(work + off);
    off += align16((size_t)nw * kCloseCap * sizeof(unsigned));
    double *red = (double *)(work + off);

    const int S = s.tile / 32;
    const int2 tt = s.items[p];
    const bool fixedj = tt.y >= s.n_mob_tiles;
    const int i0 = tt.x * s.tile;
    const int j0 = (fixedj ? tt.y - s.n_mob_tiles : tt.y) * s.tile;
    const int nj = fixedj ? s.n_fix : s.n_mob;
    __syncthreads();  // the previous item's tiles are no longer read
    for (int t = tid; t < s.tile; t += blockDim.x) {
        ti[t] = tile16_mobile<DIM>(s, b, w, i0 + t);
        tj[t] = fixedj ? tile16_fixed<DIM>(s, j0 + t) : tile16_mobile<DIM>(s, b, w, j0 + t);
    }
    __syncthreads();
    const TermK32 tk = FP<float>::term_consts(s);
    // the item's common weight (charges all equal within each kind)
    const float wq = QW ? 1.0f : s.q_mob_f[0] * (fixedj ? s.q_fix_f[0] : s.q_mob_f[0]);
    LaneRing<QW> ring{rings + (size_t)warp * kLaneRing * 32 * (QW ? 2 : 1) + lane, 0u, 0u, b.status};
    Acc<float> acc;       // FP32 terms (weighted if QW)
    double acc64 = 0.0;   // close pairs in FP64, weighted
    const bool diag = !fixedj && tt.x == tt.y;
    const int nst = diag ? S * (S + 1) / 2 : S * S;
    const int nunits = nst * jsplit, jlen = 32 / jsplit;
    for (int u = warp; u < nunits; u += nw) {
        const int st = u / jsplit, j_lo = (u - st * jsplit) * jlen;
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
        if (i0 + a * 32 >= s.n_mob) continue;  // a ragged last tile: no particle i in this sub-tile
        const int li = a * 32 + lane;
        const Tile16 pi = ti[li];
        const bool vi = i0 + li < s.n_mob;
        const bool self = diag && a == c;  // i and j from one sub-tile: j > i only
        const int j_end = min(j_lo + jlen, nj - (j0 + c * 32));
        CloseList cl{cbase + warp * kCloseCap, 0};
        for (int jj = j_lo; jj < j_end; ++jj) {
            const int lj = c * 32 + jj;
            const Tile16 pj = tj[lj];
            const bool valid = vi && (!self || lane < jj);
            const float wgt = QW ? pi.q * pj.q : 1.0f;
            bool close = false;
            pair_ring<DIM, CM, QW, kLaneRing, DIRECT>(s, ims, pi, pj, valid, wgt, ring, close, acc, tk);
            if ((jj - j_lo) % kPairsPerService<CM> == kPairsPerService<CM> - 1 || jj + 1 == j_end)
                ring_service<CM, kPairsPerService<CM>, (DIRECT == kDirectAlways && CM >= 4) ? CM - 2 : CM>(ring, acc,
                                                                                                         tk);
            const unsigned cb = __ballot_sync(0xffffffffu, close);
            if (cb) {  // uniform over the warp, rare
                const int at = cl.n + __popc(cb & ((1u << lane) - 1u));
                if (close && at < kCloseCap) cl.e[at] = ((unsigned)li << 16) | (unsigned)lj;
                cl.n += __popc(cb);
            }
        }
        if (cl.n > 0) {  // uniform over the warp; close pairs are rare
            __syncwarp();
            if (cl.n <= kCloseCap) {
                for (int e = lane; e < cl.n; e += 32) {
                    const unsigned id = cl.e[e];
                    const int gli = (int)(id >> 16), glj = (int)(id & 0xffffu);
                    float x[DIM], z2;
                    const int sc = pair_cart<DIM>(s, ti[gli], tj[glj], x, z2);
                    const int c0 = s.cand[sc * s.cand_max];
                    acc64 += close_term_global<DIM>(s, b, w, i0 + gli, j0 + glj, fixedj, c0,
                                                    (double)ti[gli].q * (double)tj[glj].q);
                }
            } else {
                // more than the list holds: find them again, lane by lane
                for (int jj = j_lo; jj < j_end; ++jj) {
                    const int lj = c * 32 + jj;
                    const Tile16 pj = tj[lj];
                    float x[DIM], z2;
                    const int sc = pair_cart<DIM>(s, pi, pj, x, z2);
                    const int c0 = s.cand[sc * s.cand_max];
                    const float r2 = image_r2<DIM>(x, s.img_f[c0], z2);
                    const bool valid = vi && (!self || lane < jj);
                    if (valid && r2 < s.rc2_f && r2 < s.close2_f)
                        acc64 += close_term_global<DIM>(s, b, w, i0 + li, j0 + lj, fixedj, c0,
                                                        (double)pi.q * (double)pj.q);
                }
            }
            __syncwarp();
        }
    }
    ring.drain(acc, tk);
    const double v = warp_sum((double)wq * acc.get() + acc64);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (tid == 0) {
        double t = 0;
        for (int k = 0; k < nw; ++k) t += red[k];
        b.part_real[(size_t)w * s.n_items + p] = t;
    }
}

// Dispatch on the candidate-list length and the charge pattern of the
// system (for kernels that take items of several systems)
template <int DIM>
__device__ void real_item_mixed(const SysDev &s, const BatchDev &b, int w, int p, const MixedImageSmem &ims,
                                unsigned char *work, int jsplit = 1) {
#define EWALD_RIM(CM)                                                                        \
    if (s.q_uniform) real_item_mixed_cm<DIM, CM, false>(s, b, w, p, ims, work, jsplit);     \
    else real_item_mixed_cm<DIM, CM, true>(s, b, w, p, ims, work, jsplit);                  \
    break;
    switch (mixed_cm(s.cand_max)) {
        case 2: EWALD_RIM(2)
        case 4: EWALD_RIM(4)
        case 6: EWALD_RIM(6)
        case 8: EWALD_RIM(8)
        default: EWALD_RIM(0)
    }
#undef EWALD_RIM
}

// real_mixed.cu: the single-system kernel, one instantiation per list
// length and charge pattern, chosen on the host
int configure_real_mixed(const SysDev &s, size_t smem, int *blocks_per_sm);
int launch_real_mixed(const SysDev &s, const BatchDev &b, int grid, size_t smem, cudaStream_t st);

}  // namespace ewald
