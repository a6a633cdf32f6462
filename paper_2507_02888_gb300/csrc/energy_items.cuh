// Work items of the full-energy path, as device functions shared by the
// single-system kernels (energy_kernels.cu) and the persistent multi-system
// kernel (multi_kernels.cu).
//
//   sfac_item : rho(G) of one walker over one chunk of G runs, and that
//               chunk's reciprocal energy (paper Eq. (3) / Eq. (5) at z = 0,
//               powers of e^{i b_k . r} buffered as in Eq. (10));
//   real_item : real-space pair sum of one walker over one tile pair
//               (Eq. (3), second term);
//   combine_walker : E = E_real + E_madR + E_recip + E_self + E_bg (Eq. (2)).
#pragma once
#include "device_common.cuh"

namespace ewald {

__host__ __device__ inline size_t sfac_bytes(const SysDev &s, int precision, int te, int threads) {
    size_t part = precision == EWALD_FP64 ? sizeof(Part<double>) : sizeof(Part<float>);
    size_t cx = precision == EWALD_FP64 ? sizeof(Cx<double>) : sizeof(Cx<float>);
    int W = (2 * s.n1max + 1) + (2 * s.n2max + 1) + (s.dim == 3 ? s.n3max + 1 : 0);
    return align16(te * part) + align16((size_t)te * W * cx) + align16((threads / 32) * sizeof(double));
}

// tiered: the FP32 tiles and queues of the mixed path plus the head queues
__host__ __device__ inline size_t real_work_bytes(const SysDev &s, int precision, int warps, bool tiered = false) {
    const bool f64 = precision == EWALD_FP64 && !tiered;
    size_t part = f64 ? sizeof(Part<double>) : sizeof(Part<float>);
    size_t qe = f64 ? kQueueCap64 * sizeof(QE<double>) : kQueueCap32 * sizeof(QE<float>);
    return 2 * align16(s.tile * part) + align16((size_t)warps * qe) +
           align16((size_t)warps * kCloseCap * sizeof(unsigned)) + align16(kRealUnits * sizeof(double)) +
           (tiered ? align16((size_t)warps * kHeadCap * sizeof(uint2)) : 0);
}

// Tables of one electron tile in shared memory (see sfac_item).
template <typename R>
struct SfacTile {
    const Part<R> *tp;
    const Cx<R> *P1, *P2, *P3;
    int W1, W2, W3, n1max, n2max, ne;
};

// Sum of one G slot over all electrons, its x and y parts together.
// FP64: plain.  FP32: Kahan compensated, term by term (the FP32 form's
// compensated accumulation per G), both parts' steps as paired
// instructions (FADD2: each part rounds as the scalar steps would; fcc
// N = 1024 structure factor 4.85 -> 4.34 ms per launch of 4096 walkers
// against scalar FADDs); stored as the float pair hi + lo.
template <typename R>
struct SlotSumXY;
template <>
struct SlotSumXY<double> {
    double sx = 0, sy = 0;
    __device__ void add(double tx, double ty) {
        sx += tx;
        sy += ty;
    }
    __device__ void get(double &x, double &y) const {
        x = sx;
        y = sy;
    }
};
template <>
struct SlotSumXY<float> {
    float2 s = {0.f, 0.f}, c = {0.f, 0.f};
    __device__ void add(float tx, float ty) {
        const float2 y = add2(make_float2(tx, ty), neg2(c)), u = add2(s, y);
        c = add2(add2(u, neg2(s)), neg2(y));
        s = u;
    }
    __device__ void get(double &x, double &y) const {
        x = (double)s.x - (double)c.x;
        y = (double)s.y - (double)c.y;
    }
    // s - c of each part as an unevaluated float pair hi + lo, exactly
    // (|c| <= ulp(s))
    __device__ void split(float &hx, float &lx, float &hy, float &ly) const {
        hx = __fsub_rn(s.x, c.x);
        lx = __fsub_rn(__fsub_rn(s.x, hx), c.x);
        hy = __fsub_rn(s.y, c.y);
        ly = __fsub_rn(__fsub_rn(s.y, hy), c.y);
    }
};

// One thread's run over the tile's electrons: the run's first G from three
// buffered powers, then one complex multiplication per G along n1.  Two
// electrons (four in 2D) are walked side by side, so independent
// multiplication chains are in flight, and their terms enter the slot sums
// together.
// L is the longest run of the warp (compile-time, so the sums stay in
// registers and the warp does no steps past its longest run).
template <typename R, int DIM, int L>
__device__ __forceinline__ void sfac_runs(const SfacTile<R> &t, int4 rn, int dir, SlotSumXY<R> *axy) {
    using C = Cx<R>;
    // the run's first term q e^{iG.r} (the charge rides along the recurrence)
    auto start = [&](int e, C &z, C &step) {
        z = cmul(t.P1[(size_t)e * t.W1 + rn.x + t.n1max], t.P2[(size_t)e * t.W2 + rn.y + t.n2max]);
        if (DIM == 3) z = cmul(z, t.P3[(size_t)e * t.W3 + rn.z]);
        const R q = t.tp[e].q;
        z = {q * z.x, q * z.y};
        step = t.P1[(size_t)e * t.W1 + t.n1max + dir];
    };
    int e = 0;
    if constexpr (DIM == 2) {
        // in 2D (two buffered powers per start) four chains side by side
        // pay: 2D gas N = 338, 0.297 -> 0.231 ms per structure factor of
        // 2048 walkers; in 3D they were slower (fcc 4.85 -> 4.91 ms)
        for (; e + 3 < t.ne; e += 4) {
            C za, sa, zb, sb, zc, sc, zd, sd;
            start(e, za, sa);
            start(e + 1, zb, sb);
            start(e + 2, zc, sc);
            start(e + 3, zd, sd);
#pragma unroll
            for (int r = 0; r < L; ++r) {
                if (r < rn.w) {
                    axy[r].add((za.x + zb.x) + (zc.x + zd.x), (za.y + zb.y) + (zc.y + zd.y));
                    if (r + 1 < L) {
                        za = cmul(za, sa);
                        zb = cmul(zb, sb);
                        zc = cmul(zc, sc);
                        zd = cmul(zd, sd);
                    }
                }
            }
        }
    }
    for (; e + 1 < t.ne; e += 2) {
        C za, sa, zb, sb;
        start(e, za, sa);
        start(e + 1, zb, sb);
#pragma unroll
        for (int r = 0; r < L; ++r) {
            if (r < rn.w) {
                axy[r].add(za.x + zb.x, za.y + zb.y);
                if (r + 1 < L) {
                    za = cmul(za, sa);
                    zb = cmul(zb, sb);
                }
            }
        }
    }
    if (e < t.ne) {
        C z, st;
        start(e, z, st);
#pragma unroll
        for (int r = 0; r < L; ++r) {
            if (r < rn.w) {
                axy[r].add(z.x, z.y);
                if (r + 1 < L) z = cmul(z, st);
            }
        }
    }
}

// One CTA; the first s.sfac_threads threads each own one run of <= kRunLen
// consecutive n1 in a row (n2, n3), walked away from the row's smallest |G|
// (chunk c holds runs c * sfac_threads ...; other threads only help stage).  Electrons are staged in tiles of te; for each
// electron of the tile the CTA buffers the powers e^{2 pi i n f_k},
// n = -n_max..n_max, built by repeated multiplication from the base phase.
// A thread starts its run from the product of three buffered powers and
// steps along n1 by one complex multiplication per G.  Tile sums are in R
// and are added into FP64.
// LAYERED: a layered 2D cell, one pass per layer (sfac_item_layers).
template <typename R, int DIM, bool LAYERED>
__device__ __forceinline__ void sfac_item_body(const SysDev &s, const BatchDev &b, int w, int chunk, int te,
                                               bool write_energy, unsigned char *smem) {
    using C = Cx<R>;
    const int W1 = 2 * s.n1max + 1, W2 = 2 * s.n2max + 1, W3 = DIM == 3 ? s.n3max + 1 : 0;
    Part<R> *tp = (Part<R> *)smem;
    C *P1 = (C *)(smem + align16(te * sizeof(Part<R>)));
    C *P2 = P1 + (size_t)te * W1;
    C *P3 = P2 + (size_t)te * W2;
    double *red = (double *)(smem + align16(te * sizeof(Part<R>)) + align16((size_t)te * (W1 + W2 + W3) * sizeof(C)));

    const int tid = threadIdx.x;
    const int run = chunk * s.sfac_threads + tid;
    const bool has = tid < s.sfac_threads && run < s.n_runs;
    const int4 rn0 = has ? s.runs[run] : make_int4(0, 0, 0, 0);
    const int dir = rn0.w < 0 ? -1 : 1;             // the run walks n1 = start + dir * r
    const int4 rn = make_int4(rn0.x, rn0.y, rn0.z, rn0.w * dir);
    // runs are stored longest first, so lane 0 holds the warp's longest run
    const int wmax = __shfl_sync(0xffffffffu, rn.w, 0);
    const int slots = s.n_runs * s.run_len;
    double epart = 0;
    // one pass per layer (a single pass unless the cell is layered 2D); each
    // layer's rho goes to its own slots
    const int nl = LAYERED ? s.n_layers : 1;
    for (int L = 0; L < nl; ++L) {
        SlotSumXY<R> axy[kRunLen];
        const int e_lo = nl > 1 ? s.lay_start[L] : 0, e_hi = nl > 1 ? s.lay_start[L + 1] : s.n_mob;
        for (int e0 = e_lo; e0 < e_hi; e0 += te) {
            const int ne = min(te, e_hi - e0);
            __syncthreads();  // the previous tile's tables are no longer read
            for (int t = tid; t < ne; t += blockDim.x)
                tp[t] = load_mobile<R>(s, b, w, nl > 1 ? s.lay_idx[e0 + t] : e0 + t, DIM);
            __syncthreads();
            // powers by repeated multiplication (Eq. (10))
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
            const SfacTile<R> tl{tp, P1, P2, P3, W1, W2, W3, s.n1max, s.n2max, ne};
            switch (wmax) {  // uniform over the warp: the loop stops at the warp's longest run
                case 8: sfac_runs<R, DIM, 8>(tl, rn, dir, axy); break;
                case 7: sfac_runs<R, DIM, 7>(tl, rn, dir, axy); break;
                case 6: sfac_runs<R, DIM, 6>(tl, rn, dir, axy); break;
                case 5: sfac_runs<R, DIM, 5>(tl, rn, dir, axy); break;
                case 4: sfac_runs<R, DIM, 4>(tl, rn, dir, axy); break;
                case 3: sfac_runs<R, DIM, 3>(tl, rn, dir, axy); break;
                case 2: sfac_runs<R, DIM, 2>(tl, rn, dir, axy); break;
                case 1: sfac_runs<R, DIM, 1>(tl, rn, dir, axy); break;
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
                    if constexpr (sizeof(R) == 4) {
                        // the float pair of the compensated sum goes to memory as it is
                        float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
                        if (r < rn.w) {
                            axy[r].split(hx, lx, hy, ly);
                        }
                        v = make_double2((double)hx + (double)lx, (double)hy + (double)ly);
                        if (rfix && r < rn.w) {
                            v.x += rfix[slot].x;
                            v.y += rfix[slot].y;
                            RhoIO<R>::set(rho, slot, v);
                        } else {
                            ((float4 *)rho)[slot] = make_float4(hx, hy, lx, ly);
                        }
                    } else {
                        if (r < rn.w) {
                            axy[r].get(v.x, v.y);
                            if (rfix) {
                                v.x += rfix[slot].x;
                                v.y += rfix[slot].y;
                            }
                        }
                        RhoIO<R>::set(rho, slot, v);
                    }
                    if (nl == 1 && r < rn.w) epart += s.gw_d[slot] * (v.x * v.x + v.y * v.y);
                }
            }
        }
    }
    if (nl > 1 && has) {
        // layered: sum_{L,L'} W_{LL'}(G) Re(rho_L conj(rho_L')) over this
        // thread's slots, from the values it has just stored
        const double2 *rho = b.rho + (size_t)w * nl * slots;
        for (int r = 0; r < s.run_len && r < rn.w; ++r) {
            const int slot = r * s.n_runs + run;
            for (int L = 0; L < nl; ++L) {
                const double2 a = RhoIO<R>::get(rho, (size_t)L * slots + slot);
                epart += s.gwl_d[((size_t)L * nl + L) * slots + slot] * (a.x * a.x + a.y * a.y);
                for (int M = L + 1; M < nl; ++M) {
                    const double2 c = RhoIO<R>::get(rho, (size_t)M * slots + slot);
                    epart += 2.0 * s.gwl_d[((size_t)L * nl + M) * slots + slot] * (a.x * c.x + a.y * c.y);
                }
            }
        }
    }
    if (write_energy) {
        double tot = block_sum(epart, red);
        if (tid == 0) b.part_recip[(size_t)w * s.n_gchunks + chunk] = tot;
    }
}

// The layered pass out of line: its extra loop and epilogue stay out of the
// register allocation of the kernels' single-plane path.
template <typename R, int DIM>
__device__ __noinline__ void sfac_item_layers(const SysDev &s, const BatchDev &b, int w, int chunk, int te,
                                              bool write_energy, unsigned char *smem) {
    sfac_item_body<R, DIM, true>(s, b, w, chunk, te, write_energy, smem);
}

template <typename R, int DIM>
__device__ inline void sfac_item(const SysDev &s, const BatchDev &b, int w, int chunk, int te, bool write_energy,
                                 unsigned char *smem) {
    if (DIM == 2 && s.n_layers > 1) sfac_item_layers<R, DIM>(s, b, w, chunk, te, write_energy, smem);
    else sfac_item_body<R, DIM, false>(s, b, w, chunk, te, write_energy, smem);
}

// One CTA, any number of warps.  The tile pair's particles are staged in
// shared memory; each warp takes units of a 32 x 32 sub-tile (lane = i,
// loop over j), diagonal tiles only their upper triangle.  A unit is the
// whole sub-tile (jsplit = 1) or one of jsplit equal slices of its 32 j, so
// that CTAs with more warps than sub-tiles keep every warp busy.  Images
// inside the cutoff go through the warp queue.  Every unit is summed on its
// own and the unit sums are added in unit order in FP64, so the item's
// partial sum depends on jsplit but not on how many warps the CTA has.
// ims must already hold this system's images; work is this item's scratch
// (its reduction array holds kRealUnits doubles: nst * jsplit must fit).
// TIER (R = float only): the tiered FP64 form, head terms in FP64 (see
// pair_images_tiered); close pairs are head terms there.
template <typename R, int DIM, bool TIER = false>
__device__ void real_item(const SysDev &s, const BatchDev &b, int w, int p, const ImageSmem<R> &ims,
                          unsigned char *work, int jsplit = 1, const float4 *img_lo = nullptr) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    size_t off = 0;
    Part<R> *ti = (Part<R> *)(work + off);
    off += align16(s.tile * sizeof(Part<R>));
    Part<R> *tj = (Part<R> *)(work + off);
    off += align16(s.tile * sizeof(Part<R>));
    QE<R> *qbase = (QE<R> *)(work + off);
    off += align16((size_t)nw * kQueueCapOf<R> * sizeof(QE<R>));
    unsigned *cbase = (unsigned *)(work + off);
    off += align16((size_t)nw * kCloseCap * sizeof(unsigned));
    double *red = (double *)(work + off);
    off += align16(kRealUnits * sizeof(double));
    uint2 *hbase = (uint2 *)(work + off);  // head queues (TIER only)

    const int S = s.tile / 32;
    const int2 tt = s.items[p];
    const bool fixedj = tt.y >= s.n_mob_tiles;
    const int i0 = tt.x * s.tile;
    const int j0 = (fixedj ? tt.y - s.n_mob_tiles : tt.y) * s.tile;
    const int nj = fixedj ? s.n_fix : s.n_mob;
    __syncthreads();  // the previous item's tiles are no longer read
    for (int t = tid; t < s.tile; t += blockDim.x) {
        ti[t] = load_mobile<R>(s, b, w, i0 + t, DIM);
        tj[t] = fixedj ? load_fixed<R>(s, j0 + t, DIM) : load_mobile<R>(s, b, w, j0 + t, DIM);
    }
    __syncthreads();
    WarpQueue<R> wq{qbase + warp * kQueueCapOf<R>, 0, FP<R>::coin2(s), b.status};
    const typename FP<R>::K tk = FP<R>::term_consts(s);
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
        const int li = a * 32 + lane;
        const Part<R> pi = ti[li];
        const bool vi = i0 + li < s.n_mob;
        auto valid = [&](int jj) { return vi && (j0 + c * 32 + jj < nj) && (!(diag && a == c) || lane < jj); };
        Acc<R> acc;
        CloseList cl{cbase + warp * kCloseCap, 0};
        if constexpr (TIER) {
            HeadQueue hq{hbase + warp * kHeadCap, 0};
            DF hacc = {0.0f, 0.0f};  // head terms, double-float
            for (int jj = j_lo; jj < j_lo + jlen; ++jj) {
                const int lj = c * 32 + jj;
                pair_images_tiered<DIM>(s, pi, tj[lj], valid(jj), ims.img, img_lo, ims.cand, wq, hq, acc, hacc,
                                        lane, ((unsigned)li << 16) | (unsigned)lj, ti, tj, i0, j0, fixedj);
            }
            wq.drain(acc, tk, lane);
            __syncwarp();
            if (lane < hq.n)
                head_term_df<DIM>(s, ti, tj, ims.img, img_lo, i0, j0, fixedj, hq.q[lane], b.status, hacc);
            __syncwarp();
            acc.add64(df_to(hacc));
        } else {
            for (int jj = j_lo; jj < j_lo + jlen; ++jj) {
                const int lj = c * 32 + jj;
                pair_images<R, DIM, true>(s, pi, tj[lj], valid(jj), R(1), ims.img, ims.cand, wq, acc, lane, &cl,
                                          ((unsigned)li << 16) | (unsigned)lj);
            }
            wq.drain(acc, tk, lane);
        }
        if constexpr (sizeof(R) == 4 && !TIER) {
            if (cl.n > 0) {  // uniform over the warp; close pairs are rare
                __syncwarp();
                if (cl.n <= kCloseCap) {
                    for (int e = lane; e < cl.n; e += 32) {
                        const unsigned id = cl.e[e];
                        const Part<R> &pa = ti[id >> 16], &pb = tj[id & 0xffffu];
                        const int c0 = ims.cand[pair_geom<R, DIM>(s, pa, pb).sc * s.cand_max];
                        acc.add64(close_pair_term<DIM>(s, pa, pb, c0, (double)(R(1) * pa.q * pb.q), b.status));
                    }
                } else {
                    // more than the list holds: find them again, with the
                    // same arithmetic as pair_images, lane by lane
                    for (int jj = j_lo; jj < j_lo + jlen; ++jj) {
                        const Part<R> &pb = tj[c * 32 + jj];
                        const PairGeom<R, DIM> g = pair_geom<R, DIM>(s, pi, pb);
                        const int c0 = ims.cand[g.sc * s.cand_max];
                        const R r2 = image_r2<DIM>(g.x, ims.img[c0], g.z2);
                        const bool pass = r2 < (valid(jj) ? FP<R>::rc2(s) : R(0));
                        if (is_close_first<R, DIM>(s, r2, pass))
                            acc.add64(close_pair_term<DIM>(s, pi, pb, c0, (double)(R(1) * pi.q * pb.q), b.status));
                    }
                }
                __syncwarp();
            }
        }
        const double v = warp_sum(acc.get());
        if (lane == 0) red[u] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0;
        for (int k = 0; k < nunits; ++k) t += red[k];
        b.part_real[(size_t)w * s.n_items + p] = t;
    }
}

// E = E_real + E_madR + E_recip + E_self + E_bg for walker w; partial sums
// are added in a fixed order, so the result does not depend on scheduling.
__device__ inline double combine_walker(const SysDev &s, const BatchDev &b, int w) {
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
    const double e = er + s.e_madR + ek + s.e_self + s.e_bg;
    b.e[w] = e;
    b.acc_count[w] = 0;
    b.pend_k[w] = -1;
    return e;
}

}  // namespace ewald
