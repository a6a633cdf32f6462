// Polynomial two-body Jastrow term u (paper Sec. 2.3, Eq. (8)) of every
// walker of a batch, with its gradient and Laplacian with respect to every
// particle:
//
//   J_u = sum_{i<j} u_{s_i s_j}(r_ij),  u(r) = (r - L_u)^C sum_{l=0}^{N_u} alpha_l r^l  (r < L_u)
//   grad_i = sum_{j != i} u'(r_ij) x_ij / r_ij
//   lap_i  = sum_{j != i} [u''(r_ij) + (d - 1) u'(r_ij) / r_ij]
//
// r_ij is the distance to the nearest image; L_u is below half the
// shortest lattice vector, so at most one image of a pair lies inside L_u.
// Like spins (both below n_up, or both not) use one coefficient set, unlike
// spins the other; alpha_1 of each follows from the Kato cusp condition
// u'(0) = Gamma (Gamma = 1/4 like, 1/2 unlike in 3D; 1/3 and 1 in 2D).
//
// One CTA per walker: the walker's fixed-point coordinates are staged in
// shared memory and every unordered pair is evaluated once (tile pairs,
// below).  The fixed-point difference selects a displacement cell whose
// short candidate list holds the lattice vectors that can bring the pair
// inside L_u; the nearest candidate decides.  u, u', u'' come from one Horner pass for P,
// P', P''/2 and the product rule on (r - L_u)^C P(r).
#include <algorithm>
#include <cmath>
#include <vector>

#include "capi_internal.h"

namespace ewald {

constexpr int kJuThreads = 256, kJuMaxOrder = 24, kJuMaxC = 8;


template <typename R>
__device__ inline const R *ju_coef(const JuDev &j);
template <>
__device__ inline const double *ju_coef<double>(const JuDev &j) { return j.coef_d; }
template <>
__device__ inline const float *ju_coef<float>(const JuDev &j) { return j.coef_f; }
template <typename R>
__device__ inline const typename FP<R>::R4 *ju_img(const JuDev &j);
template <>
__device__ inline const Img64 *ju_img<double>(const JuDev &j) { return j.img_d; }
template <>
__device__ inline const float4 *ju_img<float>(const JuDev &j) { return j.img_f; }

// shared memory: coefficients, images (32-byte aligned), candidate lists,
// then the walker's coordinates [N][DIM]
__host__ __device__ inline size_t ju_off_img(int n_u) { return (2 * (size_t)(n_u + 1) * 8 + 31) / 32 * 32; }
__host__ __device__ inline size_t ju_off_cand(int n_u, int n_img) { return ju_off_img(n_u) + (size_t)(n_img + 1) * 32; }
__host__ __device__ inline size_t ju_off_pos(int n_u, int n_img, int n_sub, int cand_max) {
    return align16(ju_off_cand(n_u, n_img) + (size_t)n_sub * cand_max * sizeof(unsigned short));
}

// Per-particle sums of one tile side in shared memory: gradient (DIM) and
// Laplacian, with a Kahan compensation in the FP32 path.
template <typename R>
struct JuSums {
    R *s, *c;  // [DIM + 1][n_pad] each (c unused in FP64)
    int n_pad;
    __device__ void add(int q, int p, double v) {
        if constexpr (sizeof(R) == 4) {
            float &S = s[q * n_pad + p], &C = c[q * n_pad + p];
            const float y = (float)v - C, t = S + y;
            C = (t - S) - y;
            S = t;
        } else {
            s[q * n_pad + p] += v;
        }
    }
    __device__ double get(int q, int p) const {
        if constexpr (sizeof(R) == 4) return (double)s[q * n_pad + p] - (double)c[q * n_pad + p];
        else return s[q * n_pad + p];
    }
};

// One CTA per walker, 32-particle tiles.  Every unordered pair is evaluated
// once: a warp takes a tile pair (A, B), lane l holds particle i = 32 A + l
// and walks the 32 j of B; i's gradient and Laplacian stay in the lane's
// registers, j's (the opposite gradient, the same Laplacian term) are summed
// over the warp for each j and kept by lane j.  Tile pairs are scheduled in
// rounds of disjoint pairs (a round-robin schedule), so no two warps touch a
// tile's sums in one round; the diagonal tiles (A, A) form the last round,
// with every ordered pair and i's side only.  Sums go to shared memory per
// particle in a fixed order: the result does not depend on timing.
template <typename R, int DIM>
__global__ void __launch_bounds__(kJuThreads)
    k_jastrow_u(SysDev s, BatchDev b, JuDev ju, double *__restrict__ j_out, double *__restrict__ grad,
                double *__restrict__ lap) {
    using T = FP<R>;
    using U = typename T::U;
    using I = typename T::I;
    using R4 = typename T::R4;
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ double red[kJuThreads / 32];
    const int w = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int N = s.n_mob, nt = (N + 31) / 32, n_pad = nt * 32;
    const int n_sub = 1 << (ju.sub_bits * DIM), nc = ju.n_u + 1;
    R *cf = (R *)smem;
    R4 *im = (R4 *)(smem + ju_off_img(ju.n_u));
    unsigned short *cd = (unsigned short *)(smem + ju_off_cand(ju.n_u, ju.n_img));
    const size_t off_pos = ju_off_pos(ju.n_u, ju.n_img, n_sub, ju.cand_max);
    U *up = (U *)(smem + off_pos);
    JuSums<R> sums;
    sums.n_pad = n_pad;
    sums.s = (R *)(smem + align16(off_pos + (size_t)n_pad * DIM * sizeof(U)));
    sums.c = sums.s + (size_t)(DIM + 1) * n_pad;
    for (int t = tid; t < 2 * nc; t += blockDim.x) cf[t] = ju_coef<R>(ju)[t];
    for (int t = tid; t <= ju.n_img; t += blockDim.x) im[t] = ju_img<R>(ju)[t];
    for (int t = tid; t < n_sub * ju.cand_max; t += blockDim.x) cd[t] = ju.cand[t];
    for (int t = tid; t < n_pad * DIM; t += blockDim.x) {
        const int e = t / DIM, k = t - e * DIM;
        up[t] = e < N ? T::from64(b.u[((size_t)w * DIM + k) * s.mob_stride + e]) : (U)0;
    }
    for (int t = tid; t < (DIM + 1) * n_pad * (sizeof(R) == 4 ? 2 : 1); t += blockDim.x) sums.s[t] = R(0);
    __syncthreads();
    const R L = sizeof(R) == 4 ? (R)ju.L_f : (R)ju.L, L2 = sizeof(R) == 4 ? (R)ju.L2_f : (R)ju.L2;
    const R coin2 = T::coin2(s);
    const int C = ju.C;

    // pair (i, j): false if j's nearest image is not inside L; else u, the
    // vector g = u'(r) (r_i - r_j) / r and the Laplacian term u'' + (d-1) u'/r
    auto pair = [&](const U *ui, int i, int j, R &u, R *g, R &lt) -> bool {
        I d[DIM];
        int sc = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            d[k] = (I)(ui[k] - up[j * DIM + k]);
            if (ju.sub_bits) {
                const U h = (U)d[k] + ((U)1 << (T::BITS - 1));
                sc |= (int)(h >> (T::BITS - ju.sub_bits)) << (k * ju.sub_bits);
            }
        }
        R x[DIM];
#pragma unroll
        for (int y = 0; y < DIM; ++y) {
            R v = 0;
#pragma unroll
            for (int k = 0; k < DIM; ++k) v = T::lat_lo(s, k, y, (R)d[k], v);
#pragma unroll
            for (int k = 0; k < DIM; ++k) v = T::lat(s, k, y, (R)d[k], v);
            x[y] = v;
        }
        // the nearest candidate image (the only one that can be inside L)
        R r2 = R(1e30), xs[DIM];
        for (int c = 0; c < ju.cand_max; ++c) {
            const R4 Rv = im[cd[sc * ju.cand_max + c]];
            const R y0 = x[0] + Rv.x, y1 = x[1] + Rv.y;
            R rr = y0 * y0 + y1 * y1;
            R y2 = 0;
            if (DIM == 3) {
                y2 = x[DIM - 1] + Rv.z;
                rr += y2 * y2;
            }
            if (rr < r2) {
                r2 = rr;
                xs[0] = y0;
                xs[1] = y1;
                if (DIM == 3) xs[DIM - 1] = y2;
            }
        }
        if (!(r2 < L2)) return false;
        if (r2 < coin2) {  // two particles on top of each other: flag, skip
            atomicOr(b.status, ST_COINCIDENT);
            return false;
        }
        const R rinv = sizeof(R) == 4 ? (R)rsqrt_nr((float)r2) : R(1) / sqrt(r2);
        const R r = r2 * rinv;
        // P, P', P''/2 by Horner
        const R *a = cf + (((i < ju.n_up) == (j < ju.n_up)) ? nc : 0);
        R p = a[ju.n_u], p1 = 0, p2 = 0;
        for (int l = ju.n_u - 1; l >= 0; --l) {
            p2 = p2 * r + p1;
            p1 = p1 * r + p;
            p = p * r + a[l];
        }
        // (r - L)^(C-2), (r - L)^(C-1), (r - L)^C
        const R t = r - L;
        R tc2 = 1;
        for (int k = 2; k < C; ++k) tc2 *= t;
        const R tc1 = C >= 2 ? tc2 * t : R(1), tc = tc1 * t;
        u = tc * p;
        const R du = R(C) * tc1 * p + tc * p1;
        const R d2u = (C >= 2 ? R(C * (C - 1)) * tc2 * p : R(0)) + R(2 * C) * tc1 * p1 + R(2) * tc * p2;
        const R gr = du * rinv;
#pragma unroll
        for (int k = 0; k < DIM; ++k) g[k] = gr * xs[k];
        lt = d2u + R(DIM - 1) * gr;
        return true;
    };

    Acc<R> jacc;  // this lane's share of J
    const int nt2 = nt + (nt & 1);  // round-robin over an even number of tiles (the extra one is a bye)
    const int n_rounds = nt2 - 1;
    for (int rnd = 0; rnd <= n_rounds; ++rnd) {
        const bool diag = rnd == n_rounds;
        const int n_jobs = diag ? nt : nt2 / 2;
        for (int job = warp; job < n_jobs; job += nw) {
            int A, B;
            if (diag) {
                A = B = job;
            } else if (job == 0) {
                A = rnd;
                B = nt2 - 1;
            } else {
                A = (rnd + job) % (nt2 - 1);
                B = (rnd - job + nt2 - 1) % (nt2 - 1);
            }
            if (A >= nt || B >= nt) continue;  // the bye
            if (A > B) {
                const int t = A;
                A = B;
                B = t;
            }
            const int i = A * 32 + lane;
            const bool vi = i < N;
            U ui[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) ui[k] = up[i * DIM + k];
            Acc<R> gi[DIM], li, gj[DIM], lj;  // i's sums; lane jj keeps j = 32 B + jj's
            for (int jj = 0; jj < 32; ++jj) {
                const int j = B * 32 + jj;
                if (j >= N) break;  // uniform over the warp
                R u = 0, g[DIM], lt = 0;
#pragma unroll
                for (int k = 0; k < DIM; ++k) g[k] = 0;
                const bool ok = vi && j != i && pair(ui, i, j, u, g, lt);
                if (ok) {
#pragma unroll
                    for (int k = 0; k < DIM; ++k) gi[k].add(g[k]);
                    li.add(lt);
                    jacc.add(diag ? R(0.5) * u : u);
                }
                if (!diag) {  // j's side: -g and lt summed over the warp's i
                    R v[DIM + 1];
#pragma unroll
                    for (int k = 0; k < DIM; ++k) v[k] = ok ? -g[k] : R(0);
                    v[DIM] = ok ? lt : R(0);
#pragma unroll
                    for (int k = 0; k <= DIM; ++k) v[k] = warp_sum(v[k]);
                    if (lane == jj) {
#pragma unroll
                        for (int k = 0; k < DIM; ++k) gj[k].add(v[k]);
                        lj.add(v[DIM]);
                    }
                }
            }
            if (vi) {
#pragma unroll
                for (int k = 0; k < DIM; ++k) sums.add(k, i, gi[k].get());
                sums.add(DIM, i, li.get());
            }
            const int jl = B * 32 + lane;
            if (!diag && jl < N) {
#pragma unroll
                for (int k = 0; k < DIM; ++k) sums.add(k, jl, gj[k].get());
                sums.add(DIM, jl, lj.get());
            }
        }
        __syncthreads();  // the next round's pairs share tiles with this round's
    }
    for (int p = tid; p < N; p += blockDim.x) {
        const size_t o = (size_t)w * N + p;
        if (grad)
            for (int k = 0; k < DIM; ++k) grad[o * DIM + k] = sums.get(k, p);
        if (lap) lap[o] = sums.get(DIM, p);
    }
    const double jsum = block_sum(jacc.get(), red);
    if (tid == 0) j_out[w] = jsum;
}

static size_t ju_smem(const SysDev &s, const JuDev &ju, int precision) {
    const size_t u = precision == EWALD_FP64 ? sizeof(unsigned long long) : sizeof(unsigned int);
    const size_t r = precision == EWALD_FP64 ? 8 : 2 * 4;  // a sum (and its compensation) per quantity
    const int n_sub = 1 << (ju.sub_bits * s.dim), n_pad = (s.n_mob + 31) / 32 * 32;
    return align16(ju_off_pos(ju.n_u, ju.n_img, n_sub, ju.cand_max) + (size_t)n_pad * s.dim * u) +
           (size_t)(s.dim + 1) * n_pad * r;
}

int launch_jastrow_u(const SysDev &s, const BatchDev &b, int precision, const JuDev &ju, double *j, double *grad,
                     double *lap, cudaStream_t st) {
    const size_t smem = ju_smem(s, ju, precision);
    cudaError_t e;
    if (precision == EWALD_FP64) {
        if (s.dim == 3) {
            if ((e = allow_max_smem(k_jastrow_u<double, 3>, smem))) return e;
            k_jastrow_u<double, 3><<<b.W, kJuThreads, smem, st>>>(s, b, ju, j, grad, lap);
        } else {
            if ((e = allow_max_smem(k_jastrow_u<double, 2>, smem))) return e;
            k_jastrow_u<double, 2><<<b.W, kJuThreads, smem, st>>>(s, b, ju, j, grad, lap);
        }
    } else {
        if (s.dim == 3) {
            if ((e = allow_max_smem(k_jastrow_u<float, 3>, smem))) return e;
            k_jastrow_u<float, 3><<<b.W, kJuThreads, smem, st>>>(s, b, ju, j, grad, lap);
        } else {
            if ((e = allow_max_smem(k_jastrow_u<float, 2>, smem))) return e;
            k_jastrow_u<float, 2><<<b.W, kJuThreads, smem, st>>>(s, b, ju, j, grad, lap);
        }
    }
    return cudaGetLastError();
}

}  // namespace ewald

using namespace ewald;
using namespace ewald_capi;

extern "C" {

int ewald_jastrow_u_set(ewald_ctx *c, int n_up, double L_u, int C, int n_u, const double *alpha_like,
                        const double *alpha_unlike) {
    if (!c) return EWALD_ERR_ARG;
    const HostTables &t = c->t;
    if (n_up < 0 || n_up > t.n_mob) return fail(c, EWALD_ERR_ARG, "n_up must be 0..n_mobile");
    if (C < 1 || C > kJuMaxC) return fail(c, EWALD_ERR_ARG, "C must be 1..8");
    if (n_u < 1 || n_u > kJuMaxOrder) return fail(c, EWALD_ERR_ARG, "N_u must be 1..24");
    if (!alpha_like || !alpha_unlike) return fail(c, EWALD_ERR_ARG, "coefficients are NULL");
    if (!std::isfinite(L_u) || !(L_u > 0) || !(2 * L_u < shortest_lattice_vector(t)))
        return fail(c, EWALD_ERR_ARG, "L_u must be positive and below half the shortest lattice vector");
    for (int l = 0; l <= n_u; ++l)
        if (!std::isfinite(alpha_like[l]) || !std::isfinite(alpha_unlike[l]))
            return fail(c, EWALD_ERR_ARG, "non-finite Jastrow coefficient");
    // tables: coefficients with the cusp alpha_1, images, candidate lists
    std::vector<double> cf(2 * (size_t)(n_u + 1));
    for (int set = 0; set < 2; ++set) {  // 0: unlike spins, 1: like spins
        const double *a = set ? alpha_like : alpha_unlike;
        const double gamma = t.dim == 3 ? (set ? 0.25 : 0.5) : (set ? 1.0 / 3.0 : 1.0);
        for (int l = 0; l <= n_u; ++l) cf[set * (n_u + 1) + l] = a[l];
        cf[set * (n_u + 1) + 1] = gamma / std::pow(-L_u, C) + C * a[0] / L_u;
    }
    std::vector<double> img;
    std::vector<unsigned short> cand;
    int bits = 0;
    const int cand_max = short_range_lists(t, L_u, t.dim == 3 ? 3 : 5, &img, &cand, &bits);
    const int n_img = (int)img.size() / 3;
    if (n_img >= 65535) return fail(c, EWALD_ERR_ARG, "too many images for the u term");
    std::vector<Img64> imd(n_img + 1);
    std::vector<float4> imf(n_img + 1);
    for (int i = 0; i < n_img; ++i) {
        imd[i] = Img64{img[3 * i], img[3 * i + 1], img[3 * i + 2], 0.0};
        imf[i] = make_float4((float)img[3 * i], (float)img[3 * i + 1], (float)img[3 * i + 2], 0.f);
    }
    imd[n_img] = Img64{1e18, 1e18, 1e18, 0.0};
    imf[n_img] = make_float4(1e18f, 1e18f, 1e18f, 0.f);
    std::vector<float> cff(cf.begin(), cf.end());
    std::vector<void *> fresh_dev;
    JuDev d{};
    d.n_up = n_up;
    d.C = C;
    d.n_u = n_u;
    d.sub_bits = bits;
    d.cand_max = std::max(cand_max, 1);
    d.n_img = n_img;
    d.L = L_u;
    d.L2 = L_u * L_u;
    d.L_f = (float)L_u;
    d.L2_f = (float)(L_u * L_u);
    auto drop = [&]() {
        for (void *p : fresh_dev) cudaFree(p);
    };
    cudaError_t e = upload(fresh_dev, (double **)&d.coef_d, cf.data(), cf.size());
    if (!e) e = upload(fresh_dev, (float **)&d.coef_f, cff.data(), cff.size());
    if (!e) e = upload(fresh_dev, (Img64 **)&d.img_d, imd.data(), imd.size());
    if (!e) e = upload(fresh_dev, (float4 **)&d.img_f, imf.data(), imf.size());
    if (!e) e = upload(fresh_dev, (unsigned short **)&d.cand, cand.data(), cand.size());
    if (e) {
        drop();
        return cuda_fail(c, e);
    }
    // shared memory of one walker's CTA must fit
    int dev = 0, optin = 0;
    if (!e) e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e) {
        drop();
        return cuda_fail(c, e);
    }
    if (ju_smem(c->s, d, t.precision) + 4096 > (size_t)optin) {
        drop();
        return fail(c, EWALD_ERR_ARG, "too many particles for the u term's shared-memory tile");
    }
    // replace the previous tables (kernels that read them are ordered
    // before this point by the synchronisation below)
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (void *p : c->ju_dev) cudaFree(p);
    c->ju_dev = fresh_dev;
    c->ju = d;
    c->ju_set = true;
    return EWALD_OK;
}

int ewald_jastrow_u(ewald_batch *b, double *j_out, double *grad_out, double *lap_out, int on_device) {
    EWALD_NVTX("ewald_jastrow_u");
    if (!b || !b->ctx || !j_out) return fail(b ? b->ctx : nullptr, EWALD_ERR_ARG);
    ewald_ctx *c = b->ctx;
    if (!b->has_pos) return fail(c, EWALD_ERR_STATE, "positions not set");
    if (!c->ju_set) return fail(c, EWALD_ERR_STATE, "no u term set (ewald_jastrow_u_set)");
    const int W = b->b.W, N = c->s.n_mob, dim = c->s.dim;
    const size_t nj = (size_t)W, ng = (size_t)W * N * dim, nl = (size_t)W * N;
    double *dj = j_out, *dg = grad_out, *dl = lap_out;
    std::vector<void *> tmp;
    cudaError_t e = cudaSuccess;
    if (!on_device) {  // device scratch for host outputs
        e = dalloc(tmp, &dj, nj);
        if (!e && grad_out) e = dalloc(tmp, &dg, ng);
        if (!e && lap_out) e = dalloc(tmp, &dl, nl);
    }
    if (!e) e = (cudaError_t)launch_jastrow_u(c->s, b->b, c->t.precision, c->ju, dj, dg, dl, c->stream);
    if (!e && !on_device) {
        e = cudaMemcpyAsync(j_out, dj, nj * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (!e && grad_out) e = cudaMemcpyAsync(grad_out, dg, ng * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (!e && lap_out) e = cudaMemcpyAsync(lap_out, dl, nl * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
    }
    for (void *p : tmp) cudaFree(p);
    if (e) return cuda_fail(c, e);
    return EWALD_OK;
}

}  // extern "C"
