// Two-body plane-wave Jastrow term p (paper Sec. 2.3, Eqs. (7), (9), (10))
// of every walker of a batch, with its gradient and Laplacian with respect to
// every electron:
//
//   J_p = sum_{i<j} p(r_i - r_j),  p(r) = sum_m a_m sum_{G in star_m^+} cos(G.r)
//
// A star is a shell of simulation-cell reciprocal-lattice vectors of equal
// length, counted from the shortest; star_m^+ keeps one of each +-G pair.
// With rho(G) = sum_i e^{iG.r_i} over those G (electrons only, unit weight):
//
//   J_p    = sum_G a_G (|rho_G|^2 - N) / 2
//   grad_i = -sum_G a_G G Im(e^{iG.r_i} conj(rho_G))
//   lap_i  = -sum_G a_G |G|^2 (Re(e^{iG.r_i} conj(rho_G)) - 1)
//
// One CTA per walker: first rho over electron tiles (thread per G), then
// the derivatives (thread per electron).  Every e^{iG.r} comes from the
// exact fixed-point phase n . u (mod 2^bits), one sincospi of an exact
// fraction, so no error builds up along recurrences; sums are in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "capi_internal.h"

namespace ewald {

constexpr int kJpThreads = 256, kJpTile = 256;

struct JastrowDev {
    int n_g;
    const int4 *nvec;
    const double4 *gvec;
};

// shared memory: rho (n_g double2), the electron tile, then (32-byte
// aligned) the per-G coefficients and rho in R for the derivative pass
__host__ __device__ inline size_t jp_coef_offset(int n_g, int dim, size_t u_bytes) {
    return (align16((size_t)n_g * sizeof(double2)) + (size_t)kJpTile * dim * u_bytes + 31) / 32 * 32;
}

template <typename R, int DIM>
__global__ void __launch_bounds__(kJpThreads)
    k_jastrow_p(SysDev s, BatchDev b, JastrowDev jd, double *__restrict__ j_out, double *__restrict__ grad,
                double *__restrict__ lap) {
    using U = typename FP<R>::U;
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ double red[kJpThreads / 32];
    double2 *rho = (double2 *)smem;
    U *ut = (U *)(smem + align16((size_t)jd.n_g * sizeof(double2)));
    const int w = blockIdx.x, tid = threadIdx.x, N = s.n_mob;
    auto phase = [&](const int4 &n, const U *u) {
        U ph = (U)n.x * u[0] + (U)n.y * u[1];
        if (DIM == 3) ph += (U)n.z * u[2];
        return ph;
    };
    for (int g = tid; g < jd.n_g; g += blockDim.x) rho[g] = make_double2(0.0, 0.0);
    for (int e0 = 0; e0 < N; e0 += kJpTile) {
        const int ne = min(kJpTile, N - e0);
        __syncthreads();  // the previous tile is no longer read
        for (int t = tid; t < ne * DIM; t += blockDim.x) {
            const int e = t / DIM, k = t - e * DIM;
            ut[t] = FP<R>::from64(b.u[((size_t)w * DIM + k) * s.mob_stride + e0 + e]);
        }
        __syncthreads();
        for (int g = tid; g < jd.n_g; g += blockDim.x) {
            const int4 n = jd.nvec[g];
            // tile sums (compensated in FP32), then FP64 across tiles
            Acc<R> sx, sy;
            for (int e = 0; e < ne; ++e) {
                R sn, cs;
                FP<R>::sincospi2(FP<R>::frac(phase(n, ut + e * DIM)), &sn, &cs);
                sx.add(cs);
                sy.add(sn);
            }
            rho[g].x += sx.get();
            rho[g].y += sy.get();
        }
    }
    __syncthreads();
    double jp = 0.0;
    for (int g = tid; g < jd.n_g; g += blockDim.x) {
        const double2 r = rho[g];
        jp += jd.gvec[g].w * 0.5 * (r.x * r.x + r.y * r.y - (double)N);
    }
    jp = block_sum(jp, red);
    if (tid == 0) j_out[w] = jp;
    if (!grad && !lap) return;
    // per G: rho and the derivative weights -a G and -a |G|^2, in R
    using R2 = typename FP<R>::R4;
    R2 *cf = (R2 *)(smem + jp_coef_offset(jd.n_g, DIM, sizeof(U)));
    R2 *rr = cf + jd.n_g;
    for (int g = tid; g < jd.n_g; g += blockDim.x) {
        const double4 G = jd.gvec[g];
        R2 c, r;
        c.x = (R)(-G.w * G.x);
        c.y = (R)(-G.w * G.y);
        c.z = (R)(-G.w * G.z);
        c.w = (R)(-G.w * (G.x * G.x + G.y * G.y + G.z * G.z));
        r.x = (R)rho[g].x;
        r.y = (R)rho[g].y;
        r.z = r.w = 0;
        cf[g] = c;
        rr[g] = r;
    }
    __syncthreads();
    for (int e = tid; e < N; e += blockDim.x) {
        U u[3] = {0, 0, 0};
        for (int k = 0; k < DIM; ++k) u[k] = FP<R>::from64(b.u[((size_t)w * DIM + k) * s.mob_stride + e]);
        Acc<R> gs[3], ls;
        for (int g = 0; g < jd.n_g; ++g) {
            const int4 n = jd.nvec[g];
            R sn, cs;
            FP<R>::sincospi2(FP<R>::frac(phase(n, u)), &sn, &cs);
            const R2 r = rr[g], c = cf[g];
            // e^{iG.r_e} conj(rho) = (cs r.x + sn r.y) + i (sn r.x - cs r.y)
            const R re = cs * r.x + sn * r.y;
            const R im = sn * r.x - cs * r.y;
            gs[0].add(c.x * im);
            gs[1].add(c.y * im);
            if (DIM == 3) gs[2].add(c.z * im);
            ls.add(c.w * (re - R(1)));
        }
        const size_t o = (size_t)w * N + e;
        if (grad)
            for (int k = 0; k < DIM; ++k) grad[o * DIM + k] = gs[k].get();
        if (lap) lap[o] = ls.get();
    }
}

static size_t jastrow_smem(const SysDev &s, int n_g, int precision) {
    const size_t u = precision == EWALD_FP64 ? sizeof(unsigned long long) : sizeof(unsigned int);
    const size_t r4 = precision == EWALD_FP64 ? sizeof(Img64) : sizeof(float4);
    return jp_coef_offset(n_g, s.dim, u) + 2 * (size_t)n_g * r4;
}

int launch_jastrow_p(const SysDev &s, const BatchDev &b, int precision, const JastrowDev &jd, double *j,
                     double *grad, double *lap, cudaStream_t st) {
    const size_t smem = jastrow_smem(s, jd.n_g, precision);
    cudaError_t e;
    if (precision == EWALD_FP64) {
        if (s.dim == 3) {
            if ((e = allow_max_smem(k_jastrow_p<double, 3>, smem))) return e;
            k_jastrow_p<double, 3><<<b.W, kJpThreads, smem, st>>>(s, b, jd, j, grad, lap);
        } else {
            if ((e = allow_max_smem(k_jastrow_p<double, 2>, smem))) return e;
            k_jastrow_p<double, 2><<<b.W, kJpThreads, smem, st>>>(s, b, jd, j, grad, lap);
        }
    } else {
        if (s.dim == 3) {
            if ((e = allow_max_smem(k_jastrow_p<float, 3>, smem))) return e;
            k_jastrow_p<float, 3><<<b.W, kJpThreads, smem, st>>>(s, b, jd, j, grad, lap);
        } else {
            if ((e = allow_max_smem(k_jastrow_p<float, 2>, smem))) return e;
            k_jastrow_p<float, 2><<<b.W, kJpThreads, smem, st>>>(s, b, jd, j, grad, lap);
        }
    }
    return cudaGetLastError();
}

// The first n_stars shells of equal |G| (relative tolerance 1e-9) of the
// reciprocal lattice, one of each +-G pair (first nonzero of (n3, n2, n1)
// positive): the search sphere grows until it holds n_stars whole shells
// (a box |n_k| <= g |a_k| / 2 pi holds every G with |G| <= g).
static bool jastrow_stars(const HostTables &t, int n_stars, std::vector<int4> &nv, std::vector<double4> &gv,
                          const double *a) {
    const int dim = t.dim;
    double g = 0.0;
    for (int k = 0; k < dim; ++k) {
        double bb = 0.0;
        for (int y = 0; y < dim; ++y) bb += t.B[k][y] * t.B[k][y];
        g = std::max(g, std::sqrt(bb));
    }
    struct Gv { double g; int n[3]; double c[3]; };
    for (int iter = 0; iter < 40; ++iter, g *= 1.5) {
        int nmax[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) {
            double aa = 0.0;
            for (int y = 0; y < dim; ++y) aa += t.A[k][y] * t.A[k][y];
            nmax[k] = (int)std::ceil(g * std::sqrt(aa) / (2 * M_PI));
        }
        std::vector<Gv> all;
        for (int n3 = (dim == 3 ? -nmax[2] : 0); n3 <= (dim == 3 ? nmax[2] : 0); ++n3)
            for (int n2 = -nmax[1]; n2 <= nmax[1]; ++n2)
                for (int n1 = -nmax[0]; n1 <= nmax[0]; ++n1) {
                    if (!n1 && !n2 && !n3) continue;
                    Gv v{0.0, {n1, n2, n3}, {0.0, 0.0, 0.0}};
                    for (int y = 0; y < dim; ++y)
                        v.c[y] = n1 * t.B[0][y] + n2 * t.B[1][y] + (dim == 3 ? n3 * t.B[2][y] : 0.0);
                    v.g = std::sqrt(v.c[0] * v.c[0] + v.c[1] * v.c[1] + v.c[2] * v.c[2]);
                    if (v.g <= g) all.push_back(v);
                }
        std::sort(all.begin(), all.end(), [](const Gv &x, const Gv &y) { return x.g < y.g; });
        std::vector<double> radius;
        for (const Gv &v : all)
            if (radius.empty() || v.g > radius.back() * (1.0 + 1e-9)) radius.push_back(v.g);
        if ((int)radius.size() < n_stars) continue;
        nv.clear();
        gv.clear();
        for (const Gv &v : all) {
            int m = -1;
            for (int k = 0; k < n_stars; ++k)
                if (std::fabs(v.g / radius[k] - 1.0) <= 1e-9) m = k;
            if (m < 0) continue;
            const int lead = v.n[2] ? v.n[2] : v.n[1] ? v.n[1] : v.n[0];
            if (lead < 0) continue;  // the other one of the pair
            nv.push_back(make_int4(v.n[0], v.n[1], v.n[2], m));
            gv.push_back(make_double4(v.c[0], v.c[1], v.c[2], a[m]));
        }
        return true;
    }
    return false;
}

}  // namespace ewald

using namespace ewald;
using namespace ewald_capi;

extern "C" {

int ewald_jastrow_p_set(ewald_ctx *c, int n_stars, const double *a) {
    if (!c) return EWALD_ERR_ARG;
    if (n_stars < 1 || n_stars > 64 || !a) return fail(c, EWALD_ERR_ARG, "n_stars must be 1..64, a non-null");
    for (int m = 0; m < n_stars; ++m)
        if (!std::isfinite(a[m])) return fail(c, EWALD_ERR_ARG, "non-finite Jastrow coefficient");
    std::vector<int4> nv;
    std::vector<double4> gv;
    if (!jastrow_stars(c->t, n_stars, nv, gv, a)) return fail(c, EWALD_ERR_ARG, "stars not found");
    // replace the previous table
    for (void *p : {(void *)c->d_jp_nvec, (void *)c->d_jp_gvec}) {
        if (!p) continue;
        cudaFree(p);
        c->dev.erase(std::remove(c->dev.begin(), c->dev.end(), p), c->dev.end());
    }
    c->d_jp_nvec = nullptr;
    c->d_jp_gvec = nullptr;
    c->jp_n_g = 0;
    cudaError_t e = upload(c->dev, &c->d_jp_nvec, nv.data(), nv.size());
    if (!e) e = upload(c->dev, &c->d_jp_gvec, gv.data(), gv.size());
    if (e) return cuda_fail(c, e);
    c->jp_n_g = (int)nv.size();
    c->jp_n_stars = n_stars;
    return EWALD_OK;
}

int ewald_jastrow_p(ewald_batch *b, double *j_out, double *grad_out, double *lap_out, int on_device) {
    EWALD_NVTX("ewald_jastrow_p");
    if (!b || !b->ctx || !j_out) return fail(b ? b->ctx : nullptr, EWALD_ERR_ARG);
    ewald_ctx *c = b->ctx;
    if (!b->has_pos) return fail(c, EWALD_ERR_STATE, "positions not set");
    if (!c->jp_n_g) return fail(c, EWALD_ERR_STATE, "no Jastrow stars set (ewald_jastrow_p_set)");
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
    const JastrowDev jd{c->jp_n_g, c->d_jp_nvec, c->d_jp_gvec};
    if (!e) e = (cudaError_t)launch_jastrow_p(c->s, b->b, c->t.precision, jd, dj, dg, dl, c->stream);
    if (!e && !on_device) {
        e = cudaMemcpyAsync(j_out, dj, nj * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (!e && grad_out) e = cudaMemcpyAsync(grad_out, dg, ng * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (!e && lap_out) e = cudaMemcpyAsync(lap_out, dl, nl * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
    }
    for (void *p : tmp) cudaFree(p);
    return e ? cuda_fail(c, e) : EWALD_OK;
}

int ewald_jastrow_p_count(const ewald_ctx *c, int *n_g) {
    if (!c || !n_g) return EWALD_ERR_ARG;
    *n_g = c->jp_n_g;
    return EWALD_OK;
}

}  // extern "C"
