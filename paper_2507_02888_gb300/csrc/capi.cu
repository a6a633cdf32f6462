// C ABI of the library (include/ewald.h): object lifetimes, argument checks,
// host<->device staging and error reporting.  All numerical work is in the
// kernels of energy_kernels.cu and move_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <set>
#include <sstream>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "capi_internal.h"
#include "real_mixed.cuh"
#include "move_tiered.h"
#include "multi.h"
#include "sfac_df.h"

using namespace ewald;

namespace {

using namespace ewald_capi;

unsigned long long to_fixed(double f) {
    f -= std::floor(f);
    if (f >= 1.0) f = 0.0;
    return (unsigned long long)std::ldexp(f, 64);
}

// The structure factor in n_ch chunks of G runs per walker (whole warps,
// at most kSfacThreads runs each; the launch configuration follows).
void set_sfac_chunks(SysDev &s, int n_ch) {
    n_ch = std::max(n_ch, (s.n_runs + kSfacThreads - 1) / kSfacThreads);
    s.sfac_threads = std::min(kSfacThreads, ((s.n_runs + n_ch - 1) / n_ch + 31) / 32 * 32);
    s.n_gchunks = (s.n_runs + s.sfac_threads - 1) / s.sfac_threads;
}

void free_one(std::vector<void *> &v, const void *p) {
    if (!p) return;
    for (size_t i = 0; i < v.size(); ++i)
        if (v[i] == p) {
            cudaFree(v[i]);
            v.erase(v.begin() + i);
            return;
        }
}

// Real-space tiling of a context: pair tiles of 32 x S particles per side
// and 2^bits displacement cells per axis; rebuilds the candidate lists and
// the item table on the device and the launch configuration.
int apply_tiling(ewald_ctx *c, int S, int bits) {
    HostTables &t = c->t;
    SysDev &s = c->s;
    cudaError_t e;
    if (bits != t.sub_bits || t.cand.empty()) set_subcells(&t, bits);
    free_one(c->dev, s.cand);
    free_one(c->dev, s.cxy);
    free_one(c->dev, s.cz);
    free_one(c->dev, s.clist);
    free_one(c->dev, s.cxy_mv);  // no-ops where they alias the energy kernels' tables
    free_one(c->dev, s.cz_mv);
    free_one(c->dev, s.clist_mv);
    free_one(c->dev, s.items);
    s.cand = nullptr;
    s.cxy = nullptr;
    s.cz = nullptr;
    s.clist = nullptr;
    s.cxy_mv = nullptr;
    s.cz_mv = nullptr;
    s.clist_mv = nullptr;
    s.items = nullptr;
    s.sub_bits = t.sub_bits;
    s.cand_max = t.cand_max;
    if ((e = upload(c->dev, (unsigned short **)&s.cand, t.cand.data(), t.cand.size()))) return cuda_fail(c, e);
    {   // the mixed loop's tables: distinct lists as pairs of FP32 images;
        // the move kernel's copy keeps the lists of cand where the energy
        // kernels' differ (mixed_direct)
        const int np = mixed_pairs(t.cand_max), n_sub = (int)(t.cand.size() / std::max(t.cand_max, 1));
        const int pstride = np | 1;  // odd: consecutive lists start in different banks
        auto imf = [&](int i, int y) {  // FP32 image component, as in the FP32 image table
            return i < s.n_img ? (float)t.img[3 * i + y] : 1e18f;
        };
        struct Tables {
            std::vector<unsigned short> clist;
            std::vector<float4> cxy;
            std::vector<float2> cz;
            int n_lists = 0;
        };
        auto tables = [&](const std::vector<unsigned short> &order, Tables &o) {
            std::map<std::vector<unsigned short>, int> ids;
            o.clist.assign(n_sub, 0);
            for (int r = 0; r < n_sub; ++r) {
                std::vector<unsigned short> l(2 * np, (unsigned short)s.n_img);
                std::copy(order.begin() + (size_t)r * t.cand_max, order.begin() + (size_t)(r + 1) * t.cand_max,
                          l.begin());
                auto it = ids.find(l);
                if (it == ids.end()) {
                    it = ids.emplace(l, (int)ids.size()).first;
                    for (int p = 0; p < pstride; ++p) {  // pairs past np: padding between lists
                        const int a = p < np ? l[2 * p] : s.n_img, b = p < np ? l[2 * p + 1] : s.n_img;
                        o.cxy.push_back(make_float4(imf(a, 0), imf(b, 0), imf(a, 1), imf(b, 1)));
                        o.cz.push_back(make_float2(t.dim == 3 ? imf(a, 2) : 0.0f, t.dim == 3 ? imf(b, 2) : 0.0f));
                    }
                }
                o.clist[r] = (unsigned short)it->second;
            }
            o.n_lists = (int)ids.size();
            return ids.size() <= 65535;
        };
        s.mixed_direct = mixed_direct_pays(t) ? 1 : 0;
        Tables te, tm;
        if (!tables(mixed_cand_order(t, s.mixed_direct), te) || (s.mixed_direct && !tables(t.cand, tm)))
            return fail(c, EWALD_ERR_ARG, "too many distinct candidate lists");
        s.n_lists = te.n_lists;
        s.cand_pairs = np;
        s.cand_pstride = pstride;
        if ((e = upload(c->dev, (float4 **)&s.cxy, te.cxy.data(), te.cxy.size()))) return cuda_fail(c, e);
        if ((e = upload(c->dev, (float2 **)&s.cz, te.cz.data(), te.cz.size()))) return cuda_fail(c, e);
        if ((e = upload(c->dev, (unsigned short **)&s.clist, te.clist.data(), te.clist.size()))) return cuda_fail(c, e);
        if (s.mixed_direct) {
            s.n_lists_mv = tm.n_lists;
            if ((e = upload(c->dev, (float4 **)&s.cxy_mv, tm.cxy.data(), tm.cxy.size()))) return cuda_fail(c, e);
            if ((e = upload(c->dev, (float2 **)&s.cz_mv, tm.cz.data(), tm.cz.size()))) return cuda_fail(c, e);
            if ((e = upload(c->dev, (unsigned short **)&s.clist_mv, tm.clist.data(), tm.clist.size())))
                return cuda_fail(c, e);
        } else {
            s.n_lists_mv = s.n_lists;
            s.cxy_mv = s.cxy;
            s.cz_mv = s.cz;
            s.clist_mv = s.clist;
        }
    }
    s.tile = 32 * S;
    s.n_mob_tiles = (t.n_mob + s.tile - 1) / s.tile;
    int nft = (t.n_fix + s.tile - 1) / s.tile;
    std::vector<int2> items;
    for (int i = 0; i < s.n_mob_tiles; ++i) {
        for (int j = i; j < s.n_mob_tiles; ++j) items.push_back(make_int2(i, j));
        for (int f = 0; f < nft; ++f) items.push_back(make_int2(i, s.n_mob_tiles + f));
    }
    s.n_items = (int)items.size();
    if ((e = upload(c->dev, (int2 **)&s.items, items.data(), items.size()))) return cuda_fail(c, e);
    if ((e = (cudaError_t)configure_launch(s, t.precision, &c->cfg))) return cuda_fail(c, e);
    return EWALD_OK;
}

size_t mixed_table_bytes(const HostTables &t0, int bits);

// A tuned configuration: real-space tiling, the mixed form's CTA warps
// (warps > 0) and the structure-factor chunks (chunks > 0).
int apply_config(ewald_ctx *c, int S, int bits, int warps, int chunks) {
    if (warps > 0) c->s.real_warps = warps;
    if (chunks > 0) set_sfac_chunks(c->s, chunks);
    return apply_tiling(c, S, bits);
}

// The real-space tiling a context starts with (the autotuner or its cache
// may change it): pair tiles of 32 x S particles per side, 2^bits
// displacement cells per axis and, for the mixed form, warps per real-space
// CTA (0: not the mixed form).  The largest item count (S = 1) sizes the
// batches' partial-sum buffers, so any tiling fits later.
static void default_tiling(const HostTables &t, int *S_out, int *bits_out, int *warps_out) {
    int S = t.n_mob >= 128 ? 4 : (t.n_mob >= 64 ? 2 : 1);
    int bits = t.sub_bits, warps = 0;
    if (t.precision == EWALD_MIXED) {
        // the mixed form's pair loop takes 256-particle tiles (no limit on
        // the units of an item: a quarter of the item boundaries) where they
        // pad the pairs no more than 128-particle tiles do
        auto padded = [&](int T) { return std::ceil(t.n_mob / (double)T) * T; };
        if (t.n_mob >= 256 && padded(256) <= padded(128)) S = 8;
        // and candidate tables that leave room for its CTAs
        while (bits > t.min_bits && mixed_table_bytes(t, bits) > kMixedTableBytes) --bits;
        // CTAs of 16 warps for 256-particle tiles, 8 for smaller ones (an item
        // then still gives every warp several units)
        warps = S == 8 ? 16 : 8;
    }
    *S_out = S;
    *bits_out = bits;
    *warps_out = warps;
}

int build_device(ewald_ctx *c) {
    HostTables &t = c->t;
    SysDev &s = c->s;
    std::vector<void *> &o = c->dev;
    const int dim = t.dim;
    s.dim = dim;
    s.n_mob = t.n_mob;
    s.n_fix = t.n_fix;
    s.mob_stride = (t.n_mob + 31) / 32 * 32;
    s.fix_stride = std::max(1, (t.n_fix + 31) / 32 * 32);
    for (int k = 0; k < 3; ++k)
        for (int x = 0; x < 3; ++x) {
            s.A[k][x] = t.A[k][x];
            s.A64[k][x] = std::ldexp(t.A[k][x], -64);
            s.A32[k][x] = (float)std::ldexp(t.A[k][x], -32);
            s.A32lo[k][x] = (float)(std::ldexp(t.A[k][x], -32) - (double)s.A32[k][x]);
            s.Binv[k][x] = t.Ainv[x][k];
        }
    s.q_uniform = 1;
    for (double q : t.q_mob) s.q_uniform &= (float)q == (float)t.q_mob[0];
    for (double q : t.q_fix) s.q_uniform &= (float)q == (float)t.q_fix[0];
    s.alpha = t.alpha;
    s.alpha_f = (float)t.alpha;
    s.alpha_lo_f = (float)(t.alpha - (double)s.alpha_f);
    s.alpha2_f = (float)(t.alpha * t.alpha);
    s.alpha2_lo_f = (float)(t.alpha * t.alpha - (double)s.alpha2_f);
    s.rc2 = t.r_c * t.r_c;
    s.rc2_f = (float)s.rc2;
    double L = std::pow(t.volume, 1.0 / dim);
    s.coin2 = 1e-20 * L * L;
    s.coin2_f = (float)s.coin2;
    // close radius of the FP32 path (set-up: r_close)
    s.close2_f = (float)(t.r_close * t.r_close);
    {   // tiered FP64: FP64 for images with erfc(alpha r) > kTierErfc
        double x = 3.0;  // erfc(x) = kTierErfc by Newton steps on log erfc
        for (int it = 0; it < 50; ++it) {
            const double f = std::log(std::erfc(x)) - std::log(kTierErfc);
            const double fp = -2.0 / std::sqrt(M_PI) * std::exp(-x * x) / std::erfc(x);
            x -= f / fp;
        }
        const double rt = x / t.alpha;
        s.tier2_f = t.tiered ? (float)(rt * rt) : 0.0f;
    }
    cudaError_t e;
    // images
    int n_img = (int)t.img.size() / 3;
    std::vector<Img64> imd(n_img + 1);
    std::vector<float4> imf(n_img + 1), iml(n_img + 1, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int i = 0; i < n_img; ++i) {
        imd[i] = Img64{t.img[3 * i], t.img[3 * i + 1], t.img[3 * i + 2], 0.0};
        imf[i] = make_float4((float)t.img[3 * i], (float)t.img[3 * i + 1], (float)t.img[3 * i + 2], 0.f);
        iml[i] = make_float4((float)(t.img[3 * i] - (double)imf[i].x), (float)(t.img[3 * i + 1] - (double)imf[i].y),
                             (float)(t.img[3 * i + 2] - (double)imf[i].z), 0.f);
    }
    // sentinel that pads the candidate lists: |d + R|^2 ~ 3e36 never passes the cutoff
    imd[n_img] = Img64{1e18, 1e18, 1e18, 0.0};
    imf[n_img] = make_float4(1e18f, 1e18f, 1e18f, 0.f);
    s.n_img = n_img;
    if ((e = upload(o, (Img64 **)&s.img_d, imd.data(), imd.size()))) return cuda_fail(c, e);
    if ((e = upload(o, (float4 **)&s.img_f, imf.data(), imf.size()))) return cuda_fail(c, e);
    if ((e = upload(o, (float4 **)&s.img_lo_f, iml.data(), iml.size()))) return cuda_fail(c, e);
    // reciprocal
    s.n_runs = (int)t.runs.size() / 4;
    s.run_len = t.run_len;
    s.n_gh = (int)t.g2slot.size();
    // as few chunks as kSfacThreads allows, split evenly (whole warps)
    set_sfac_chunks(s, (s.n_runs + kSfacThreads - 1) / kSfacThreads);
    c->max_gchunks = (s.n_runs + 31) / 32;  // the finest chunking (32 runs each) sizes the partial sums
    s.real_warps = kRealMixedWarps;
    s.n1max = std::max(t.n1max, 1);
    s.n2max = std::max(t.n2max, 1);
    s.n3max = std::max(t.n3max, 1);
    std::vector<int4> runs(s.n_runs);
    for (int r = 0; r < s.n_runs; ++r)
        runs[r] = make_int4(t.runs[4 * r], t.runs[4 * r + 1], t.runs[4 * r + 2], t.runs[4 * r + 3]);
    if ((e = upload(o, (int4 **)&s.runs, runs.data(), runs.size()))) return cuda_fail(c, e);
    std::vector<float> gwf(t.gw.begin(), t.gw.end());
    if ((e = upload(o, (double **)&s.gw_d, t.gw.data(), t.gw.size()))) return cuda_fail(c, e);
    if ((e = upload(o, (float **)&s.gw_f, gwf.data(), gwf.size()))) return cuda_fail(c, e);
    s.rho_fix = nullptr;
    if (t.n_fix > 0) {
        std::vector<double2> rf(t.rho_fix.size() / 2);
        for (size_t i = 0; i < rf.size(); ++i) rf[i] = make_double2(t.rho_fix[2 * i], t.rho_fix[2 * i + 1]);
        if ((e = upload(o, (double2 **)&s.rho_fix, rf.data(), rf.size()))) return cuda_fail(c, e);
    }
    if ((e = upload(o, &c->d_g2slot, t.g2slot.data(), t.g2slot.size()))) return cuda_fail(c, e);
    // charges and fixed particles
    std::vector<float> qmf(t.q_mob.begin(), t.q_mob.end()), qff(t.q_fix.begin(), t.q_fix.end());
    if ((e = upload(o, (double **)&s.q_mob, t.q_mob.data(), t.q_mob.size()))) return cuda_fail(c, e);
    if ((e = upload(o, (float **)&s.q_mob_f, qmf.data(), qmf.size()))) return cuda_fail(c, e);
    if ((e = upload(o, (double **)&s.q_fix, t.q_fix.data(), t.q_fix.size()))) return cuda_fail(c, e);
    if ((e = upload(o, (float **)&s.q_fix_f, qff.data(), qff.size()))) return cuda_fail(c, e);
    {
        auto pairs = [](const std::vector<double> &q) {
            std::vector<float2> v(std::max<size_t>(q.size(), 1), make_float2(0.f, 0.f));
            for (size_t i = 0; i < q.size(); ++i) {
                const float h = (float)q[i];
                v[i] = make_float2(h, (float)(q[i] - (double)h));
            }
            return v;
        };
        const std::vector<float2> qm = pairs(t.q_mob), qf = pairs(t.q_fix);
        if ((e = upload(o, (float2 **)&s.q_mob_df, qm.data(), qm.size()))) return cuda_fail(c, e);
        if ((e = upload(o, (float2 **)&s.q_fix_df, qf.data(), qf.size()))) return cuda_fail(c, e);
    }
    std::vector<unsigned long long> fu((size_t)dim * s.fix_stride, 0ull);
    for (int I = 0; I < t.n_fix; ++I)
        for (int k = 0; k < dim; ++k) {
            double f = 0;
            for (int x = 0; x < dim; ++x) f += t.Ainv[x][k] * t.fix_pos[(size_t)I * dim + x];
            fu[(size_t)k * s.fix_stride + I] = to_fixed(f);
        }
    if ((e = upload(o, (unsigned long long **)&s.fix_u, fu.data(), fu.size()))) return cuda_fail(c, e);
    s.e_madR = t.e_madR;
    s.e_self = t.e_self;
    s.e_bg = t.e_bg;
    s.e_II = t.e_II;
    // layered 2D
    s.n_layers = t.n_layers;
    for (int L = 0; L <= EWALD_MAX_LAYERS; ++L) s.lay_start[L] = L < (int)t.lay_start.size() ? t.lay_start[L] : 0;
    s.lay_start[0] = 0;
    if (t.n_layers == 1) s.lay_start[1] = t.n_mob;
    s.lay_idx = nullptr;
    s.mob_layer = nullptr;
    s.z_mob = s.z_fix = s.gwl_d = nullptr;
    s.z_mob_f = s.z_fix_f = s.gwl_f = nullptr;
    if (t.n_layers > 1) {
        std::vector<unsigned char> ml(t.mob_layer.begin(), t.mob_layer.end());
        std::vector<float> zmf(t.z_mob.begin(), t.z_mob.end()), gwlf(t.gwl.begin(), t.gwl.end());
        std::vector<double> zf(t.z_fix);
        if (zf.empty()) zf.push_back(0.0);
        std::vector<float> zff(zf.begin(), zf.end());
        if ((e = upload(o, (int **)&s.lay_idx, t.lay_idx.data(), t.lay_idx.size()))) return cuda_fail(c, e);
        if ((e = upload(o, (unsigned char **)&s.mob_layer, ml.data(), ml.size()))) return cuda_fail(c, e);
        if ((e = upload(o, (double **)&s.z_mob, t.z_mob.data(), t.z_mob.size()))) return cuda_fail(c, e);
        if ((e = upload(o, (float **)&s.z_mob_f, zmf.data(), zmf.size()))) return cuda_fail(c, e);
        if ((e = upload(o, (double **)&s.z_fix, zf.data(), zf.size()))) return cuda_fail(c, e);
        if ((e = upload(o, (float **)&s.z_fix_f, zff.data(), zff.size()))) return cuda_fail(c, e);
        if ((e = upload(o, (double **)&s.gwl_d, t.gwl.data(), t.gwl.size()))) return cuda_fail(c, e);
        if ((e = upload(o, (float **)&s.gwl_f, gwlf.data(), gwlf.size()))) return cuda_fail(c, e);
    }
    int S, bits, warps;
    default_tiling(t, &S, &bits, &warps);
    if (warps > 0) s.real_warps = warps;
    {
        int nt1 = (t.n_mob + 31) / 32, nf1 = (t.n_fix + 31) / 32;
        c->max_items = nt1 * (nt1 + 1) / 2 + nt1 * nf1;
    }
    return apply_tiling(c, S, bits);
}

// The structure factor of a context's batch: the tiered FP64 form takes the
// double-float kernel, every other form its own precision's.
int run_sfac(ewald_ctx *c, const BatchDev &b, int precision, const unsigned char *only) {
    if (c->t.tiered) return launch_sfac_df(c->s, b, c->cfg, only, c->stream);
    return launch_sfac(c->s, b, precision, c->cfg, only, c->stream);
}

cudaEvent_t take_event(ewald_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Run one launcher, bracketed by events when the context's timers are on.
template <typename F>
int timed(ewald_ctx *c, int kid, F &&launch) {
    if (!c->timing) return launch();
    cudaEvent_t a = take_event(c), b = take_event(c);
    cudaEventRecord(a, c->stream);
    int e = launch();
    cudaEventRecord(b, c->stream);
    c->ev_open.push_back({kid, {a, b}});
    return e;
}

int collect_timers(ewald_ctx *c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    for (auto &o : c->ev_open) {
        float ms = 0;
        if (!e) e = cudaEventElapsedTime(&ms, o.second.first, o.second.second);
        c->t_ms[o.first] += ms;
        c->t_n[o.first] += 1;
        c->ev_pool.push_back(o.second.first);
        c->ev_pool.push_back(o.second.second);
    }
    c->ev_open.clear();
    return e;
}

void free_all(std::vector<void *> &v) {
    for (void *p : v) cudaFree(p);
    v.clear();
}

// Wait for the stream and turn device-side error bits into an error code.
int sync_status(ewald_batch *b) {
    ewald_ctx *c = b->ctx;
    int *h = (int *)b->pin;
    cudaError_t e = cudaMemcpyAsync(h, b->b.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e);
    int st = *h;
    if (!st) return EWALD_OK;
    if ((e = cudaMemsetAsync(b->b.status, 0, sizeof(int), c->stream))) return cuda_fail(c, e);
    if (st & ST_DEBUG_RANGE) {
        c->why = "debug build: a kernel caught an index out of range (check at source line " +
                 std::to_string((st >> 8) & 0xffff) + ")";
        return fail(c, EWALD_ERR_STATE);
    }
    if (st & ST_COINCIDENT) return fail(c, EWALD_ERR_COINCIDENT, "coincident particles");
    if (st & ST_TIMEOUT) return fail(c, EWALD_ERR_TIMEOUT, "device wait timed out");
    return fail(c, EWALD_ERR_ARG, st & ST_BAD_INDEX ? "move index or position invalid" : "non-finite position");
}

// Page-locked host memory (cudaMallocHost / cudaHostRegister): copied by
// DMA directly, without the staging buffer.
bool is_pinned_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // not a pointer CUDA knows: ordinary host memory
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// Copy n bytes of device memory to a host or device destination.
int copy_out(ewald_batch *b, void *dst, const void *src, size_t n, int on_device) {
    ewald_ctx *c = b->ctx;
    cudaError_t e;
    if (on_device) {
        e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, c->stream);
        return e ? cuda_fail(c, e) : EWALD_OK;
    }
    if (is_pinned_host(dst)) {
        e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, c->stream);
        if (e) return cuda_fail(c, e);
        return sync_status(b);
    }
    // status word first, then the payload behind it in the pinned buffer
    char *pin = (char *)b->pin;
    e = cudaMemcpyAsync(pin + 16, src, n, cudaMemcpyDeviceToHost, c->stream);
    if (e) return cuda_fail(c, e);
    int st = sync_status(b);
    std::memcpy(dst, pin + 16, n);
    return st;
}

// Stage a host array into device scratch; returns the device pointer.
const void *copy_in(ewald_batch *b, const void *src, size_t n, void *dscratch, int *err) {
    ewald_ctx *c = b->ctx;
    const bool direct = is_pinned_host(src);
    char *pin = (char *)b->pin + 16;
    if (!direct) std::memcpy(pin, src, n);
    cudaError_t e = cudaMemcpyAsync(dscratch, direct ? src : pin, n, cudaMemcpyHostToDevice, c->stream);
    if (e) {
        *err = cuda_fail(c, e);
        return nullptr;
    }
    // the staging buffer (or the caller's array) is reused after the call
    // returns: wait for the copy
    if ((e = cudaStreamSynchronize(c->stream))) {
        *err = cuda_fail(c, e);
        return nullptr;
    }
    *err = EWALD_OK;
    return dscratch;
}

// Structure factor + reciprocal energy, real-space pairs, combine (paper
// Sec. 5.1: independent reciprocal and real-space loops, then a combine).
int run_energy(ewald_batch *b) {
    ewald_ctx *c = b->ctx;
    const int p = c->t.precision;
    int e = timed(c, KT_SFAC, [&] { return run_sfac(c, b->b, p, nullptr); });
    if (!e) e = timed(c, KT_REAL, [&] { return launch_real(c->s, b->b, p, c->cfg, c->stream); });
    if (!e) e = timed(c, KT_COMBINE, [&] { return launch_combine(c->s, b->b, c->stream); });
    if (e) return cuda_fail(c, (cudaError_t)e);
    b->rho_stale = false;
    return EWALD_OK;
}

// rho(G) is rebuilt lazily after new positions: by the next energy, or here
// by the first call that reads it without one.
int ensure_rho(ewald_batch *b) {
    if (!b->rho_stale) return EWALD_OK;
    ewald_ctx *c = b->ctx;
    int e = timed(c, KT_RESUM, [&] { return run_sfac(c, b->b, c->t.precision, nullptr); });
    if (e) return cuda_fail(c, (cudaError_t)e);
    b->rho_stale = false;
    return EWALD_OK;
}

// ---------------------------------------------------------------- autotune
// Cache file: one JSON object {"entries": [{"key": K, "tile": T, "bits": B,
// "ms": X}, ...]}, one entry per line, keyed by the system's shape.

std::string tune_key(const ewald_ctx *c) {
    const HostTables &t = c->t;
    std::ostringstream k;
    k.precision(9);
    k << "dim=" << t.dim << " n=" << t.n_mob << " nfix=" << t.n_fix << " prec=" << (t.tiered ? 2 : t.precision)
      << " alpha=" << t.alpha << " rc=" << t.r_c << " gc=" << t.g_c << " A=";
    for (int i = 0; i < t.dim; ++i)
        for (int j = 0; j < t.dim; ++j) k << t.A[i][j] << (i == t.dim - 1 && j == t.dim - 1 ? "" : ",");
    int dev = 0;
    cudaDeviceProp pr;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&pr, dev) == cudaSuccess) k << " gpu=" << pr.name;
    return k.str();
}

struct TuneEntry {
    int tile, bits;
    double ms;
    int warps = 0, chunks = 0;  // real-space CTA warps (mixed form), structure-factor chunks (0: default)
};

std::map<std::string, TuneEntry> read_tune_cache(const char *path) {
    std::map<std::string, TuneEntry> m;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        size_t a = line.find("\"key\": \"");
        if (a == std::string::npos) continue;
        a += 8;
        size_t b = line.find('"', a);
        if (b == std::string::npos) continue;
        TuneEntry e{0, 0, 0};
        size_t p;
        if ((p = line.find("\"tile\": ", b)) != std::string::npos) e.tile = std::atoi(line.c_str() + p + 8);
        if ((p = line.find("\"bits\": ", b)) != std::string::npos) e.bits = std::atoi(line.c_str() + p + 8);
        if ((p = line.find("\"ms\": ", b)) != std::string::npos) e.ms = std::atof(line.c_str() + p + 6);
        if ((p = line.find("\"warps\": ", b)) != std::string::npos) e.warps = std::atoi(line.c_str() + p + 9);
        if ((p = line.find("\"chunks\": ", b)) != std::string::npos) e.chunks = std::atoi(line.c_str() + p + 10);
        if (e.tile == 32 || e.tile == 64 || e.tile == 128 || e.tile == 256) m[line.substr(a, b - a)] = e;
    }
    return m;
}

bool write_tune_cache(const char *path, const std::map<std::string, TuneEntry> &m) {
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{\"entries\": [\n");
    size_t i = 0;
    for (auto &kv : m)
        std::fprintf(f, "  {\"key\": \"%s\", \"tile\": %d, \"bits\": %d, \"warps\": %d, \"chunks\": %d, \"ms\": %.6f}%s\n",
                     kv.first.c_str(), kv.second.tile, kv.second.bits, kv.second.warps, kv.second.chunks,
                     kv.second.ms, ++i < m.size() ? "," : "");
    std::fprintf(f, "]}\n");
    std::fclose(f);
    return std::rename(tmp.c_str(), path) == 0;
}

// Shared memory of the mixed loop's candidate tables for 2^bits cells per
// axis: the distinct candidate lists as pairs of FP32 images.
size_t mixed_table_bytes(const HostTables &t0, int bits) {
    HostTables t = t0;
    if (bits != t.sub_bits || t.cand.empty()) set_subcells(&t, bits);
    const int np = mixed_pairs(t.cand_max), n_sub = (int)(t.cand.size() / std::max(t.cand_max, 1));
    std::set<std::vector<unsigned short>> lists;
    const std::vector<unsigned short> mc = mixed_cand_order(t, mixed_direct_pays(t));
    for (int r = 0; r < n_sub; ++r)
        lists.insert(std::vector<unsigned short>(mc.begin() + (size_t)r * t.cand_max,
                                                 mc.begin() + (size_t)(r + 1) * t.cand_max));
    return lists.size() * (np | 1) * (t.dim == 3 ? sizeof(float4) + sizeof(float2) : sizeof(float4));
}

bool tiling_allowed(const ewald_ctx *c, int S, int bits) {
    const HostTables &t = c->t;
    if (32 * S > std::max(32, 2 * t.n_mob)) return false;
    // 256-particle tiles: the mixed form's pair loop only (the FP64 and tiered
    // loops sum at most 16 sub-tile units per item)
    if (S > 4 && (t.precision != EWALD_MIXED || S != 8)) return false;
    int max_bits = t.dim == 3 ? 4 : 6;
    if (bits < t.min_bits || bits > max_bits || subcell_bytes(t, bits) > 48 * 1024) return false;
    return t.precision != EWALD_MIXED || mixed_table_bytes(t, bits) <= kMixedTableBytes;
}

bool ready(ewald_batch *b) {
    if (!b || !b->ctx) return false;
    if (!b->has_pos) {
        fail(b->ctx, EWALD_ERR_STATE, "positions not set");
        return false;
    }
    return true;
}

}  // namespace

extern "C" {

int ewald_build_flags(void) {
#ifdef EWALD_DEBUG
    return EWALD_BUILD_DEBUG_CHECKS;
#else
    return 0;
#endif
}

const char *ewald_strerror(int code) {
    switch (code) {
        case EWALD_OK: return "ok";
        case EWALD_ERR_ARG: return "invalid argument";
        case EWALD_ERR_LATTICE: return "singular or left-handed lattice";
        case EWALD_ERR_COINCIDENT: return "coincident particles";
        case EWALD_ERR_NO_PROPOSAL: return "accept without a pending proposal";
        case EWALD_ERR_OOM: return "out of memory";
        case EWALD_ERR_CUDA: return "CUDA runtime error";
        case EWALD_ERR_TIMEOUT: return "device wait timed out";
        case EWALD_ERR_STATE: return "call not valid in the current state";
        case EWALD_ERR_CANCELLED: return "request cancelled";
        default: return "unknown error";
    }
}

int ewald_create(const ewald_desc *desc, void *cuda_stream, ewald_ctx **out) {
    EWALD_NVTX("ewald_create");
    if (!out) return EWALD_ERR_ARG;
    *out = nullptr;
    ewald_ctx *c = new (std::nothrow) ewald_ctx();
    if (!c) return EWALD_ERR_OOM;
    int st = build_tables(desc, &c->t, &c->why);
    if (st) {
        delete c;
        return st;
    }
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreate(&c->stream);
        if (e) {
            delete c;
            return EWALD_ERR_CUDA;
        }
        c->own_stream = true;
    }
    st = build_device(c);
    if (st) {
        ewald_destroy(c);
        return st;
    }
    if (const char *path = std::getenv("EWALD_TUNE_CACHE")) {
        auto cache = read_tune_cache(path);
        auto it = cache.find(tune_key(c));
        if (it != cache.end() && tiling_allowed(c, it->second.tile / 32, it->second.bits)) {
            st = apply_config(c, it->second.tile / 32, it->second.bits, it->second.warps, it->second.chunks);
            if (st) {
                ewald_destroy(c);
                return st;
            }
        }
    }
    *out = c;
    return EWALD_OK;
}

static void destroy_now(ewald_ctx *c) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    collect_timers(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    free_all(c->dev);
    free_all(c->ju_dev);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

void ewald_destroy(ewald_ctx *c) {
    if (!c) return;
    if (c->n_batches > 0) {  // freed when its last batch is destroyed
        c->destroy_pending = true;
        return;
    }
    destroy_now(c);
}

// ewald_info of host tables t with pair tiles of `tile` particles per side
static void fill_info(const HostTables &t, int tile, int mixed_direct, ewald_info *i) {
    i->dim = t.dim;
    i->n_mobile = t.n_mob;
    i->n_fixed = t.n_fix;
    i->precision = t.tiered ? EWALD_FP64_TIERED : t.precision;
    i->alpha = t.alpha;
    i->r_cutoff = t.r_c;
    i->g_cutoff = t.g_c;
    i->volume = t.volume;
    i->n_g_half = (int)t.g2slot.size();
    i->n_images = (int)t.img.size() / 3;
    i->subcell_bits = t.sub_bits;
    i->pair_tile = tile;
    i->max_candidates = t.cand_max;
    i->n_runs = (int)t.runs.size() / 4;
    i->run_len = t.run_len;
    i->e_madelung = t.e_madR;
    i->e_self = t.e_self;
    i->e_background = t.e_bg;
    i->e_fixed_real = t.e_II;
    i->n_layers = t.n_layers;
    i->mixed_direct = mixed_direct;
}

int ewald_get_info(const ewald_ctx *c, ewald_info *i) {
    if (!c || !i) return EWALD_ERR_ARG;
    fill_info(c->t, c->s.tile, c->s.mixed_direct, i);
    return EWALD_OK;
}

int ewald_plan(const ewald_desc *desc, ewald_info *i) {
    EWALD_NVTX("ewald_plan");
    if (!desc || !i) return EWALD_ERR_ARG;
    HostTables t;
    std::string why;
    const int st = build_tables(desc, &t, &why);
    if (st) return st;
    int S, bits, warps;
    default_tiling(t, &S, &bits, &warps);
    if (bits != t.sub_bits || t.cand.empty()) set_subcells(&t, bits);
    fill_info(t, 32 * S, mixed_direct_pays(t) ? 1 : 0, i);
    return EWALD_OK;
}

int ewald_get_gvectors(const ewald_ctx *c, int *nvec) {
    if (!c || !nvec) return EWALD_ERR_ARG;
    std::memcpy(nvec, c->t.gn.data(), c->t.gn.size() * sizeof(int));
    return EWALD_OK;
}

const char *ewald_last_error_message(const ewald_ctx *c) {
    if (!c) return "no context";
    return c->why.c_str();
}

int ewald_last_error(const ewald_ctx *c) {
    if (!c) return EWALD_ERR_ARG;
    int e = c->last_error;
    const_cast<ewald_ctx *>(c)->last_error = EWALD_OK;
    return e;
}

int ewald_batch_create(ewald_ctx *c, int W, ewald_batch **out) {
    EWALD_NVTX("ewald_batch_create");
    if (!out) return fail(c, EWALD_ERR_ARG);
    *out = nullptr;
    if (!c || W < 1) return fail(c, EWALD_ERR_ARG, "need a context and W >= 1");
    ewald_batch *b = new (std::nothrow) ewald_batch();
    if (!b) return fail(c, EWALD_ERR_OOM);
    b->ctx = c;
    const SysDev &s = c->s;
    BatchDev &d = b->b;
    d.W = W;
    const size_t slots = (size_t)s.n_runs * s.run_len * s.n_layers;  // rho of every layer
    std::vector<void *> &o = b->dev;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (!e) e = x; };
    chk(dalloc(o, &d.u, (size_t)W * s.dim * s.mob_stride));
    chk(dalloc(o, &d.rho, (size_t)W * slots));
    chk(dalloc(o, &d.pend_k, W));
    chk(dalloc(o, &d.pend_u, (size_t)W * 3));
    chk(dalloc(o, &d.acc_count, W));
    chk(dalloc(o, &d.resum_flag, W));
    chk(dalloc(o, &d.resum_list, (size_t)W + 1));
    chk(dalloc(o, &d.part_real, (size_t)W * std::max(c->max_items, s.n_items)));
    chk(dalloc(o, &d.part_recip, (size_t)W * std::max(c->max_gchunks, s.n_gchunks)));
    chk(dalloc(o, &d.e, W));
    chk(dalloc(o, &d.comp, (size_t)W * 5));
    chk(dalloc(o, &d.status, 1));
    chk(dalloc(o, &b->d_k, W));
    chk(dalloc(o, &b->d_rnew, (size_t)W * 3));
    chk(dalloc(o, &b->d_de, W));
    chk(dalloc(o, &b->d_acc, W));
    size_t io = std::max({(size_t)W * s.n_mob * s.dim, (size_t)W * s.n_layers * s.n_gh * 2, (size_t)W * 5});
    b->d_io_bytes = io * sizeof(double);
    chk(dalloc(o, &b->d_io, io));
    if (!e) {
        b->pin_bytes = b->d_io_bytes + (size_t)W * 8 + 64;
        e = cudaMallocHost(&b->pin, b->pin_bytes);
    }
    if (!e) e = cudaMemsetAsync(d.status, 0, sizeof(int), c->stream);
    if (!e) e = cudaMemsetAsync(d.pend_k, 0xff, W * sizeof(int), c->stream);
    if (!e) e = cudaMemsetAsync(d.acc_count, 0, W * sizeof(int), c->stream);
    if (!e) e = cudaMemsetAsync(d.resum_flag, 0, W, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) {
        int code = (e == cudaErrorMemoryAllocation) ? EWALD_ERR_OOM : EWALD_ERR_CUDA;
        ewald_batch_destroy(b);
        cudaGetLastError();
        return fail(c, code, cudaGetErrorString(e));
    }
    c->n_batches += 1;
    b->counted = true;
    *out = b;
    return EWALD_OK;
}

void ewald_batch_destroy(ewald_batch *b) {
    if (!b) return;
    ewald_ctx *c = b->ctx;
    const bool counted = b->counted;
    if (c && c->stream) cudaStreamSynchronize(c->stream);
    free_all(b->dev);
    if (b->pin) cudaFreeHost(b->pin);
    delete b;
    if (counted) {
        c->n_batches -= 1;
        if (c->n_batches == 0 && c->destroy_pending) destroy_now(c);
    }
}

int ewald_batch_set_positions(ewald_batch *b, const double *pos, int on_device) {
    EWALD_NVTX("ewald_batch_set_positions");
    if (!b || !pos) return fail(b ? b->ctx : nullptr, EWALD_ERR_ARG);
    ewald_ctx *c = b->ctx;
    const double *src = pos;
    int err = EWALD_OK;
    if (!on_device) {
        src = (const double *)copy_in(b, pos, (size_t)b->b.W * c->s.n_mob * c->s.dim * sizeof(double),
                                      b->d_io, &err);
        if (err) return err;
    }
    int e = timed(c, KT_INGEST, [&] { return launch_ingest(c->s, b->b, src, c->stream); });
    if (e) return cuda_fail(c, (cudaError_t)e);
    b->has_pos = true;
    b->has_pending = false;
    b->rho_stale = true;  // rho(G) follows the new positions at its next use
    if (!on_device) return sync_status(b);
    return EWALD_OK;
}

int ewald_batch_get_positions(ewald_batch *b, double *pos, int on_device) {
    EWALD_NVTX("ewald_batch_get_positions");
    if (!ready(b) || !pos) return fail(b ? b->ctx : nullptr, EWALD_ERR_ARG);
    ewald_ctx *c = b->ctx;
    size_t n = (size_t)b->b.W * c->s.n_mob * c->s.dim * sizeof(double);
    double *dst = on_device ? pos : b->d_io;
    int e = launch_positions_out(c->s, b->b, dst, c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e);
    if (on_device) return EWALD_OK;
    return copy_out(b, pos, b->d_io, n, 0);
}

int ewald_batch_sync(ewald_batch *b) {
    if (!b) return EWALD_ERR_ARG;
    return sync_status(b);
}

int ewald_energy(ewald_batch *b, double *e_out, int on_device) {
    EWALD_NVTX("ewald_energy");
    if (!ready(b) || !e_out) return fail(b ? b->ctx : nullptr, EWALD_ERR_ARG);
    int e = run_energy(b);
    if (e) return e;
    b->has_pending = false;
    return copy_out(b, e_out, b->b.e, (size_t)b->b.W * sizeof(double), on_device);
}

int ewald_energy_components(ewald_batch *b, double *comp_out, int on_device) {
    EWALD_NVTX("ewald_energy_components");
    if (!ready(b) || !comp_out) return fail(b ? b->ctx : nullptr, EWALD_ERR_ARG);
    int e = run_energy(b);
    if (e) return e;
    b->has_pending = false;
    return copy_out(b, comp_out, b->b.comp, (size_t)b->b.W * 5 * sizeof(double), on_device);
}

int ewald_propose_move(ewald_batch *b, const int *k, const double *r_new, double *de_out, int on_device) {
    EWALD_NVTX("ewald_propose_move");
    if (!ready(b) || !k || !r_new || !de_out) return fail(b ? b->ctx : nullptr, EWALD_ERR_ARG);
    ewald_ctx *c = b->ctx;
    const int W = b->b.W, dim = c->s.dim;
    const int *dk = k;
    const double *dr = r_new;
    if (!on_device) {
        for (int w = 0; w < W; ++w) {
            if (k[w] < 0 || k[w] >= c->s.n_mob) return fail(c, EWALD_ERR_ARG, "move index out of range");
            for (int x = 0; x < dim; ++x)
                if (!std::isfinite(r_new[(size_t)w * dim + x])) return fail(c, EWALD_ERR_ARG, "non-finite position");
        }
        // k and r_new share the pinned buffer: stage both, then one sync
        char *pin = (char *)b->pin + 16;
        size_t nk = (size_t)W * sizeof(int), nr = (size_t)W * dim * sizeof(double);
        std::memcpy(pin, k, nk);
        std::memcpy(pin + align16(nk), r_new, nr);
        cudaError_t e = cudaMemcpyAsync(b->d_k, pin, nk, cudaMemcpyHostToDevice, c->stream);
        if (!e) e = cudaMemcpyAsync(b->d_rnew, pin + align16(nk), nr, cudaMemcpyHostToDevice, c->stream);
        if (e) return cuda_fail(c, e);
        dk = b->d_k;
        dr = b->d_rnew;
    }
    double *dde = on_device ? de_out : b->d_de;
    if (int r = ensure_rho(b)) return r;
    int e = timed(c, KT_PROPOSE, [&] {
        if (c->t.tiered) return launch_propose_tiered(c->s, b->b, dk, dr, dde, c->stream);
        return launch_propose(c->s, b->b, c->t.precision, c->cfg, dk, dr, dde, c->stream);
    });
    if (e) return cuda_fail(c, (cudaError_t)e);
    b->has_pending = true;
    if (on_device) return EWALD_OK;
    return copy_out(b, de_out, b->d_de, (size_t)W * sizeof(double), 0);
}

int ewald_accept_move(ewald_batch *b, const unsigned char *accept, int on_device) {
    EWALD_NVTX("ewald_accept_move");
    if (!ready(b) || !accept) return fail(b ? b->ctx : nullptr, EWALD_ERR_ARG);
    ewald_ctx *c = b->ctx;
    if (!b->has_pending) return fail(c, EWALD_ERR_NO_PROPOSAL, "no pending proposal");
    const unsigned char *da = accept;
    if (!on_device) {
        int err;
        da = (const unsigned char *)copy_in(b, accept, b->b.W, b->d_acc, &err);
        if (err) return err;
    }
    const int p = c->t.precision;
    int e = timed(c, KT_ACCEPT, [&] { return launch_accept(c->s, b->b, p, c->cfg, da, c->t.resum_every, c->stream); });
    // rebuild rho(G) of the walkers that reached resum_every accepted moves
    // (the mixed accept lists them; the other forms flag them)
    if (!e) e = timed(c, KT_RESUM, [&] {
        return p == EWALD_MIXED ? launch_sfac_listed(c->s, b->b, p, c->cfg, c->stream)
                                : run_sfac(c, b->b, p, b->b.resum_flag);
    });
    if (e) return cuda_fail(c, (cudaError_t)e);
    b->has_pending = false;
    if (!on_device) return sync_status(b);
    return EWALD_OK;
}

int ewald_resum(ewald_batch *b) {
    EWALD_NVTX("ewald_resum");
    if (!ready(b)) return fail(b ? b->ctx : nullptr, EWALD_ERR_ARG);
    b->rho_stale = true;
    return ensure_rho(b);
}

int ewald_batch_get_rho(ewald_batch *b, double *rho_out, int on_device) {
    EWALD_NVTX("ewald_batch_get_rho");
    if (!ready(b) || !rho_out) return fail(b ? b->ctx : nullptr, EWALD_ERR_ARG);
    ewald_ctx *c = b->ctx;
    if (int r = ensure_rho(b)) return r;
    double *dst = on_device ? rho_out : b->d_io;
    int e = launch_rho_out(c->s, b->b, c->t.precision, c->d_g2slot, dst, c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e);
    if (on_device) return EWALD_OK;
    return copy_out(b, rho_out, b->d_io, (size_t)b->b.W * c->s.n_layers * c->s.n_gh * 2 * sizeof(double), 0);
}

int ewald_set_timing(ewald_ctx *c, int enable) {
    if (!c) return EWALD_ERR_ARG;
    if (c->timing && !enable) collect_timers(c);
    c->timing = enable != 0;
    return EWALD_OK;
}

int ewald_get_timing(ewald_ctx *c, double *ms, long long *launches) {
    if (!c) return EWALD_ERR_ARG;
    cudaError_t e = (cudaError_t)collect_timers(c);
    for (int k = 0; k < KT_COUNT; ++k) {
        if (ms) ms[k] = c->t_ms[k];
        if (launches) launches[k] = c->t_n[k];
        c->t_ms[k] = 0;
        c->t_n[k] = 0;
    }
    return e ? cuda_fail(c, e) : EWALD_OK;
}

// ------------------------------------------------------------------ multi

struct ewald_multi {
    ewald::MultiFn fn = nullptr;  // the energy kernel for these systems
    std::vector<ewald_batch *> batches;
    std::vector<ewald_ctx *> ctxs;        // distinct contexts, in first-use order
    int precision = 0;
    cudaStream_t stream = nullptr;
    std::vector<void *> dev;
    MultiDev m{};
    size_t smem = 0;
    int grid = 0;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev_out = nullptr;
    std::vector<cudaEvent_t> ev_in;
    double *pin = nullptr;
};

namespace {

// Estimated cost of an item, for longest-first ordering (relative units:
// one electron-G term = 1; a pair costs its candidate tests and its terms).
double item_cost(const SysDev &s, int kind, int sub) {
    if (kind == kItemSfac) {
        int runs = std::min(s.sfac_threads, s.n_runs - sub * s.sfac_threads);  // run lengths vary; bound
        return (double)runs * s.run_len * s.n_mob;
    }
    return 1.0;  // scaled by the caller
}

}  // namespace

int ewald_multi_create(ewald_batch *const *batches, int n, ewald_multi **out) {
    EWALD_NVTX("ewald_multi_create");
    if (!out) return EWALD_ERR_ARG;
    *out = nullptr;
    if (!batches || n < 1) return EWALD_ERR_ARG;
    ewald_multi *m = new (std::nothrow) ewald_multi();
    if (!m) return EWALD_ERR_OOM;
    std::vector<SysDev> sys;
    std::vector<BatchDev> bat;
    std::vector<int> bat_sys, wbase;
    int nw = 0;
    for (int i = 0; i < n; ++i) {
        ewald_batch *b = batches[i];
        if (!b || !b->ctx || !b->has_pos) {
            delete m;
            return EWALD_ERR_ARG;
        }
        if (i == 0) m->precision = b->ctx->t.precision;
        if (b->ctx->t.precision != m->precision) {
            delete m;
            return EWALD_ERR_ARG;
        }
        int si = -1;
        for (size_t k = 0; k < m->ctxs.size(); ++k)
            if (m->ctxs[k] == b->ctx) si = (int)k;
        if (si < 0) {
            si = (int)m->ctxs.size();
            m->ctxs.push_back(b->ctx);
            SysDev sd = b->ctx->s;
            // the FP32 launch has CTAs of kMultiThreads32 threads: its
            // structure-factor items take as many G runs as fit (chunks of
            // the context merged), so that no thread of the CTA idles
            if (m->precision != EWALD_FP64)
                while (sd.n_gchunks > 1 && 2 * sd.sfac_threads <= kMultiThreads32) {
                    sd.sfac_threads *= 2;
                    sd.n_gchunks = (sd.n_runs + sd.sfac_threads - 1) / sd.sfac_threads;
                }
            sys.push_back(sd);
        }
        m->batches.push_back(b);
        bat.push_back(b->b);
        bat_sys.push_back(si);
        wbase.push_back(nw);
        nw += b->b.W;
    }
    // work items, longest first
    struct It { double cost; int4 d; };
    std::vector<It> items;
    for (int i = 0; i < n; ++i) {
        const SysDev &s = sys[bat_sys[i]];
        const double ipp = s.dim == 3 ? 4.18879 * std::pow(std::sqrt(s.rc2), 3) : 3.14159 * s.rc2;
        const double vol = m->ctxs[bat_sys[i]]->t.volume;
        const double pair_cost = 3.0 * s.cand_max + 6.0 * ipp / vol;
        const std::vector<int> &rt = m->ctxs[bat_sys[i]]->t.runs;
        (void)rt;
        for (int w = 0; w < bat[i].W; ++w) {
            for (int c = 0; c < s.n_gchunks; ++c)
                items.push_back({item_cost(s, kItemSfac, c), make_int4(kItemSfac, i, w, c)});
            for (int p = 0; p < s.n_items; ++p) {
                // pairs of the tile pair (ragged tails and diagonal triangles)
                const HostTables &t = m->ctxs[bat_sys[i]]->t;
                int ti = p, tj = 0;
                (void)ti; (void)tj;
                double pairs = (double)s.tile * s.tile;
                int nt = s.n_mob_tiles;
                // recover (ti, tj) from the item order used by build_device
                int q = p, a = 0;
                int nft = (t.n_fix + s.tile - 1) / s.tile;
                while (q >= (nt - a) + nft) { q -= (nt - a) + nft; ++a; }
                int ni = std::min(s.tile, t.n_mob - a * s.tile);
                if (q < nt - a) {
                    int b2 = a + q;
                    int nj = std::min(s.tile, t.n_mob - b2 * s.tile);
                    pairs = b2 == a ? 0.5 * ni * (ni - 1) : (double)ni * nj;
                } else {
                    int f = q - (nt - a);
                    pairs = (double)ni * std::min(s.tile, t.n_fix - f * s.tile);
                }
                items.push_back({pairs * pair_cost, make_int4(kItemReal, i, w, p)});
            }
        }
    }
    // grouped by batch (a CTA then re-stages a system's tables about once per
    // batch), the batch with the longest items first, longest first within one
    std::vector<double> top(n, 0.0);
    for (const It &x : items) top[x.d.y] = std::max(top[x.d.y], x.cost);
    std::stable_sort(items.begin(), items.end(), [&](const It &x, const It &y) {
        if (x.d.y != y.d.y) return top[x.d.y] != top[y.d.y] ? top[x.d.y] > top[y.d.y] : x.d.y < y.d.y;
        return x.cost > y.cost;
    });
    std::vector<int4> id(items.size());
    for (size_t k = 0; k < items.size(); ++k) id[k] = items[k].d;

    cudaError_t e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
    std::vector<void *> &o = m->dev;
    const char *step = "stream";
    auto chk = [&](cudaError_t x, const char *what = "") {
        if (!e && x) {
            e = x;
            step = what;
        }
    };
    SysDev *d_sys = nullptr;
    BatchDev *d_bat = nullptr;
    int *d_bs = nullptr, *d_wb = nullptr;
    int4 *d_items = nullptr;
    if (!e) chk(upload(o, &d_sys, sys.data(), sys.size()), "upload systems");
    if (!e) chk(upload(o, &d_bat, bat.data(), bat.size()), "upload batches");
    if (!e) chk(upload(o, &d_bs, bat_sys.data(), bat_sys.size()), "upload map");
    if (!e) chk(upload(o, &d_wb, wbase.data(), wbase.size()), "upload bases");
    if (!e) chk(upload(o, &d_items, id.data(), id.size()), "upload items");
    MultiDev &md = m->m;
    if (!e) chk(dalloc(o, &md.next, 1), "alloc");
    if (!e) chk(dalloc(o, &md.done, nw), "alloc");
    if (!e) chk(dalloc(o, &md.e_all, nw), "alloc");
    if (!e) chk(cudaMallocHost((void **)&m->pin, sizeof(double) * nw), "pinned");
    md.sys = d_sys;
    md.bat = d_bat;
    md.bat_sys = d_bs;
    md.wbase = d_wb;
    md.items = d_items;
    md.n_items = (int)id.size();
    md.n_walkers = nw;
    m->smem = multi_energy_smem(sys, m->precision, &md.img_bytes);
    m->fn = multi_kernel(m->precision, sys);
    if (!e) chk((cudaError_t)configure_multi(m->fn, m->precision, m->smem, &m->grid), "configure");
    if (!e) chk(cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming), "event");
    for (size_t k = 0; k < m->ctxs.size() && !e; ++k) {
        cudaEvent_t ev;
        chk(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        if (!e) m->ev_in.push_back(ev);
    }
    // capture the launch (counter resets + kernel) once; every call replays it
    if (!e) {
        cudaGraph_t g = nullptr;
        chk(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        if (!e) {
            int le = launch_multi_energy(m->fn, md, m->precision, m->grid, m->smem, m->stream);
            cudaError_t ce = cudaStreamEndCapture(m->stream, &g);
            chk((cudaError_t)le, "launch in capture");
            chk(ce, "end capture");
        }
        if (!e) chk(cudaGraphInstantiate(&m->exec, g, 0), "instantiate");
        if (g) cudaGraphDestroy(g);
    }
    if (e) {
        ewald_ctx *c0 = m->ctxs.empty() ? nullptr : m->ctxs[0];
        if (c0)
            c0->why = std::string("multi create, ") + step + ": " + cudaGetErrorName(e) + " (dynamic smem " +
                      std::to_string(m->smem) + " B, grid " + std::to_string(m->grid) + ")";
        ewald_multi_destroy(m);
        cudaGetLastError();
        return fail(c0, e == cudaErrorMemoryAllocation ? EWALD_ERR_OOM : EWALD_ERR_CUDA);
    }
    *out = m;
    return EWALD_OK;
}

void ewald_multi_destroy(ewald_multi *m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->exec) cudaGraphExecDestroy(m->exec);
    for (cudaEvent_t ev : m->ev_in) cudaEventDestroy(ev);
    if (m->ev_out) cudaEventDestroy(m->ev_out);
    free_all(m->dev);
    if (m->pin) cudaFreeHost(m->pin);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

int ewald_multi_energy(ewald_multi *m, double *e_out, int on_device) {
    EWALD_NVTX("ewald_multi_energy");
    if (!m || !e_out) return EWALD_ERR_ARG;
    cudaError_t e = cudaSuccess;
    // the batches' own streams first finish what they have queued
    for (size_t k = 0; k < m->ctxs.size() && !e; ++k) {
        e = cudaEventRecord(m->ev_in[k], m->ctxs[k]->stream);
        if (!e) e = cudaStreamWaitEvent(m->stream, m->ev_in[k], 0);
    }
    if (!e) e = cudaGraphLaunch(m->exec, m->stream);
    const size_t bytes = sizeof(double) * (size_t)m->m.n_walkers;
    if (!e) e = cudaMemcpyAsync(on_device ? (void *)e_out : (void *)m->pin, m->m.e_all, bytes,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream);
    if (!e) e = cudaEventRecord(m->ev_out, m->stream);
    for (size_t k = 0; k < m->ctxs.size() && !e; ++k) e = cudaStreamWaitEvent(m->ctxs[k]->stream, m->ev_out, 0);
    for (ewald_batch *b : m->batches) {
        b->has_pending = false;
        b->rho_stale = false;  // the launch rebuilt every batch's rho(G)
    }
    if (e) return cuda_fail(m->ctxs[0], e);
    if (on_device) return EWALD_OK;
    if ((e = cudaStreamSynchronize(m->stream))) return cuda_fail(m->ctxs[0], e);
    std::memcpy(e_out, m->pin, bytes);
    int st = EWALD_OK;
    for (ewald_batch *b : m->batches) {
        int s2 = sync_status(b);
        if (s2 && !st) st = s2;
    }
    return st;
}

int ewald_autotune(ewald_batch *b, const char *cache_path, ewald_tune_result *res) {
    EWALD_NVTX("ewald_autotune");
    if (!b || !b->ctx) return EWALD_ERR_ARG;
    if (!b->has_pos) return fail(b->ctx, EWALD_ERR_STATE, "positions not set");
    ewald_ctx *c = b->ctx;
    const std::string key = tune_key(c);
    std::map<std::string, TuneEntry> cache;
    if (cache_path) cache = read_tune_cache(cache_path);
    ewald_tune_result r{};
    auto it = cache.find(key);
    if (it != cache.end() && tiling_allowed(c, it->second.tile / 32, it->second.bits)) {
        int st = apply_config(c, it->second.tile / 32, it->second.bits, it->second.warps, it->second.chunks);
        if (st) return st;
        r.pair_tile = it->second.tile;
        r.subcell_bits = it->second.bits;
        r.ms = it->second.ms;
        r.from_cache = 1;
        r.real_threads = c->t.precision == EWALD_MIXED && !c->t.tiered ? 32 * c->s.real_warps : kRealThreads;
        r.sfac_chunks = c->s.n_gchunks;
        if (res) *res = r;
        return EWALD_OK;
    }
    // time the kernels on up to 512 of this batch's walkers
    BatchDev view = b->b;
    view.W = std::min(view.W, 512);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto best_of_3 = [&](auto &&launch, double *t_min) -> int {
        *t_min = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, c->stream);
            int le = launch();
            cudaEventRecord(e1, c->stream);
            cudaError_t ce = cudaEventSynchronize(e1);
            if (le || ce) return le ? le : (int)ce;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) *t_min = std::min(*t_min, (double)ms);  // the first launch warms up
        }
        return 0;
    };
    auto done = [&](int st) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
    };
    const bool mixed = c->t.precision == EWALD_MIXED && !c->t.tiered;
    double best = 1e300;
    int bestS = c->s.tile / 32, bestBits = c->s.sub_bits, bestWarps = c->s.real_warps;
    const int Ss[4] = {1, 2, 4, 8};
    const int warps_opts[2] = {8, 16};
    for (int S : Ss)
        for (int bits = 0; bits <= (c->t.dim == 3 ? 4 : 6); ++bits)
            for (int wi = mixed ? 0 : 1; wi < 2; ++wi) {
                if (!tiling_allowed(c, S, bits)) continue;
                int st = apply_config(c, S, bits, warps_opts[wi], 0);
                if (st) return done(st);
                double t_min;
                int le = best_of_3([&] { return launch_real(c->s, view, c->t.precision, c->cfg, c->stream); }, &t_min);
                if (le) return done(cuda_fail(c, (cudaError_t)le));
                r.n_tried += 1;
                if (t_min < best) {
                    best = t_min;
                    bestS = S;
                    bestBits = bits;
                    bestWarps = warps_opts[wi];
                }
            }
    int st = apply_config(c, bestS, bestBits, bestWarps, 0);
    if (st) return done(st);
    // structure factor: 1 to 4 chunks of G runs per walker
    double best_sf = 1e300;
    int bestCh = c->s.n_gchunks, last_ng = -1;
    for (int ch = 1; ch <= 4; ++ch) {
        SysDev trial = c->s;
        set_sfac_chunks(trial, ch);
        if (trial.n_gchunks == last_ng || trial.n_gchunks > c->max_gchunks) continue;
        last_ng = trial.n_gchunks;
        if ((st = apply_config(c, bestS, bestBits, bestWarps, ch))) return done(st);
        double t_min;
        int le = best_of_3([&] { return run_sfac(c, view, c->t.precision, nullptr); }, &t_min);
        if (le) return done(cuda_fail(c, (cudaError_t)le));
        if (t_min < best_sf) {
            best_sf = t_min;
            bestCh = ch;
        }
    }
    if ((st = apply_config(c, bestS, bestBits, bestWarps, bestCh))) return done(st);
    r.pair_tile = 32 * bestS;
    r.subcell_bits = bestBits;
    r.ms = best;
    r.real_threads = mixed ? 32 * bestWarps : kRealThreads;
    r.sfac_chunks = c->s.n_gchunks;
    r.sfac_ms = best_sf;
    if (cache_path) {
        TuneEntry te{32 * bestS, bestBits, best};
        te.warps = mixed ? bestWarps : 0;
        te.chunks = bestCh;
        cache[key] = te;
        write_tune_cache(cache_path, cache);
    }
    if (res) *res = r;
    return done(EWALD_OK);
}

}  // extern "C"
