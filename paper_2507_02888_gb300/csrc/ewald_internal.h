// Internal declarations of the GB300 Ewald library (not part of the ABI).
//
// Data layout in device memory (per context = one periodic system):
//   images   : candidate lattice vectors R (Cartesian), FP64 and FP32 copies
//   cand     : per displacement cell, indices into images (uint16), padded
//   runs     : G rows split into runs of <= run_len consecutive n1 walked away
//              from the row's smallest |G| (int4: n1 start, n2, n3, dir * len)
//   gw       : weight of every G slot, 2 C f(G) (0 for padding slots)
//   rho_fix  : fixed particles' rho(G) per layer and slot
//   gwl      : layered 2D only: weight of Re(rho_L conj(rho_L')) per layer
//              pair and slot, (pi/A) F(G, z_L - z_L') (paper Eq. (5) at z != 0)
// and per walker batch:
//   u        : [W][dim][stride] fixed-point fractional coordinates (uint64,
//              2^64 = one lattice period); FP32 loops use the top 32 bits
//   rho      : [W][n_layers][run_len * n_runs] rho(G) (double2);
//              slot = r * n_runs + run
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ewald.h"

namespace ewald {

constexpr int kRealWarps = 4;          // warps per real-space CTA
constexpr int kRealThreads = 32 * kRealWarps;
// resident real-space CTAs per SM the registers are sized for (FP32, FP64 path)
constexpr int kRealMinBlocks32 = 11, kRealMinBlocks64 = 8;
// the mixed path's real-space kernel: warps per CTA (sharing one copy of the
// candidate tables) and resident CTAs per SM its registers are sized for
constexpr int kRealMixedWarps = 16, kRealMixedThreads = 32 * kRealMixedWarps, kRealMinBlocksMixed = 2;
// largest shared-memory footprint of the mixed loop's candidate tables
// chosen by default or by the autotuner
constexpr size_t kMixedTableBytes = 24 * 1024;
// per-warp queues of accepted (r^2, weight) terms: the FP32 one a ring
// flushed 64 entries at a time, the FP64 one flushed 32 at a time
constexpr int kQueueCap32 = 128, kQueueCap64 = 96;
template <typename R>
constexpr int kQueueCapOf = sizeof(R) == 4 ? kQueueCap32 : kQueueCap64;
constexpr int kSfacThreads = 256;      // threads (= runs) per structure-factor CTA, at most
// resident structure-factor CTAs per SM the registers are sized for (FP32, FP64 path)
constexpr int kSfacMinBlocks32 = 3, kSfacMinBlocks64 = 2;
constexpr int kMoveThreads = 256;      // threads per walker in propose / accept
constexpr int kRunLen = 8;             // maximum G run length (compile-time)
// default real-space cutoff of the mixed path: erfc(alpha r_c) = kMixedRealTol
// (the FP64 path and every G cutoff use 1e-16)
constexpr double kMixedRealTol = 1e-10;
// tiered FP64 path: pair images with erfc(alpha r) above kTierErfc are
// evaluated in FP64, the rest in FP32
constexpr double kTierErfc = 1e-7;
constexpr int kHeadCap = 64;           // per-warp queue of FP64 (head) terms of the tiered path
constexpr int kRealUnits = 16;         // work units (sub-tiles x j slices) of one pair item, at most

// FP64 image vector (x, y, z, unused), 32-byte aligned for two 16-byte loads.
struct __align__(32) Img64 {
    double x, y, z, w;
};

// Device-side error bits, OR-ed into the batch status word by kernels.
enum : int { ST_COINCIDENT = 1, ST_BAD_INDEX = 2, ST_NONFINITE = 4, ST_TIMEOUT = 8, ST_DEBUG_RANGE = 16 };

// Index checks of the debug build (compiled with -DEWALD_DEBUG): where
// EWALD_IN_RANGE(cond, status) is false the kernel ORs ST_DEBUG_RANGE into
// the status word, records the check's source line in bits 8-23 (the first
// miss that gets there), and skips the access (the call then reports
// EWALD_ERR_STATE with that line); in the ordinary build the check compiles
// to nothing.
#ifdef EWALD_DEBUG
#ifdef __CUDACC__
__device__ inline bool ewald_debug_miss(int *status, int line) {
    const int old = atomicOr(status, ST_DEBUG_RANGE) | ST_DEBUG_RANGE;
    if (!(old >> 8)) atomicCAS(status, old, old | ((line & 0xffff) << 8));  // one try: a clash keeps the first
    return false;
}
#endif
#define EWALD_IN_RANGE(cond, status) ((cond) ? true : ewald_debug_miss((status), __LINE__))
#else
#define EWALD_IN_RANGE(cond, status) ((void)sizeof(cond), true)
#endif

// Per-system constants and table pointers; passed by value to kernels.
struct SysDev {
    int dim, n_mob, n_fix, mob_stride, fix_stride;
    double A64[3][3];   // A[k][x] * 2^-64: Cartesian x of a uint64 fractional difference
    float A32[3][3];    // A[k][x] * 2^-32 for the FP32 path (rounded) ...
    float A32lo[3][3];  // ... and its rounding residual: A * 2^-32 = A32 + A32lo
    double A[3][3];     // lattice rows a_k
    double Binv[3][3];  // f_k = sum_x Binv[k][x] r_x (fractional coordinates)
    double alpha, rc2, coin2;
    float alpha_f, rc2_f, coin2_f;
    float alpha_lo_f, alpha2_f, alpha2_lo_f;  // alpha = alpha_f + alpha_lo_f, alpha^2 likewise
    float close2_f;  // FP32 path: pairs closer than this (squared) get their R = 0 term in FP64
    float tier2_f;   // tiered FP64 path (> 0): images with r^2 below this are evaluated in FP64
    // real space
    int n_img, sub_bits, cand_max;  // images [n_img + 1]: the last is a far sentinel
    const Img64 *img_d;
    const float4 *img_f;
    const float4 *img_lo_f;  // img_d - img_f: the rounding of the FP32 images (tiered path)
    const unsigned short *cand;
    // the same lists for the mixed path's pair loop: each distinct list once,
    // as cand_pairs pairs of FP32 images (X_a, X_b, Y_a, Y_b) and (Z_a, Z_b),
    // padded with the sentinel; clist[cell] = the cell's list.  With
    // mixed_direct the second nearest image to the cell's centre comes second.
    const float4 *cxy;
    const float2 *cz;
    const unsigned short *clist;
    int n_lists, cand_pairs;
    int cand_pstride;  // pairs from one list to the next: odd, so that lanes reading pair p of
                       // different lists fall in different banks of shared memory
    int mixed_direct;  // the energy kernels' pair loop evaluates each pair's first two images
                       // (the two nearest to the cell's centre) without the lane rings
    // the move kernel's copy of these tables, lists in the order of cand (the
    // same arrays unless mixed_direct reorders the energy kernels' lists)
    const float4 *cxy_mv;
    const float2 *cz_mv;
    const unsigned short *clist_mv;
    int n_lists_mv;
    int q_uniform;  // every mobile charge equal and every fixed charge equal
    int tile, n_mob_tiles, n_items;  // pair tiles (T = tile) and items per walker
    int real_warps;                  // mixed form: warps per real-space CTA (8 or 16)
    const int2 *items;               // (ti, tj); tj >= n_mob_tiles -> fixed tile tj - n_mob_tiles
    // reciprocal space
    int n_runs, run_len, n_gh, n_gchunks, sfac_te;
    int sfac_threads;  // runs per structure-factor chunk (multiple of 32, <= kSfacThreads)
    int n1max, n2max, n3max;
    const int4 *runs;  // (n1 start, n2, n3, dir * length), dir = +-1
    const double *gw_d;
    const float *gw_f;
    const double2 *rho_fix;  // may be null
    // charges and fixed particles
    const double *q_mob, *q_fix;
    const float *q_mob_f, *q_fix_f;
    const float2 *q_mob_df, *q_fix_df;  // charges as float pairs hi + lo (tiered path)
    const unsigned long long *fix_u;  // [dim][fix_stride]
    // constants (FP64)
    double e_madR, e_self, e_bg, e_II;
    // layered 2D (n_layers > 1): heights, per-layer particle lists, weights
    int n_layers;                          // 1: one plane (or 3D); the fields below are unused
    int lay_start[EWALD_MAX_LAYERS + 1];   // mobile particles of layer L: lay_idx[lay_start[L] ..]
    const int *lay_idx;                    // mobile particle indices grouped by layer
    const unsigned char *mob_layer;        // [n_mob] layer of each mobile particle
    const double *z_mob, *z_fix;           // heights
    const float *z_mob_f, *z_fix_f;
    const double *gwl_d;                   // [n_layers][n_layers][slots]
    const float *gwl_f;
};

// Per-batch device state.
struct BatchDev {
    int W;
    unsigned long long *u;       // [W][dim][mob_stride]
    double2 *rho;                // [W][slots]
    int *pend_k;                 // [W], -1 = nothing pending
    unsigned long long *pend_u;  // [W][3]
    int *acc_count;              // [W]
    unsigned char *resum_flag;   // [W]
    int *resum_list;             // [1 + W]: count, then the walkers to re-sum (mixed accept; may be null)
    double *part_real;           // [W][n_items]
    double *part_recip;          // [W][n_gchunks]
    double *e;                   // [W]
    double *comp;                // [W][5]
    int *status;                 // [1]
};

// Host-side tables built in FP64 by setup.cpp.
struct HostTables {
    int dim = 0, n_mob = 0, n_fix = 0, precision = 0, resum_every = 64;
    bool tiered = false;  // EWALD_FP64_TIERED: precision is EWALD_FP64, real space tiered
    double A[3][3] = {}, Ainv[3][3] = {}, B[3][3] = {};  // B rows = b_k, a_i.b_j = 2 pi d_ij
    double volume = 0, alpha = 0, r_c = 0, g_c = 0;
    std::vector<double> q_mob, q_fix, fix_pos;
    // real space
    std::vector<double> img;   // [n_img][3]
    int sub_bits = 0, cand_max = 0;
    int min_bits = 0;      // coarsest displacement cells for which candidate 0 covers r_close
    double r_close = 0;    // FP32 path: pairs closer than this (any image) go to FP64
    std::vector<unsigned short> cand;  // [n_sub][cand_max]
    std::vector<int> cand_len;         // [n_sub]
    // reciprocal space
    std::vector<int> gn;       // [n_gh][3] integer coordinates, storage order
    std::vector<int> runs;     // [n_runs][4]
    int run_len = kRunLen;
    std::vector<double> gw;    // [run_len * n_runs]
    std::vector<int> g2slot;   // [n_gh]
    std::vector<double> rho_fix;  // [n_layers][slots][2]
    // layered 2D
    int n_layers = 1;
    std::vector<double> z_mob, z_fix, layer_z;  // heights; layer_z ascending
    std::vector<int> mob_layer, fix_layer, lay_idx, lay_start;
    std::vector<double> gwl;      // [n_layers][n_layers][slots]
    int n1max = 0, n2max = 0, n3max = 0;
    // constants
    double e_madR = 0, e_self = 0, e_bg = 0, e_II = 0;
};

// setup.cpp
int build_tables(const ewald_desc *d, HostTables *t, std::string *why);
int pick_subcells(HostTables *t, int max_bytes);
int set_subcells(HostTables *t, int bits);
double shortest_lattice_vector(const HostTables &t);
int short_range_lists(const HostTables &t, double cutoff, int max_bits, std::vector<double> *img,
                      std::vector<unsigned short> *cand, int *bits_out);
size_t subcell_bytes(const HostTables &t, int bits);
// The mixed form's candidate lists (mixed_cand_order) and whether its energy
// loop evaluates their first two images directly (mixed_direct_pays).
bool mixed_direct_pays(const HostTables &t);
std::vector<unsigned short> mixed_cand_order(const HostTables &t, bool direct);

// kernels.cu launchers (return cudaError_t as int)
struct LaunchCfg {
    int sm_count;
    int real_grid;      // persistent grid of the real-space kernel
    size_t real_smem, sfac_smem, move_smem;
    int sfac_te;        // electrons per structure-factor tile
    int sfac_grid;      // persistent grid of the listed (re-sum) structure factor
    int propose_grid;   // persistent grid of the mixed-precision propose kernel
};
int configure_launch(SysDev &s, int precision, LaunchCfg *cfg);
int launch_ingest(const SysDev &s, const BatchDev &b, const double *pos, cudaStream_t st);
int launch_positions_out(const SysDev &s, const BatchDev &b, double *pos, cudaStream_t st);
int launch_real(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg,
                cudaStream_t st);
int launch_combine(const SysDev &s, const BatchDev &b, cudaStream_t st);
int launch_sfac(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg,
                const unsigned char *only, cudaStream_t st);
int launch_propose(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg,
                   const int *k, const double *r_new, double *de, cudaStream_t st);
int launch_accept(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg,
                  const unsigned char *acc, int resum_every, cudaStream_t st);
// move_mixed.cu: the mixed-precision propose kernel (persistent CTAs)
int configure_propose_mixed(const SysDev &s, int sm_count, int *grid);
int launch_propose_mixed(const SysDev &s, const BatchDev &b, int grid, const int *k, const double *r_new, double *de,
                         cudaStream_t st);
// rho(G) of the walkers in b.resum_list (after a mixed-precision accept)
int launch_sfac_listed(const SysDev &s, const BatchDev &b, int precision, const LaunchCfg &cfg, cudaStream_t st);

// Polynomial two-body Jastrow term u (jastrow_u.cu): device tables.
struct JuDev {
    int n_up, C, n_u, sub_bits, cand_max, n_img;
    double L, L2;
    float L_f, L2_f;
    const double *coef_d;  // [2][n_u + 1]: unlike, like spins (alpha_1 from the cusp)
    const float *coef_f;
    const Img64 *img_d;    // [n_img + 1], the last a far sentinel
    const float4 *img_f;
    const unsigned short *cand;  // [2^(sub_bits dim)][cand_max]
};

// Kernel ids of the per-context timers (ewald_get_timing).
enum { KT_INGEST = 0, KT_SFAC, KT_REAL, KT_COMBINE, KT_PROPOSE, KT_ACCEPT, KT_RESUM, KT_COUNT };
int launch_rho_out(const SysDev &s, const BatchDev &b, int precision, const int *g2slot, double *out,
                   cudaStream_t st);

}  // namespace ewald
