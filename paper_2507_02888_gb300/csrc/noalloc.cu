// ewald_energy_noalloc: full energies of a batch of walkers without any
// device allocation at call time.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool that must not fragment it, or an embedded host
// that reserves all device memory up front.  This entry point takes the walkers' positions and the
// output array from the caller and keeps every intermediate (fixed-point
// coordinates, rho(G), partial sums, status word) in one file-scope
// __device__ array of fixed size, kNoAllocScratchBytes, that every GPU which
// loads the library holds until the process exits.  It reuses the kernels
// of the ordinary ewald_energy path on that scratch.
#include <mutex>
#include <string>

#include "capi_internal.h"
#include "sfac_df.h"

namespace ewald {

constexpr size_t kNoAllocScratchBytes = 32u << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array, looked up once per device (host code
// cannot use the symbol's name as an address).
static std::mutex g_scratch_mutex;
static void *g_scratch_ptr[kMaxDevices];

static int scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Carve a BatchDev of W walkers out of the scratch; returns the bytes needed.
static size_t carve(const SysDev &s, int W, unsigned char *base, BatchDev *b) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    const size_t slots = (size_t)s.n_runs * s.run_len * s.n_layers;  // rho of every layer
    b->W = W;
    b->status = (int *)take(sizeof(int));
    b->u = (unsigned long long *)take((size_t)W * s.dim * s.mob_stride * sizeof(unsigned long long));
    b->rho = (double2 *)take((size_t)W * slots * sizeof(double2));
    b->part_real = (double *)take((size_t)W * s.n_items * sizeof(double));
    b->part_recip = (double *)take((size_t)W * s.n_gchunks * sizeof(double));
    b->comp = (double *)take((size_t)W * 5 * sizeof(double));
    b->acc_count = (int *)take((size_t)W * sizeof(int));
    b->pend_k = (int *)take((size_t)W * sizeof(int));
    b->pend_u = nullptr;
    b->resum_flag = nullptr;
    b->e = nullptr;
    return off;
}

// tiered: an EWALD_FP64_TIERED context (precision EWALD_FP64), whose
// structure factor is the double-float kernel, as in ewald_energy
static int noalloc_energy(const SysDev &s, const LaunchCfg &cfg, int precision, bool tiered, const double *pos,
                          int W, double *e_out, int *status_out, cudaStream_t st) {
    BatchDev b{};
    if (carve(s, W, nullptr, &b) > kNoAllocScratchBytes) return -1;  // too many walkers
    void *base = nullptr;
    int e = scratch_address(&base);
    if (e) return e;
    carve(s, W, (unsigned char *)base, &b);
    b.e = e_out;
    // the status word is the only scratch that must start at zero
    if ((e = cudaMemsetAsync(b.status, 0, sizeof(int), st))) return e;
    if ((e = launch_ingest(s, b, pos, st))) return e;
    if ((e = tiered ? launch_sfac_df(s, b, cfg, nullptr, st) : launch_sfac(s, b, precision, cfg, nullptr, st)))
        return e;
    if ((e = launch_real(s, b, precision, cfg, st))) return e;
    if ((e = launch_combine(s, b, st))) return e;
    if (status_out && (e = cudaMemcpyAsync(status_out, b.status, sizeof(int), cudaMemcpyDeviceToDevice, st)))
        return e;
    return cudaSuccess;
}

static size_t noalloc_walker_limit(const SysDev &s) {
    BatchDev b{};
    int lo = 0, hi = 1 << 24;
    while (lo < hi) {  // largest W whose carve fits
        int mid = lo + (hi - lo + 1) / 2;
        if (carve(s, mid, nullptr, &b) <= kNoAllocScratchBytes) lo = mid;
        else hi = mid - 1;
    }
    return (size_t)lo;
}

}  // namespace ewald

extern "C" int ewald_energy_noalloc(ewald_ctx *c, const double *pos, int n_walkers, double *e_out,
                                    int *status_out) {
    EWALD_NVTX("ewald_energy_noalloc");
    using namespace ewald_capi;
    if (!c) return EWALD_ERR_ARG;
    if (!pos || !e_out || n_walkers < 1)
        return fail(c, EWALD_ERR_ARG, "need device positions, output and n_walkers >= 1");
    const size_t limit = ewald::noalloc_walker_limit(c->s);
    if ((size_t)n_walkers > limit) {
        c->why = "n_walkers " + std::to_string(n_walkers) + " exceeds the static scratch: at most " +
                 std::to_string(limit) + " walkers of this system";
        return fail(c, EWALD_ERR_OOM);
    }
    int e = ewald::noalloc_energy(c->s, c->cfg, c->t.precision, c->t.tiered, pos, n_walkers, e_out, status_out, c->stream);
    return e ? cuda_fail(c, (cudaError_t)e) : EWALD_OK;
}
