// Private definitions of the C ABI objects, shared by the files that
// implement entry points (capi.cu, serve.cu, noalloc.cu).
#pragma once
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "device_common.cuh"

struct ewald_ctx {
    using HostTables = ewald::HostTables;
    using SysDev = ewald::SysDev;
    using LaunchCfg = ewald::LaunchCfg;
    HostTables t;
    SysDev s{};
    LaunchCfg cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<void *> dev;
    int *d_g2slot = nullptr;
    int n_batches = 0;        // live batches; the context outlives them
    int max_items = 0;        // pair-tile items per walker at the finest tiling
    int max_gchunks = 0;      // structure-factor chunks per walker at the finest chunking
    bool destroy_pending = false;
    int last_error = EWALD_OK;
    std::string why;
    // two-body plane-wave Jastrow term (jastrow.cu): the stars' G vectors,
    // one of each +-G pair
    int jp_n_g = 0, jp_n_stars = 0;
    int4 *d_jp_nvec = nullptr;     // (n1, n2, n3, star)
    double4 *d_jp_gvec = nullptr;  // (Gx, Gy, Gz, a of its star)
    // polynomial two-body Jastrow term (jastrow_u.cu)
    bool ju_set = false;
    ewald::JuDev ju{};
    std::vector<void *> ju_dev;    // its device tables
    // kernel timers
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_open;
    double t_ms[ewald::KT_COUNT] = {};
    long long t_n[ewald::KT_COUNT] = {};
};

struct ewald_batch {
    ewald_ctx *ctx = nullptr;
    ewald::BatchDev b{};
    std::vector<void *> dev;
    bool has_pos = false, has_pending = false;
    bool rho_stale = false;  // positions changed since rho(G) was last built
    bool counted = false;  // included in ctx->n_batches
    // host-I/O staging: pinned host buffer and device scratch for host inputs
    void *pin = nullptr;
    size_t pin_bytes = 0;
    double *d_io = nullptr;   // [W][N][dim] doubles (positions, rho, components)
    size_t d_io_bytes = 0;
    int *d_k = nullptr;
    double *d_rnew = nullptr, *d_de = nullptr;
    unsigned char *d_acc = nullptr;
};

namespace ewald_capi {

// An NVTX range over an entry point (named "ewald_energy" and so on), so that
// a profiler's timeline shows each library call around the kernels it
// launched.  Without a tool attached a range costs a few instructions.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define EWALD_NVTX(name) ewald_capi::NvtxRange ewald_nvtx_range_(name)

inline int fail(ewald_ctx *c, int code, const char *why = nullptr) {
    if (c && code) {
        c->last_error = code;
        if (why) c->why = why;
    }
    return code;
}

inline int cuda_fail(ewald_ctx *c, cudaError_t e) {
    if (c) c->why = std::string("CUDA: ") + cudaGetErrorName(e) + ": " + cudaGetErrorString(e);
    return fail(c, EWALD_ERR_CUDA);
}

template <typename T>
cudaError_t dalloc(std::vector<void *> &owned, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e == cudaSuccess) owned.push_back(*p);
    return e;
}

template <typename T>
cudaError_t upload(std::vector<void *> &owned, T **p, const T *src, size_t count) {
    cudaError_t e = dalloc(owned, p, count);
    if (e) return e;
    if (count) e = cudaMemcpy(*p, src, count * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace ewald_capi
