// Serving loop (continuous batching) of walker batches from concurrent runs.
//
// Requests - W walkers of some system (context) that must each make n_steps
// single-particle moves - are queued on submission and admitted between
// steps while walker slots and the device-memory budget allow.  Admission
// uploads the walkers, builds their rho(G) and initial energies; from then
// on rho(G) stays on the device.  Every step advances every active request
// by one move in one launch of k_serve_step, replayed from a CUDA graph (the
// work list and the per-request step counters live in device memory, so the
// graph never changes while the set of systems does not).  Finished
// requests are retired between steps: their energies and acceptance counts
// are copied out and their memory is returned, all stream-ordered, so the
// device never waits for the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "capi_internal.h"
#include "serve.h"
#include "sfac_df.h"

using namespace ewald;
using namespace ewald_capi;

namespace {

constexpr int kMaxSystems = 64;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
    int id = 0;
    ewald_ctx *ctx = nullptr;
    // state: 0 queued, 1 active, 2 draining, 3 done, 4 cancelled
    int W = 0, n_steps = 0, sys = -1, slot = -1, steps_done = 0, state = 0;
    bool cancel = false;  // active, cancelled by the host: retire at the next step without results
    int acc_base = 0;
    unsigned long long seed = 0;
    double sigma = 0, accept_p = 0;
    std::vector<double> pos;
    BatchDev b{};
    std::vector<void *> dev;
    size_t bytes = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    cudaEvent_t ev_done = nullptr;
    double *pin_e = nullptr;
    int *pin_acc = nullptr;
};

}  // namespace

struct ewald_server {
    int precision = 0;
    int max_walkers = 0;
    size_t budget = 0, used_bytes = 0;
    int used_walkers = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<ewald_ctx *> systems;
    std::vector<SysDev> sys_host;
    std::map<int, Req> reqs;
    std::deque<int> queue;
    std::vector<int> draining;   // retired requests whose results are on their way to the host
    std::vector<int> completed;  // finished since the last ewald_server_completed
    std::vector<int> slot_req;  // slot -> request id or -1
    std::vector<std::pair<int, int>> acc_free;  // free ranges [base, base + len) of the n_acc array
    int next_id = 1;
    // device tables
    SysDev *d_sys = nullptr;
    SlotDev *d_slots = nullptr;
    int2 *d_items = nullptr;
    int *d_n_items = nullptr, *d_next = nullptr, *d_n_acc = nullptr;
    SlotDev *pin_slots[2] = {nullptr, nullptr};
    int2 *pin_items[2] = {nullptr, nullptr};
    int *pin_n[2] = {nullptr, nullptr};
    cudaEvent_t ev_stage[2] = {nullptr, nullptr};
    int parity = 0;
    bool items_dirty = true, systems_dirty = false;
    size_t smem = 0, img_bytes = 0;
    int grid = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<void *> dev;
    std::string why;
};

namespace {

int srv_fail(ewald_server *s, int code, const std::string &why) {
    if (s) s->why = why;
    return code;
}

int srv_cuda(ewald_server *s, cudaError_t e, const char *what) {
    return srv_fail(s, EWALD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e));
}

// Device bytes a request needs (everything allocated at admission).
size_t request_bytes(const ewald_ctx *c, int W) {
    const SysDev &s = c->s;
    const size_t slots = (size_t)s.n_runs * s.run_len * s.n_layers;  // rho of every layer
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
    add((size_t)W * s.dim * s.mob_stride * 8);                  // u
    add((size_t)W * slots * 16);                                // rho
    add((size_t)W * std::max(c->max_items, s.n_items) * 8);     // part_real
    add((size_t)W * s.n_gchunks * 8);                           // part_recip
    add((size_t)W * 8 * 7);                                     // e, comp
    add((size_t)W * 4 * 2);                                     // acc_count, pend_k
    add(256);                                                   // status
    add((size_t)W * s.n_mob * s.dim * 8);                       // upload buffer (freed after admission)
    return b;
}

template <typename T>
cudaError_t aalloc(Req &r, T **p, size_t count, cudaStream_t st) {
    cudaError_t e = cudaMallocAsync((void **)p, std::max<size_t>(count, 1) * sizeof(T), st);
    if (!e) r.dev.push_back(*p);
    return e;
}

int take_acc_range(ewald_server *s, int W) {
    for (size_t i = 0; i < s->acc_free.size(); ++i)
        if (s->acc_free[i].second >= W) {
            int base = s->acc_free[i].first;
            s->acc_free[i].first += W;
            s->acc_free[i].second -= W;
            if (!s->acc_free[i].second) s->acc_free.erase(s->acc_free.begin() + i);
            return base;
        }
    return -1;
}

void give_acc_range(ewald_server *s, int base, int W) {
    s->acc_free.push_back({base, W});
    std::sort(s->acc_free.begin(), s->acc_free.end());
    std::vector<std::pair<int, int>> merged;
    for (auto &r : s->acc_free) {
        if (!merged.empty() && merged.back().first + merged.back().second == r.first) merged.back().second += r.second;
        else merged.push_back(r);
    }
    s->acc_free = merged;
}

int system_index(ewald_server *s, ewald_ctx *c) {
    for (size_t i = 0; i < s->systems.size(); ++i)
        if (s->systems[i] == c) return (int)i;
    if ((int)s->systems.size() >= kMaxSystems) return -1;
    s->systems.push_back(c);
    s->sys_host.push_back(c->s);
    s->systems_dirty = true;
    return (int)s->systems.size() - 1;
}

int capture_step(ewald_server *s) {
    if (s->exec) {
        cudaGraphExecDestroy(s->exec);
        s->exec = nullptr;
    }
    ServeDev d{s->d_sys, s->d_slots, s->d_items, s->d_n_items, s->d_next, s->d_n_acc, s->img_bytes};
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e) return srv_cuda(s, e, "begin capture");
    int le = launch_serve_step(d, s->precision, s->grid, s->smem, s->stream);
    e = cudaStreamEndCapture(s->stream, &g);
    if (le) {
        if (g) cudaGraphDestroy(g);
        return srv_cuda(s, (cudaError_t)le, "launch in capture");
    }
    if (e) return srv_cuda(s, e, "end capture");
    e = cudaGraphInstantiate(&s->exec, g, 0);
    cudaGraphDestroy(g);
    return e ? srv_cuda(s, e, "instantiate") : EWALD_OK;
}

int refresh_systems(ewald_server *s) {
    cudaError_t e = cudaMemcpyAsync(s->d_sys, s->sys_host.data(), sizeof(SysDev) * s->sys_host.size(),
                                    cudaMemcpyHostToDevice, s->stream);
    if (e) return srv_cuda(s, e, "system table");
    // the host copy must stay valid until the copy ran
    if ((e = cudaStreamSynchronize(s->stream))) return srv_cuda(s, e, "system table");
    size_t img = 0;
    size_t smem = serve_smem(s->sys_host, s->precision, &img);
    if (smem != s->smem || img != s->img_bytes || !s->exec) {
        s->smem = smem;
        s->img_bytes = img;
        if ((e = (cudaError_t)configure_serve(s->precision, smem, &s->grid))) return srv_cuda(s, e, "configure");
        int st = capture_step(s);
        if (st) return st;
    }
    s->systems_dirty = false;
    return EWALD_OK;
}

int admit(ewald_server *s, Req &r) {
    ewald_ctx *c = r.ctx;
    const SysDev &sd = c->s;
    cudaStream_t st = s->stream;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (!e) e = x; };
    BatchDev &b = r.b;
    b.W = r.W;
    const size_t slots = (size_t)sd.n_runs * sd.run_len * sd.n_layers;  // rho of every layer
    chk(aalloc(r, &b.u, (size_t)r.W * sd.dim * sd.mob_stride, st));
    chk(aalloc(r, &b.rho, (size_t)r.W * slots, st));
    chk(aalloc(r, &b.part_real, (size_t)r.W * std::max(c->max_items, sd.n_items), st));
    chk(aalloc(r, &b.part_recip, (size_t)r.W * sd.n_gchunks, st));
    chk(aalloc(r, &b.e, (size_t)r.W, st));
    chk(aalloc(r, &b.comp, (size_t)r.W * 5, st));
    chk(aalloc(r, &b.acc_count, (size_t)r.W, st));
    chk(aalloc(r, &b.pend_k, (size_t)r.W, st));
    chk(aalloc(r, &b.status, 1, st));
    b.pend_u = nullptr;
    b.resum_flag = nullptr;
    double *d_pos = nullptr;
    if (!e) e = cudaMallocAsync((void **)&d_pos, r.pos.size() * sizeof(double), st);
    if (!e) e = cudaMemcpyAsync(d_pos, r.pos.data(), r.pos.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemsetAsync(b.status, 0, sizeof(int), st);
    if (!e) e = (cudaError_t)launch_ingest(sd, b, d_pos, st);
    if (s->precision == EWALD_FP64_TIERED) {
        if (!e) e = (cudaError_t)launch_sfac_df(sd, b, c->cfg, nullptr, st);
    } else {
        if (!e) e = (cudaError_t)launch_sfac(sd, b, s->precision, c->cfg, nullptr, st);
    }
    // the real-space launch follows the context (tiered if it is)
    if (!e) e = (cudaError_t)launch_real(sd, b, c->t.precision, c->cfg, st);
    if (!e) e = (cudaError_t)launch_combine(sd, b, st);  // e = E0, acc_count = 0
    if (d_pos) cudaFreeAsync(d_pos, st);
    if (!e) e = cudaMemsetAsync(s->d_n_acc + r.acc_base, 0, sizeof(int) * r.W, st);
    if (e) return srv_cuda(s, e, "admission");
    r.pos.clear();
    r.pos.shrink_to_fit();
    return EWALD_OK;
}

}  // namespace

extern "C" {

int ewald_server_create(int precision, int max_walkers, double hbm_budget_bytes, void *stream, ewald_server **out) {
    if (!out) return EWALD_ERR_ARG;
    *out = nullptr;
    if ((precision != EWALD_FP64 && precision != EWALD_MIXED && precision != EWALD_FP64_TIERED) || max_walkers < 1)
        return EWALD_ERR_ARG;
    ewald_server *s = new (std::nothrow) ewald_server();
    if (!s) return EWALD_ERR_OOM;
    s->precision = precision;
    s->max_walkers = max_walkers;
    cudaError_t e = cudaSuccess;
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        s->own_stream = true;
    }
    size_t free_b = 0, total_b = 0;
    if (!e) e = cudaMemGetInfo(&free_b, &total_b);
    s->budget = hbm_budget_bytes > 0 ? (size_t)hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
    // keep freed request memory in the stream-ordered pool instead of
    // returning it to the CUDA driver at every synchronisation
    if (!e) {
        int dev = 0;
        cudaMemPool_t pool;
        e = cudaGetDevice(&dev);
        if (!e) e = cudaDeviceGetDefaultMemPool(&pool, dev);
        unsigned long long thr = ~0ull;
        if (!e) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    const int max_slots = 1024;
    auto dal = [&](void **p, size_t bytes) {
        if (e) return;
        e = cudaMalloc(p, bytes);
        if (!e) s->dev.push_back(*p);
    };
    dal((void **)&s->d_sys, sizeof(SysDev) * kMaxSystems);
    dal((void **)&s->d_slots, sizeof(SlotDev) * max_slots);
    dal((void **)&s->d_items, sizeof(int2) * max_walkers);
    dal((void **)&s->d_n_items, sizeof(int));
    dal((void **)&s->d_next, sizeof(int));
    dal((void **)&s->d_n_acc, sizeof(int) * max_walkers);
    for (int i = 0; i < 2 && !e; ++i) {
        e = cudaMallocHost((void **)&s->pin_slots[i], sizeof(SlotDev) * max_slots);
        if (!e) e = cudaMallocHost((void **)&s->pin_items[i], sizeof(int2) * max_walkers);
        if (!e) e = cudaMallocHost((void **)&s->pin_n[i], sizeof(int));
        if (!e) e = cudaEventCreateWithFlags(&s->ev_stage[i], cudaEventDisableTiming);
    }
    if (!e) e = cudaMemsetAsync(s->d_n_items, 0, sizeof(int), s->stream);
    s->slot_req.assign(max_slots, -1);
    s->acc_free.push_back({0, max_walkers});
    if (e) {
        ewald_server_destroy(s);
        return e == cudaErrorMemoryAllocation ? EWALD_ERR_OOM : EWALD_ERR_CUDA;
    }
    *out = s;
    return EWALD_OK;
}

void ewald_server_destroy(ewald_server *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (auto &kv : s->reqs) {
        Req &r = kv.second;
        for (void *p : r.dev) cudaFree(p);
        if (r.ev_done) cudaEventDestroy(r.ev_done);
        if (r.pin_e) cudaFreeHost(r.pin_e);
        if (r.pin_acc) cudaFreeHost(r.pin_acc);
    }
    if (s->exec) cudaGraphExecDestroy(s->exec);
    for (int i = 0; i < 2; ++i) {
        if (s->pin_slots[i]) cudaFreeHost(s->pin_slots[i]);
        if (s->pin_items[i]) cudaFreeHost(s->pin_items[i]);
        if (s->pin_n[i]) cudaFreeHost(s->pin_n[i]);
        if (s->ev_stage[i]) cudaEventDestroy(s->ev_stage[i]);
    }
    for (void *p : s->dev) cudaFree(p);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char *ewald_server_error_message(const ewald_server *s) { return s ? s->why.c_str() : "no server"; }

int ewald_server_submit(ewald_server *s, ewald_ctx *system, const double *pos, int n_walkers, int n_steps,
                        double sigma, double accept_prob, unsigned long long seed, int *request_id) {
    EWALD_NVTX("ewald_server_submit");
    if (!s || !system || !pos || !request_id || n_walkers < 1 || n_steps < 0 || !(sigma >= 0) ||
        !(accept_prob >= 0 && accept_prob <= 1))
        return srv_fail(s, EWALD_ERR_ARG, "bad request");
    // an FP64 server takes FP64 and tiered contexts, a tiered server tiered ones
    const bool ok = s->precision == EWALD_FP64_TIERED ? system->t.tiered : system->t.precision == s->precision;
    if (!ok) return srv_fail(s, EWALD_ERR_ARG, "system precision differs from the server's");
    if (n_walkers > s->max_walkers) return srv_fail(s, EWALD_ERR_ARG, "more walkers than the server's slots");
    const size_t nb = request_bytes(system, n_walkers);
    if (nb > s->budget) return srv_fail(s, EWALD_ERR_OOM, "request larger than the memory budget");
    const size_t n = (size_t)n_walkers * system->t.n_mob * system->t.dim;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(pos[i])) return srv_fail(s, EWALD_ERR_ARG, "non-finite position");
    Req r;
    r.id = s->next_id++;
    r.ctx = system;
    r.W = n_walkers;
    r.n_steps = n_steps;
    r.sigma = sigma;
    r.accept_p = accept_prob;
    r.seed = seed;
    r.pos.assign(pos, pos + n);
    r.bytes = nb;
    r.t_submit = now_s();
    *request_id = r.id;
    s->queue.push_back(r.id);
    s->reqs.emplace(r.id, std::move(r));
    return EWALD_OK;
}

int ewald_server_step(ewald_server *s, int *n_active, int *n_queued) {
    EWALD_NVTX("ewald_server_step");
    if (!s) return EWALD_ERR_ARG;
    cudaError_t e;
    // 1. requests whose results have arrived
    for (size_t i = 0; i < s->draining.size();) {
        Req &r = s->reqs[s->draining[i]];
        if (r.state == 2 && cudaEventQuery(r.ev_done) == cudaSuccess) {
            r.state = 3;
            r.t_done = now_s();
        }
        if (r.state == 3) {
            s->completed.push_back(r.id);
            s->draining[i] = s->draining.back();
            s->draining.pop_back();
        } else {
            ++i;
        }
    }
    // 2. retire finished requests (copies and frees are stream-ordered)
    for (size_t slot = 0; slot < s->slot_req.size(); ++slot) {
        int id = s->slot_req[slot];
        if (id < 0) continue;
        Req &r = s->reqs[id];
        if (r.cancel) {  // memory back to the pool after the moves already queued; no results
            for (void *p : r.dev) cudaFreeAsync(p, s->stream);
            r.dev.clear();
            r.state = 4;
            r.t_done = now_s();
            s->completed.push_back(r.id);
            s->slot_req[slot] = -1;
            s->used_walkers -= r.W;
            s->used_bytes -= r.bytes;
            give_acc_range(s, r.acc_base, r.W);
            s->items_dirty = true;
            continue;
        }
        if (r.steps_done < r.n_steps) continue;
        if (!r.pin_e) {
            if ((e = cudaMallocHost((void **)&r.pin_e, sizeof(double) * r.W))) return srv_cuda(s, e, "result buffer");
            if ((e = cudaMallocHost((void **)&r.pin_acc, sizeof(int) * r.W))) return srv_cuda(s, e, "result buffer");
        }
        e = cudaMemcpyAsync(r.pin_e, r.b.e, sizeof(double) * r.W, cudaMemcpyDeviceToHost, s->stream);
        if (!e) e = cudaMemcpyAsync(r.pin_acc, s->d_n_acc + r.acc_base, sizeof(int) * r.W, cudaMemcpyDeviceToHost, s->stream);
        if (!e && !r.ev_done) e = cudaEventCreateWithFlags(&r.ev_done, cudaEventDisableTiming);
        if (!e) e = cudaEventRecord(r.ev_done, s->stream);
        if (e) return srv_cuda(s, e, "retire");
        for (void *p : r.dev) cudaFreeAsync(p, s->stream);
        r.dev.clear();
        r.state = 2;
        s->draining.push_back(r.id);
        s->slot_req[slot] = -1;
        s->used_walkers -= r.W;
        s->used_bytes -= r.bytes;
        give_acc_range(s, r.acc_base, r.W);
        s->items_dirty = true;
    }
    // 3. admit queued requests while walker slots and memory allow
    while (!s->queue.empty()) {
        Req &r = s->reqs[s->queue.front()];
        if (s->used_walkers + r.W > s->max_walkers || s->used_bytes + r.bytes > s->budget) break;
        int slot = -1;
        for (size_t i = 0; i < s->slot_req.size(); ++i)
            if (s->slot_req[i] < 0) {
                slot = (int)i;
                break;
            }
        if (slot < 0) break;
        int base = take_acc_range(s, r.W);
        if (base < 0) break;  // fragmented: wait for a retirement
        r.sys = system_index(s, r.ctx);
        if (r.sys < 0) {
            give_acc_range(s, base, r.W);
            return srv_fail(s, EWALD_ERR_ARG, "too many distinct systems");
        }
        r.acc_base = base;
        r.slot = slot;
        int st = admit(s, r);
        if (st) return st;
        r.state = 1;
        r.t_admit = now_s();
        s->slot_req[slot] = r.id;
        s->used_walkers += r.W;
        s->used_bytes += r.bytes;
        s->items_dirty = true;
        s->queue.pop_front();
    }
    if (s->systems_dirty) {
        int st = refresh_systems(s);
        if (st) return st;
    }
    // 4. one move for every walker of every active request
    int n_act = 0;
    for (int id : s->slot_req)
        if (id >= 0 && s->reqs[id].steps_done < s->reqs[id].n_steps) ++n_act;
    if (n_act) {
        const int p = s->parity;
        if ((e = cudaEventSynchronize(s->ev_stage[p]))) return srv_cuda(s, e, "staging");
        SlotDev *ps = s->pin_slots[p];
        int n_items = 0, max_slot = 0;
        for (size_t slot = 0; slot < s->slot_req.size(); ++slot) {
            int id = s->slot_req[slot];
            if (id < 0) continue;
            Req &r = s->reqs[id];
            SlotDev &sl = ps[slot];
            sl.b = r.b;
            sl.sys = r.sys;
            sl.step = r.steps_done;
            sl.resum_every = r.ctx->t.resum_every;
            sl.walker_base = r.acc_base;
            sl.seed = r.seed;
            sl.sigma = r.sigma;
            sl.accept_p = r.accept_p;
            max_slot = (int)slot + 1;
            if (r.steps_done < r.n_steps)
                for (int w = 0; w < r.W; ++w) s->pin_items[p][n_items++] = make_int2((int)slot, w);
        }
        e = cudaMemcpyAsync(s->d_slots, ps, sizeof(SlotDev) * max_slot, cudaMemcpyHostToDevice, s->stream);
        // the item list changes only when requests come, go or finish; it is
        // rebuilt above every step (cheap) and uploaded when it changed
        if (!e && s->items_dirty) {
            *s->pin_n[p] = n_items;
            e = cudaMemcpyAsync(s->d_items, s->pin_items[p], sizeof(int2) * n_items, cudaMemcpyHostToDevice, s->stream);
            if (!e) e = cudaMemcpyAsync(s->d_n_items, s->pin_n[p], sizeof(int), cudaMemcpyHostToDevice, s->stream);
            s->items_dirty = false;
        }
        if (!e) e = cudaEventRecord(s->ev_stage[p], s->stream);
        if (!e) e = cudaGraphLaunch(s->exec, s->stream);
        if (e) return srv_cuda(s, e, "step");
        s->parity ^= 1;
        for (int id : s->slot_req)
            if (id >= 0 && s->reqs[id].steps_done < s->reqs[id].n_steps) {
                Req &r = s->reqs[id];
                r.steps_done += 1;
                if (r.steps_done == r.n_steps) s->items_dirty = true;
            }
    }
    if (n_active) {
        *n_active = 0;
        for (int id : s->slot_req) *n_active += id >= 0;
    }
    if (n_queued) *n_queued = (int)s->queue.size();
    return EWALD_OK;
}

int ewald_server_result(ewald_server *s, int request_id, double *energies, int *n_accepted, double *latency_ms) {
    if (!s) return EWALD_ERR_ARG;
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return srv_fail(s, EWALD_ERR_ARG, "unknown request");
    Req &r = it->second;
    if (r.state == 2 && cudaEventQuery(r.ev_done) == cudaSuccess) {
        r.state = 3;
        r.t_done = now_s();
    }
    if (r.state == 4) return EWALD_ERR_CANCELLED;
    if (r.state != 3) return EWALD_ERR_STATE;
    if (energies) std::memcpy(energies, r.pin_e, sizeof(double) * r.W);
    if (n_accepted) std::memcpy(n_accepted, r.pin_acc, sizeof(int) * r.W);
    if (latency_ms) *latency_ms = 1e3 * (r.t_done - r.t_submit);
    return EWALD_OK;
}

int ewald_server_completed(ewald_server *s, int *ids, int max_ids, int *n) {
    if (!s || !n || (max_ids > 0 && !ids)) return EWALD_ERR_ARG;
    const int k = std::min<int>(max_ids, (int)s->completed.size());
    for (int i = 0; i < k; ++i) ids[i] = s->completed[i];
    s->completed.erase(s->completed.begin(), s->completed.begin() + k);
    *n = k;
    return EWALD_OK;
}

int ewald_server_request_bytes(const ewald_ctx *system, int n_walkers, double *bytes) {
    if (!system || n_walkers < 1 || !bytes) return EWALD_ERR_ARG;
    *bytes = (double)request_bytes(system, n_walkers);
    return EWALD_OK;
}

int ewald_server_cancel(ewald_server *s, int request_id) {
    if (!s) return EWALD_ERR_ARG;
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return srv_fail(s, EWALD_ERR_ARG, "unknown request");
    Req &r = it->second;
    if (r.state == 0) {  // queued: nothing on the device yet
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r.id));
        r.state = 4;
        r.t_done = now_s();
        r.pos.clear();
        r.pos.shrink_to_fit();
        s->completed.push_back(r.id);
        return EWALD_OK;
    }
    if (r.state == 1 && !r.cancel && r.steps_done < r.n_steps) {
        r.cancel = true;
        return EWALD_OK;
    }
    return srv_fail(s, EWALD_ERR_STATE, "request already finished or cancelled");
}

int ewald_server_drain(ewald_server *s) {
    if (!s) return EWALD_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    return e ? srv_cuda(s, e, "drain") : EWALD_OK;
}

}  // extern "C"
