// Device-side tables of the serving loop (serve_kernels.cu, serve.cu).
#pragma once
#include <vector>

#include "ewald_internal.h"

namespace ewald {

constexpr int kServeMinBlocks = 4;  // resident serving CTAs per SM the registers are sized for

// One active request: its walkers' state and its move stream.
struct SlotDev {
    BatchDev b;               // positions, rho(G), running energies e[W], acc_count
    int sys;                  // index into the system table
    int step;                 // moves already made (the generator's counter)
    int resum_every;
    int walker_base;          // first entry of this request in the n_acc array
    unsigned long long seed;
    double sigma, accept_p;
};

struct ServeDev {
    const SysDev *sys;
    const SlotDev *slots;
    const int2 *items;        // (slot, walker)
    const int *n_items;       // device count, so the launch can be replayed unchanged
    int *next;                // work counter
    int *n_acc;               // accepted moves per walker
    size_t img_bytes;
};

size_t serve_smem(const std::vector<SysDev> &sys, int precision, size_t *img_bytes);
int configure_serve(int precision, size_t smem, int *grid);
int launch_serve_step(const ServeDev &d, int precision, int grid, size_t smem, cudaStream_t st);

}  // namespace ewald
