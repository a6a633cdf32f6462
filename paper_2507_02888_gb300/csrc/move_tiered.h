// Proposed moves of the tiered FP64 form (move_tiered.cu): the same launch
// as launch_propose for an FP64 context whose real space is tiered.
#pragma once
#include "ewald_internal.h"

namespace ewald {
int launch_propose_tiered(const SysDev &s, const BatchDev &b, const int *k, const double *r_new, double *de,
                          cudaStream_t st);
}
