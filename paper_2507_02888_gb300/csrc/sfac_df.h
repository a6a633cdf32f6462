// Structure factor of the tiered FP64 form in double-float arithmetic
// (sfac_df.cu): the same launch as launch_sfac for an FP64 context.
#pragma once
#include "ewald_internal.h"

namespace ewald {
int launch_sfac_df(const SysDev &s, const BatchDev &b, const LaunchCfg &cfg, const unsigned char *only,
                   cudaStream_t st);
}
