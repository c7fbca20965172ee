// Instantiation helper of the persistent chain launcher (value kinds that a
// chain supports: float64, float32, int64, Boolean).
#pragma once

#include "plan.h"
#include "chain.cuh"

#define SG_INSTANTIATE_CHAIN(IT, V, THREADS)                                                     \
    template cudaError_t launch_chain<IT, V, THREADS>(const ChainProduct*, ChainSync*, int, int, \
                                                      cudaStream_t, int*);                       \
    template size_t chain_smem_bytes<IT, V, THREADS>(int);
