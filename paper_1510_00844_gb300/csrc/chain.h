// Types of the persistent chain executor (see chain.cuh for the kernel):
// the per-product table the kernel walks, its barrier state, and the
// launcher templates instantiated in inst_chain_*.cu.
#pragma once

#include "plan.h"

namespace sg {

// Threads of a persistent block: 768 (24 warps at up to 80 registers, what
// the dense numeric stage needs), or 1024 (32 warps at up to 64 registers,
// for chains of short rows whose stages wait on memory latency).
constexpr int kChainThreads = 768;
constexpr int kChainThreadsWide = 1024;
constexpr int kChainMaxWarps = kChainThreadsWide / 32;
// Warps that run the dense numeric stage: 1024-column chunks on 24 warps,
// 2048-column chunks on 12 (their accumulators fill the shared memory).
constexpr int kChainDense0 = 24;
constexpr int kChainDense1 = 12;
constexpr int kDevTimeout = 8;       // a chain barrier wait expired

// One product of a chain: everything its stages read, from a device-sized
// plan, its workspace and its output arrays.
struct ChainProduct {
    const ProdDesc* D;
    const long long* rb;
    const long long* bb;
    DevCounters* cnt;
    int64_t* flops;
    unsigned char* cls;
    int32_t* rows;
    int64_t* cap;
    const float* prm;
    int32_t* chunkcnt;
    int32_t* segtab;
    int32_t* runlen;
    int2* nextrun;
    DenseCursor* arena;
    int64_t* scan;        // tile sums of the row-pointer scan
    int64_t* rowptrC;
    void* colC;
    void* valC;
    long long R, LB, max_dense_n, arena_stride, capacity;
    float margin;
    int nprod, W, dense_min, hash_shift, seg_log2, max_words;
};

// Barrier state (first 16 bytes cleared by the host before every launch)
// and the chain's configuration.
struct ChainSync {
    unsigned int arrived;   // barrier arrivals of this launch
    int status;             // kDevOk or kDevTimeout
    int abort;
    int pad0;
    unsigned long long timeout_ns;
    int withhold;           // stage whose completion no block signals (-1: none)
    int nsteps;
    unsigned long long* stamps;  // NULL, or 2 + 6 * nsteps %globaltimer readings
};

template <class IT, class V, int THREADS>
size_t chain_smem_bytes(int max_words);
template <class IT, class V, int THREADS>
cudaError_t launch_chain(const ChainProduct* steps, ChainSync* sync, int max_words, int sm_count,
                         cudaStream_t s, int* grid_out);

}  // namespace sg
