// Persistent execution of a chain of device-sized products in ONE kernel
// launch (batched and dependent products, e.g. the levels of a Galerkin
// hierarchy R^T A R, Sec. 5.4).  Not in the paper: the paper runs each
// multiplication as its own step; here every phase of every product of the
// chain runs inside one resident grid, and the grid waits at a device-side
// barrier wherever a phase needs the previous phase's results:
//
//   stage 0        zero every product's counters and the last row pointer
//   per product p  analyze | class offsets + binning | symbolic (empty rows,
//                  hash bins, dense tables, dense rows) | scan: tile sums |
//                  scan: apply | numeric (hash bins, dense rows)
//
// with one barrier after every stage.  The stage bodies are the same device
// code the standalone kernels run, called with the persistent block as their
// block, so a chain gives the same result, bit for bit, as the launch sequence
// of spgemm_execute.  Product p+1 may read what product p wrote (its A or B
// arrays may be product p's output): the barrier after p's numeric stage
// orders them.
//
// Every barrier wait is bounded: a block that has waited longer than the
// chain's timeout records kDevTimeout in the chain's status word, raises the
// abort flag and returns; blocks that see the abort flag return at their
// next barrier.  The grid is sized to be resident (blocks per SM from the
// occupancy calculator); if it is not (another kernel holds SMs), the wait
// times out instead of hanging.
#pragma once

#include "chain.h"

namespace sg {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier after stage `idx`: true when every block has finished stage
// idx, false when the wait expired or another block gave up.
__device__ __forceinline__ bool chain_barrier(ChainSync* s, int idx) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (idx != s->withhold) atomicAdd(&s->arrived, 1u);
        const unsigned target = (unsigned)(idx + 1) * gridDim.x;
        const unsigned long long t0 = globaltimer_ns();
        const unsigned long long limit = s->timeout_ns;
        volatile unsigned* arrived = &s->arrived;
        volatile int* abort = &s->abort;
        int res = 1;
        while (*arrived < target) {
            if (*abort) {
                res = 0;
                break;
            }
            if (globaltimer_ns() - t0 > limit) {
                atomicExch(&s->status, kDevTimeout);
                atomicExch(&s->abort, 1);
                res = 0;
                break;
            }
            __nanosleep(128);
        }
        ok = res;
        if (res && blockIdx.x == 0 && s->stamps) s->stamps[idx + 1] = globaltimer_ns();
    }
    __syncthreads();
    __threadfence();   // every thread orders its later loads after the barrier
    return ok != 0;
}

// Class offsets and row binning in one stage.  Block 0 records the offsets
// and dense work-unit prefix in the counters (later stages read them); every
// block computes the offsets itself and places its rows at offset + a slot
// taken from a cursor that starts at zero.
__device__ __forceinline__ void chain_bin(const ChainProduct& c, long long bid, long long nb) {
    __shared__ unsigned long long off[kNumClasses];
    __shared__ unsigned long long loc[kNumClasses];
    __shared__ unsigned long long base[kNumClasses];
    DevCounters* cnt = c.cnt;
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int t = 0; t < kNumClasses; ++t) {
            off[t] = s;
            s += cnt->class_count[t];
        }
        if (bid == 0) {
            cnt->seg_log2 = c.seg_log2;
            for (int t = 0; t < kNumClasses; ++t) cnt->class_off[t] = off[t];
            cnt->class_off[kNumClasses] = s;
            unsigned long long u = 0;
            for (int t = 0; t < kMaxDenseClasses; ++t) {
                cnt->unit_begin[t] = u;
                u += cnt->class_count[kClassDense0 + t] *
                     (unsigned long long)dense_class_segments(t, c.seg_log2);
            }
            cnt->unit_begin[kMaxDenseClasses] = u;
        }
    }
    for (int t = threadIdx.x; t < kNumClasses; t += blockDim.x) loc[t] = 0;
    __syncthreads();
    const long long per_block = (c.R + nb - 1) / nb;
    const long long r0 = bid * per_block;
    const long long r1 = min(c.R, r0 + per_block);
    bin_block_rows(c.cls, c.rows, r0, r1, loc, nullptr);
    __syncthreads();
    for (int t = threadIdx.x; t < kNumClasses; t += blockDim.x) {
        base[t] = off[t] + (loc[t] ? atomicAdd(&cnt->class_cursor[t], loc[t]) : 0ull);
        loc[t] = 0;
    }
    __syncthreads();
    bin_block_rows(c.cls, c.rows, r0, r1, loc, base);
}

// Row-pointer scan, first stage: sums of tiles of kScanTile entries.
__device__ __forceinline__ void chain_scan_sums(const int64_t* x, long long N, int64_t* part,
                                                long long bid, long long nb) {
    __shared__ long long ws[kChainMaxWarps];
    const long long ntiles = (N + kScanTile - 1) / kScanTile;
    for (long long tile = bid; tile < ntiles; tile += nb) {
        long long s = 0;
        for (long long idx = tile * kScanTile + threadIdx.x; idx < min(N, (tile + 1) * kScanTile);
             idx += blockDim.x)
            s += x[idx];
        s = warp_sum(s);
        if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x < 32) {
            long long v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0;
            v = warp_sum(v);
            if (threadIdx.x == 0) part[tile] = v;
        }
        __syncthreads();
    }
}

// Second stage: every tile adds the sums of the tiles before it (read by the
// block itself) and scans its entries in place (exclusive).
__device__ __forceinline__ void chain_scan_apply(int64_t* x, long long N, const int64_t* part,
                                                 long long bid, long long nb) {
    __shared__ long long ws[kChainMaxWarps];
    __shared__ long long carry;
    const long long ntiles = (N + kScanTile - 1) / kScanTile;
    for (long long tile = bid; tile < ntiles; tile += nb) {
        long long pre = 0;
        for (long long u = threadIdx.x; u < tile; u += blockDim.x) pre += part[u];
        pre = warp_sum(pre);
        if (lane_id() == 0) ws[threadIdx.x >> 5] = pre;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
            carry = t;
        }
        __syncthreads();
        const long long lim = min(N, (tile + 1) * kScanTile);
        for (long long b0 = tile * kScanTile; b0 < lim; b0 += blockDim.x) {
            const long long idx = b0 + threadIdx.x;
            const long long v = idx < lim ? x[idx] : 0;
            const long long inc = warp_incl_scan(v);
            if (lane_id() == 31) ws[threadIdx.x >> 5] = inc;
            __syncthreads();
            if (threadIdx.x < 32) {
                const long long w = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0;
                const long long wi = warp_incl_scan(w);
                if (threadIdx.x < (blockDim.x >> 5)) ws[threadIdx.x] = wi - w;
            }
            __syncthreads();
            const long long excl = carry + ws[threadIdx.x >> 5] + inc - v;
            if (idx < lim) x[idx] = excl;
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1) carry = excl + v;
            __syncthreads();
        }
    }
}

// Empty rows: count 0.
__device__ __forceinline__ void chain_zero_rows(const ChainProduct& c, long long bid, long long nb) {
    const long long nrows = (long long)c.cnt->class_count[kClassEmpty];
    const int32_t* erow = c.rows + c.cnt->class_off[kClassEmpty];
    for (long long r = bid * blockDim.x + threadIdx.x; r < nrows; r += nb * blockDim.x)
        c.rowptrC[erow[r]] = 0;
}

// Warps of a persistent block of BW warps that run a hash bin with tables
// of 2^LOG2T slots: as many as their tables fit in the shared-memory budget
// (the others wait at the stage's end).  The budget is what a block may hold
// on sm_103 (227 KB) less the kernel's own static arrays (under 8 KB); it
// lets 24 warps hold float32 tables of 1024 slots.
constexpr size_t kChainSmemBudget = 216 * 1024;
template <class K, class V, int LOG2T, bool NUMERIC, int BW>
constexpr int chain_bin_warps() {
    constexpr size_t vb = NUMERIC && VOps<V>::has_val ? sizeof(V) : 0;
    constexpr size_t per = (size_t(1) << LOG2T) * (sizeof(K) + vb) + (NUMERIC ? 1024 : 0);
    return (int)(kChainSmemBudget / per) >= BW ? BW : (int)(kChainSmemBudget / per);
}

// One hash bin of the symbolic / numeric stage on the warps its tables allow.
template <class IT, class K, int LOG2T, int BW>
__device__ __forceinline__ void chain_sym_bin(const ChainProduct& c, int* err, long long bid,
                                              long long nb) {
    constexpr int WARPS = chain_bin_warps<K, NoVal, LOG2T, false, BW>();
    static_assert(WARPS >= 1, "a hash bin's table must fit the shared-memory budget");
    const int cls = kClassHash0 + (LOG2T == 6 ? 0 : LOG2T == 8 ? 1 : LOG2T == 10 ? 2 : 3);
    if (threadIdx.x < WARPS * 32)
        symbolic_hash_kernel_body<IT, LOG2T, WARPS>(c.D, c.rb, c.nprod, c.rows, c.cnt, cls,
                                                    c.rowptrC, err, bid, nb);
    __syncthreads();
}

template <class IT, class V, class K, int LOG2T, int BW>
__device__ __forceinline__ void chain_num_bin(const ChainProduct& c, IT* colC, V* valC, int* err,
                                              long long bid, long long nb) {
    constexpr int WARPS = chain_bin_warps<K, V, LOG2T, true, BW>();
    static_assert(WARPS >= 1, "a hash bin's table must fit the shared-memory budget");
    const int cls = kClassHash0 + (LOG2T == 6 ? 0 : LOG2T == 8 ? 1 : LOG2T == 10 ? 2 : 3);
    if (threadIdx.x < WARPS * 32)
        numeric_hash_kernel_body<IT, V, LOG2T, WARPS>(c.D, c.rb, c.nprod, c.rows, c.cnt, cls,
                                                      c.rowptrC, c.capacity, colC, valC, err,
                                                      nullptr, nullptr, nullptr, bid, nb);
    __syncthreads();
}

template <class IT, class V, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
    chain_kernel(const ChainProduct* __restrict__ steps, ChainSync* sync, int sym_groups) {
    constexpr int BW = THREADS / 32;
    const long long bid = blockIdx.x, nb = gridDim.x;
    const int nsteps = sync->nsteps;
    if (bid == 0 && threadIdx.x == 0 && sync->stamps) sync->stamps[0] = globaltimer_ns();
    int stage = 0;
    // stage 0: counters of every product and the last row pointer to zero
    for (int p = 0; p < nsteps; ++p) {
        unsigned long long* w = reinterpret_cast<unsigned long long*>(steps[p].cnt);
        constexpr int nw = (int)(sizeof(DevCounters) / sizeof(unsigned long long));
        for (long long t = bid * blockDim.x + threadIdx.x; t < nw; t += nb * blockDim.x) w[t] = 0ull;
        if (bid == 0 && threadIdx.x == 0) steps[p].rowptrC[steps[p].R] = 0;
    }
    if (!chain_barrier(sync, stage++)) return;
    for (int p = 0; p < nsteps; ++p) {
        const ChainProduct c = steps[p];
        int* err = &c.cnt->err;
        // row analysis
        analyze_kernel_body<IT>(c.R, c.D, c.rb, c.nprod, c.max_dense_n, c.dense_min, c.flops,
                                c.cls, c.cnt, c.prm, c.margin, c.cap, c.hash_shift, bid, nb);
        if (!chain_barrier(sync, stage++)) return;
        chain_bin(c, bid, nb);
        if (!chain_barrier(sync, stage++)) return;
        // symbolic phase: row counts into rowptrC
        chain_zero_rows(c, bid, nb);
        using K = typename KeyT<IT>::type;
        chain_sym_bin<IT, K, 6, BW>(c, err, bid, nb);
        chain_sym_bin<IT, K, 8, BW>(c, err, bid, nb);
        chain_sym_bin<IT, K, 10, BW>(c, err, bid, nb);
        chain_sym_bin<IT, K, 11, BW>(c, err, bid, nb);
        if (c.LB > 0) {
            segtab_kernel_body<IT>(c.LB, c.D, c.bb, c.nprod, c.W, c.segtab, c.cnt, bid, nb);
            runlen_kernel_body<IT>(c.LB, c.D, c.bb, c.nprod, c.W, c.runlen, c.nextrun, c.cnt, bid,
                                   nb);
        }
        symbolic_dense_kernel_body<IT, THREADS, 1>(
            c.D, c.rb, c.nprod, c.rows, c.cnt, c.max_words, c.W / 32, c.chunkcnt, c.rowptrC,
            &c.cnt->work_counter[0], err, bid, nb, sym_groups);
        if (!chain_barrier(sync, stage++)) return;
        // row pointers: exclusive scan of the counts (R + 1 entries)
        chain_scan_sums(c.rowptrC, c.R + 1, c.scan, bid, nb);
        if (!chain_barrier(sync, stage++)) return;
        chain_scan_apply(c.rowptrC, c.R + 1, c.scan, bid, nb);
        if (!chain_barrier(sync, stage++)) return;
        // numeric phase
        IT* colC = (IT*)c.colC;
        V* valC = (V*)c.valC;
        chain_num_bin<IT, V, K, 6, BW>(c, colC, valC, err, bid, nb);
        chain_num_bin<IT, V, K, 8, BW>(c, colC, valC, err, bid, nb);
        chain_num_bin<IT, V, K, 10, BW>(c, colC, valC, err, bid, nb);
        chain_num_bin<IT, V, K, 11, BW>(c, colC, valC, err, bid, nb);
        if (c.W == kDenseW0) {
            if (threadIdx.x < kChainDense0 * 32)
                numeric_dense_kernel_body<IT, V, kDenseW0, kChainDense0>(
                c.D, c.rb, c.nprod, c.rows, c.cnt, c.chunkcnt, c.segtab, c.runlen, c.nextrun,
                c.arena, c.arena_stride, c.rowptrC, c.capacity, colC, valC, c.max_dense_n,
                &c.cnt->work_counter[1], err, nullptr, nullptr, nullptr, nullptr, bid, nb);
        } else if (threadIdx.x < kChainDense1 * 32) {
            numeric_dense_kernel_body<IT, V, kDenseW1, kChainDense1>(
                c.D, c.rb, c.nprod, c.rows, c.cnt, c.chunkcnt, c.segtab, c.runlen, c.nextrun,
                c.arena, c.arena_stride, c.rowptrC, c.capacity, colC, valC, c.max_dense_n,
                &c.cnt->work_counter[1], err, nullptr, nullptr, nullptr, nullptr, bid, nb);
        }
        if (!chain_barrier(sync, stage++)) return;
    }
}

// Shared memory of the persistent block: the largest stage of the chain.
template <class IT, class V, int THREADS>
size_t chain_smem_bytes(int max_words) {
    constexpr int BW = THREADS / 32;
    using K = typename KeyT<IT>::type;
    constexpr size_t vb = VOps<V>::has_val ? sizeof(V) : 0;
    auto bin = [&](int log2t, int warps, bool numeric) {
        return (size_t)warps * (((size_t)1 << log2t) * (sizeof(K) + (numeric ? vb : 0)) +
                                (numeric ? 1024 : 0));
    };
    size_t b = 0;
    b = std::max(b, bin(10, chain_bin_warps<K, NoVal, 10, false, BW>(), false));
    b = std::max(b, bin(11, chain_bin_warps<K, NoVal, 11, false, BW>(), false));
    b = std::max(b, bin(8, chain_bin_warps<K, V, 8, true, BW>(), true));
    b = std::max(b, bin(10, chain_bin_warps<K, V, 10, true, BW>(), true));
    b = std::max(b, bin(11, chain_bin_warps<K, V, 11, true, BW>(), true));
    b = std::max(b, (size_t)kChainDense0 * ((vb * kDenseW0) + kDenseW0 / 8 + 32 * sizeof(DenseRun<V>)));
    b = std::max(b, (size_t)kChainDense1 * ((vb * kDenseW1) + kDenseW1 / 8 + 32 * sizeof(DenseRun<V>)));
    b = std::max(b, (size_t)max_words * 4);                                         // dense symbolic
    return b;
}

template <class IT, class V, int THREADS>
cudaError_t launch_chain(const ChainProduct* steps, ChainSync* sync, int max_words, int sm_count,
                         cudaStream_t s, int* grid_out) {
    auto k = chain_kernel<IT, V, THREADS>;
    const size_t smem = chain_smem_bytes<IT, V, THREADS>(max_words);
    // the dense symbolic stage runs one row per group of at least four
    // warps, as many groups as their bitmaps fit the block's shared memory
    int sym_groups = 1;
    for (int gg : {8, 6, 4, 3, 2})
        if ((THREADS / 32) % gg == 0 && THREADS / 32 / gg >= 4 &&
            (size_t)gg * (size_t)max_words * 4 <= smem) {
            sym_groups = gg;
            break;
        }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, THREADS, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int grid = sm_count * occ;
    if (grid_out) *grid_out = grid;
    if ((e = cudaMemsetAsync(sync, 0, 16, s)) != cudaSuccess) return e;
    count_launches(1);
    k<<<grid, THREADS, smem, s>>>(steps, sync, sym_groups);
    return cudaGetLastError();
}

}  // namespace sg
