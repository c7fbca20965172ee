// Template host launchers; included by the per-index-type instantiation units.
// Every class kernel reads its row range from the device counters, so a
// launch sequence needs no host readback (host-synced plans only use their
// copies of the counts to skip empty classes and to size grids).
#pragma once

#include "plan.h"

namespace sg {

template <class F>
int occupancy_blocks(F kernel, int threads, size_t smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess ||
        b < 1)
        b = 1;
    return b;
}

template <class F>
cudaError_t allow_smem(F kernel, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

inline long long grid_for(long long work_items, int per_block, int sm_count, int occ) {
    long long need = (work_items + per_block - 1) / per_block;
    long long cap = (long long)sm_count * occ;
    return std::max<long long>(1, std::min(need, cap));
}

// Grid of a class kernel: the class's rows when known, one resident wave when not.
inline long long class_grid(const Plan& P, long long rows_known, int per_block, int occ) {
    if (P.device_sized) return (long long)P.sm_count * occ;
    return grid_for(rows_known, per_block, P.sm_count, occ);
}

// Shared memory per warp of the dense numeric kernel (accumulator, bitmap,
// table of the current batch's runs).
template <class V, int W>
constexpr size_t dense_warp_bytes() {
    return (VOps<V>::has_val ? sizeof(V) * W : 0) + W / 8 + 32 * sizeof(DenseRun<V>);
}

template <class IT>
cudaError_t launch_analyze(Plan& P) {
    if (P.R <= 0) return cudaSuccess;
    auto k = analyze_kernel<IT>;
    int occ = occupancy_blocks(k, 256, 0);
    // a warp per tile of 32 rows
    long long g = grid_for(P.R, 256, P.sm_count, occ);
    count_launches(1);
    k<<<(unsigned)g, 256, 0, P.stream>>>(P.R, P.d_descs, P.rb, P.nprod, P.max_dense_n,
                                           P.dense_min, P.flops, P.cls, P.cnt, P.prm, P.margin,
                                           P.cap, P.hash_shift);
    return cudaGetLastError();
}

template <class IT>
cudaError_t launch_row_features(Plan& P, float* X) {
    if (P.R <= 0) return cudaSuccess;
    long long g = grid_for(P.R, 8, P.sm_count, 8);
    count_launches(1);
    row_features_kernel<IT><<<(unsigned)g, 256, 0, P.stream>>>(P.R, P.d_descs, P.rb, P.nprod, X);
    return cudaGetLastError();
}

template <class IT>
cudaError_t launch_validate(const spgemm_csr& M, int* err, int sm_count, cudaStream_t s) {
    if (M.nrows <= 0) return cudaSuccess;
    auto k = validate_kernel<IT>;
    long long g = grid_for(M.nrows, 8, sm_count, 8);
    count_launches(1);
    k<<<(unsigned)g, 256, 0, s>>>(M.nrows, M.ncols, M.nnz, M.rowptr, M.rowend, (const IT*)M.col,
                                  err);
    return cudaGetLastError();
}

template <class IT>
cudaError_t launch_kslice_bounds(const spgemm_csr& A, int c, int64_t* bounds, int sm_count,
                                 cudaStream_t s) {
    long long total = A.nrows * (long long)(c + 1);
    if (total <= 0) return cudaSuccess;
    long long g = grid_for(total, 256, sm_count, 8);
    count_launches(1);
    kslice_bounds_kernel<IT><<<(unsigned)g, 256, 0, s>>>(A.nrows, A.ncols, c, A.rowptr,
                                                         (const IT*)A.col, bounds);
    return cudaGetLastError();
}

template <class IT, int LOG2T, int WARPS>
cudaError_t sym_hash_bin(Plan& P, int bin, int64_t* rowcnt) {
    using K = typename KeyT<IT>::type;
    const int c = kClassHash0 + bin;
    const long long nrows = (long long)P.class_count[c];
    if (!P.device_sized && nrows == 0) return cudaSuccess;
    if (P.device_sized && bin > 0 && (hash_bin_flops(bin - 1) >> P.hash_shift) >= P.dense_min)
        return cudaSuccess;
    auto k = symbolic_hash_kernel<IT, LOG2T, WARPS>;
    size_t smem = LOG2T == kShortLog2T ? 0 : (size_t)WARPS * (1u << LOG2T) * sizeof(K);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    int occ = occupancy_blocks(k, WARPS * 32, smem);
    long long g = class_grid(P, nrows, WARPS, occ);
    count_launches(1);
    k<<<(unsigned)g, WARPS * 32, smem, P.stream>>>(P.d_descs, P.rb, P.nprod, P.rows, P.cnt, c,
                                                   rowcnt, &P.cnt->err);
    return cudaGetLastError();
}

// Tables of B the dense numeric kernel walks with: segment starts per B row,
// the run length of every B entry inside its chunk and each run's successor.
template <class IT>
cudaError_t launch_dense_tables(Plan& P, unsigned char* ws) {
    WsLayout L = workspace_layout(P);
    cudaError_t e = cudaSuccess;
    const bool dense = P.device_sized || P.ndense > 0;
    if (dense && P.LB > 0) {
        long long total = P.LB * (kSegGrid + 1);
        long long g = grid_for(total, 256, P.sm_count, 8);
        count_launches(1);
        segtab_kernel<IT><<<(unsigned)g, 256, 0, P.stream>>>(P.LB, P.d_descs, P.bb, P.nprod, P.W,
                                                             (int32_t*)(ws + L.segtab), P.cnt);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        long long g2 = grid_for(P.LB, 8, P.sm_count, 8);
        count_launches(1);
        runlen_kernel<IT><<<(unsigned)g2, 256, 0, P.stream>>>(P.LB, P.d_descs, P.bb, P.nprod, P.W,
                                                              (int32_t*)(ws + L.runlen),
                                                              (int2*)(ws + L.nextrun), P.cnt);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return e;
}

template <class IT>
cudaError_t launch_symbolic(Plan& P, unsigned char* ws, int64_t* rowcnt) {
    WsLayout L = workspace_layout(P);
    cudaError_t e = launch_zero_rows(P, rowcnt);
    if (e != cudaSuccess) return e;
    if ((e = sym_hash_bin<IT, 6, 8>(P, 0, rowcnt)) != cudaSuccess) return e;
    if ((e = sym_hash_bin<IT, 8, 8>(P, 1, rowcnt)) != cudaSuccess) return e;
    if ((e = sym_hash_bin<IT, 10, 8>(P, 2, rowcnt)) != cudaSuccess) return e;
    if ((e = sym_hash_bin<IT, 11, 8>(P, 3, rowcnt)) != cudaSuccess) return e;
    const bool dense = P.device_sized || P.ndense > 0;
    if ((e = launch_dense_tables<IT>(P, ws)) != cudaSuccess) return e;
    if (dense) {
        // one block per row; the block size follows the bitmap: the most
        // resident warps, and among equals the smaller blocks (more rows in
        // flight) -- 256 threads while six blocks fit, 1024 when only one does
        auto ks = symbolic_dense_kernel<IT, 512, 3>;
        auto kb = symbolic_dense_kernel<IT, 1024, 1>;
        const int max_words = (int)((std::min(P.max_n, P.max_dense_n) + 31) / 32);
        size_t smem = (size_t)max_words * 4;
        if ((e = allow_smem(ks, smem)) != cudaSuccess) return e;
        if ((e = allow_smem(kb, smem)) != cudaSuccess) return e;
        int threads = 256, occ = occupancy_blocks(ks, 256, smem);
        const int o512 = occupancy_blocks(ks, 512, smem);
        if (o512 * 512 > occ * threads) { threads = 512; occ = o512; }
        const int o1024 = occupancy_blocks(kb, 1024, smem);
        if (o1024 * 1024 > occ * threads) { threads = 1024; occ = o1024; }
        long long g = class_grid(P, P.ndense, 1, occ);
        unsigned long long* work = &P.cnt->work_counter[0];
        if ((e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), P.stream)) != cudaSuccess)
            return e;
        count_launches(1);
        if (threads == 1024)
            kb<<<(unsigned)g, threads, smem, P.stream>>>(P.d_descs, P.rb, P.nprod, P.rows, P.cnt,
                                                         max_words, P.W / 32,
                                                         (int32_t*)(ws + L.chunkcnt), rowcnt, work,
                                                         &P.cnt->err);
        else
            ks<<<(unsigned)g, threads, smem, P.stream>>>(P.d_descs, P.rb, P.nprod, P.rows, P.cnt,
                                                         max_words, P.W / 32,
                                                         (int32_t*)(ws + L.chunkcnt), rowcnt, work,
                                                         &P.cnt->err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class IT, class V, int LOG2T, int WARPS>
cudaError_t num_hash_bin(Plan& P, int bin, const int64_t* rpC, long long cap, IT* colC,
                         V* valC, int64_t* rowend, int32_t* overflow, unsigned* overflow_count) {
    using K = typename KeyT<IT>::type;
    const int c = kClassHash0 + bin;
    const long long nrows = (long long)P.class_count[c];
    if (!P.device_sized && nrows == 0) return cudaSuccess;
    if (P.device_sized && bin > 0 && (hash_bin_flops(bin - 1) >> P.hash_shift) >= P.dense_min)
        return cudaSuccess;
    auto k = numeric_hash_kernel<IT, V, LOG2T, WARPS>;
    constexpr size_t vb = VOps<V>::has_val ? sizeof(V) : 0;
    size_t smem = LOG2T == kShortLog2T
                      ? 0
                      : (size_t)WARPS * ((1u << LOG2T) * (sizeof(K) + vb) + 256 * sizeof(int));
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    int occ = occupancy_blocks(k, WARPS * 32, smem);
    long long g = class_grid(P, nrows, WARPS, occ);
    count_launches(1);
    k<<<(unsigned)g, WARPS * 32, smem, P.stream>>>(P.d_descs, P.rb, P.nprod, P.rows, P.cnt, c,
                                                   rpC, cap, colC, valC, &P.cnt->err, rowend,
                                                   overflow, overflow_count);
    return cudaGetLastError();
}

template <class IT, class V, int W, int WARPS>
cudaError_t launch_numeric_dense(Plan& P, unsigned char* ws, const int64_t* rpC, long long cap,
                                 IT* colC, V* valC, int64_t* rowend, int32_t* overflow,
                                 unsigned* overflow_count) {
    WsLayout L = workspace_layout(P);
    auto k = numeric_dense_kernel<IT, V, W, WARPS>;
    size_t smem = (size_t)WARPS * dense_warp_bytes<V, W>();
    cudaError_t e;
    if ((e = allow_smem(k, smem)) != cudaSuccess) return e;
    unsigned long long* work = &P.cnt->work_counter[1];
    if ((e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), P.stream)) != cudaSuccess)
        return e;
    count_launches(1);
    k<<<(unsigned)P.dense_grid, WARPS * 32, smem, P.stream>>>(
        P.d_descs, P.rb, P.nprod, P.rows, P.cnt, (const int32_t*)(ws + L.chunkcnt),
        (const int32_t*)(ws + L.segtab), (const int32_t*)(ws + L.runlen),
        (const int2*)(ws + L.nextrun), (DenseCursor*)(ws + L.arena), L.arena_stride, rpC, cap, colC, valC, P.max_dense_n, work,
        &P.cnt->err, rowend, overflow, overflow_count, P.unit_cnt);
    return cudaGetLastError();
}

template <class IT, class V>
cudaError_t launch_numeric(Plan& P, unsigned char* ws, const int64_t* rpC, long long cap,
                           void* colC_, void* valC_, int64_t* rowend, int32_t* overflow,
                           unsigned* overflow_count) {
    IT* colC = (IT*)colC_;
    V* valC = (V*)valC_;
    cudaError_t e;
    if ((e = num_hash_bin<IT, V, 6, 8>(P, 0, rpC, cap, colC, valC, rowend, overflow, overflow_count)) != cudaSuccess) return e;
    if ((e = num_hash_bin<IT, V, 8, 8>(P, 1, rpC, cap, colC, valC, rowend, overflow, overflow_count)) != cudaSuccess) return e;
    if ((e = num_hash_bin<IT, V, 10, 8>(P, 2, rpC, cap, colC, valC, rowend, overflow, overflow_count)) != cudaSuccess) return e;
    if ((e = num_hash_bin<IT, V, 11, 4>(P, 3, rpC, cap, colC, valC, rowend, overflow, overflow_count)) != cudaSuccess) return e;
    if (P.device_sized || P.ndense > 0) {
        e = P.W == kDenseW0
                ? launch_numeric_dense<IT, V, kDenseW0, kDenseWarps0>(P, ws, rpC, cap, colC, valC,
                                                                      rowend, overflow, overflow_count)
                : launch_numeric_dense<IT, V, kDenseW1, kDenseWarps1>(P, ws, rpC, cap, colC, valC,
                                                                      rowend, overflow, overflow_count);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class IT, class V, int W, int WARPS>
cudaError_t prepare_numeric_dense(Plan& P) {
    auto k = numeric_dense_kernel<IT, V, W, WARPS>;
    size_t smem = (size_t)WARPS * dense_warp_bytes<V, W>();
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    int occ = occupancy_blocks(k, WARPS * 32, smem);
    P.dense_warps_per_block = WARPS;
    P.dense_grid = (long long)P.sm_count * occ;
    return cudaSuccess;
}

// Grid of the dense numeric kernel (one resident wave; units are grabbed
// dynamically), fixed at plan time so the workspace can size the cursor arena.
template <class IT, class V>
cudaError_t prepare_numeric(Plan& P) {
    return P.W == kDenseW0 ? prepare_numeric_dense<IT, V, kDenseW0, kDenseWarps0>(P)
                           : prepare_numeric_dense<IT, V, kDenseW1, kDenseWarps1>(P);
}

template <class IT, class V>
cudaError_t launch_dense_slot_pack(Plan& P, const int64_t* rpC, void* colC, void* valC,
                                   int64_t* rowend) {
    if (P.ndense == 0) return cudaSuccess;
    long long g = grid_for(P.ndense, 8, P.sm_count, 8);
    count_launches(1);
    dense_slot_pack_kernel<IT, V><<<(unsigned)g, 256, 0, P.stream>>>(
        P.d_descs, P.rb, P.nprod, P.rows, P.cnt, rpC, P.unit_cnt, rowend, (IT*)colC, (V*)valC);
    return cudaGetLastError();
}

#define SG_INSTANTIATE_IT(IT)                                                                   \
    template cudaError_t launch_analyze<IT>(Plan&);                                            \
    template cudaError_t launch_dense_tables<IT>(Plan&, unsigned char*);                       \
    template cudaError_t launch_dense_slot_pack<IT, double>(Plan&, const int64_t*, void*,      \
                                                            void*, int64_t*);                  \
    template cudaError_t launch_dense_slot_pack<IT, float>(Plan&, const int64_t*, void*,       \
                                                           void*, int64_t*);                   \
    template cudaError_t launch_dense_slot_pack<IT, int64_t>(Plan&, const int64_t*, void*,     \
                                                             void*, int64_t*);                 \
    template cudaError_t launch_dense_slot_pack<IT, NoVal>(Plan&, const int64_t*, void*,       \
                                                           void*, int64_t*);                   \
    template cudaError_t launch_validate<IT>(const spgemm_csr&, int*, int, cudaStream_t);      \
    template cudaError_t launch_symbolic<IT>(Plan&, unsigned char*, int64_t*);                 \
    template cudaError_t launch_kslice_bounds<IT>(const spgemm_csr&, int, int64_t*, int,       \
                                                  cudaStream_t);                               \
    template cudaError_t prepare_numeric<IT, double>(Plan&);                                   \
    template cudaError_t prepare_numeric<IT, float>(Plan&);                                    \
    template cudaError_t prepare_numeric<IT, int64_t>(Plan&);                                  \
    template cudaError_t prepare_numeric<IT, NoVal>(Plan&);                                    \
    template cudaError_t launch_numeric<IT, double>(Plan&, unsigned char*, const int64_t*,     \
                                                    long long, void*, void*, int64_t*,         \
                                                    int32_t*, unsigned*);                      \
    template cudaError_t launch_numeric<IT, float>(Plan&, unsigned char*, const int64_t*,      \
                                                   long long, void*, void*, int64_t*,          \
                                                   int32_t*, unsigned*);                       \
    template cudaError_t launch_numeric<IT, int64_t>(Plan&, unsigned char*, const int64_t*,    \
                                                     long long, void*, void*, int64_t*,        \
                                                     int32_t*, unsigned*);                     \
    template cudaError_t launch_numeric<IT, NoVal>(Plan&, unsigned char*, const int64_t*,      \
                                                   long long, void*, void*, int64_t*,          \
                                                   int32_t*, unsigned*);                       \
    template cudaError_t launch_row_features<IT>(Plan&, float*);

// The numeric launchers of one value type (used for the min semirings, which
// are instantiated in their own translation units so they compile in
// parallel with the others).
#define SG_INSTANTIATE_IT_V(IT, V)                                                              \
    template cudaError_t prepare_numeric<IT, V>(Plan&);                                        \
    template cudaError_t launch_numeric<IT, V>(Plan&, unsigned char*, const int64_t*,          \
                                               long long, void*, void*, int64_t*, int32_t*,    \
                                               unsigned*);                                     \
    template cudaError_t launch_dense_slot_pack<IT, V>(Plan&, const int64_t*, void*, void*,    \
                                                       int64_t*);

}  // namespace sg
