// Template host launchers; included by the per-index-type instantiation units.
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

template <class IT, class V, int W, int WARPS>
cudaError_t launch_numeric_dense(Plan& P, unsigned char* ws, const int64_t* rpC, IT* colC, V* valC);

template <class IT>
cudaError_t launch_analyze(Plan& P) {
    if (P.m <= 0) return cudaSuccess;
    auto k = analyze_kernel<IT>;
    int occ = occupancy_blocks(k, 256, 0);
    long long g = grid_for(P.m, 8, P.sm_count, occ);
    count_launches(1);
    k<<<(unsigned)g, 256, 0, P.stream>>>(P.m, P.n, P.max_dense_n, P.A.rowptr, P.A.rowend,
                                           (const IT*)P.A.col, P.B.rowptr, P.flops, P.cnt);
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
    if (nrows == 0) return cudaSuccess;
    auto k = symbolic_hash_kernel<IT, LOG2T, WARPS>;
    size_t smem = (size_t)WARPS * (1u << LOG2T) * sizeof(K);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    int occ = occupancy_blocks(k, WARPS * 32, smem);
    long long g = grid_for(nrows, WARPS, P.sm_count, occ);
    count_launches(1);
    k<<<(unsigned)g, WARPS * 32, smem, P.stream>>>(
        P.rows + P.class_off[c], nrows, P.A.rowptr, P.A.rowend, (const IT*)P.A.col, P.B.rowptr,
        (const IT*)P.B.col, rowcnt, &P.cnt->err);
    return cudaGetLastError();
}

template <class IT>
cudaError_t launch_symbolic(Plan& P, unsigned char* ws, int64_t* rowcnt) {
    WsLayout L = workspace_layout(P);
    cudaError_t e = launch_zero_rows(P.rows + P.class_off[kClassEmpty],
                                     (long long)P.class_count[kClassEmpty], rowcnt, P.sm_count,
                                     P.stream);
    if (e != cudaSuccess) return e;
    if ((e = sym_hash_bin<IT, 6, 8>(P, 0, rowcnt)) != cudaSuccess) return e;
    if ((e = sym_hash_bin<IT, 8, 8>(P, 1, rowcnt)) != cudaSuccess) return e;
    if ((e = sym_hash_bin<IT, 10, 8>(P, 2, rowcnt)) != cudaSuccess) return e;
    if ((e = sym_hash_bin<IT, 11, 8>(P, 3, rowcnt)) != cudaSuccess) return e;
    if (P.ndense > 0 && P.l > 0) {
        long long total = P.l * (kSegGrid + 1);
        long long g = grid_for(total, 256, P.sm_count, 8);
        count_launches(1);
        segtab_kernel<IT><<<(unsigned)g, 256, 0, P.stream>>>(P.l, P.B.rowptr, (const IT*)P.B.col,
                                                             P.W, P.P, (int32_t*)(ws + L.segtab));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        long long g2 = grid_for(P.l, 8, P.sm_count, 8);
        count_launches(1);
        runlen_kernel<IT><<<(unsigned)g2, 256, 0, P.stream>>>(P.l, P.B.rowptr, (const IT*)P.B.col,
                                                              P.W, (int32_t*)(ws + L.runlen));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (P.ndense > 0) {
        auto k = symbolic_dense_kernel<IT>;
        const int threads = 512;
        size_t smem = (size_t)((P.n + 31) / 32) * 4;
        if ((e = allow_smem(k, smem)) != cudaSuccess) return e;
        int occ = occupancy_blocks(k, threads, smem);
        long long g = grid_for(P.ndense, 1, P.sm_count, occ);
        unsigned long long* work = &P.cnt->work_counter[0];
        if ((e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), P.stream)) != cudaSuccess)
            return e;
        count_launches(1);
        k<<<(unsigned)g, threads, smem, P.stream>>>(
            P.rows + P.class_off[kClassDense0], P.ndense, P.A.rowptr, P.A.rowend,
            (const IT*)P.A.col, P.B.rowptr, (const IT*)P.B.col, P.n, P.W / 32, P.P,
            (int32_t*)(ws + L.chunkcnt), rowcnt, work);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class IT, class V, int LOG2T, int WARPS>
cudaError_t num_hash_bin(Plan& P, int bin, const int64_t* rpC, IT* colC, V* valC) {
    using K = typename KeyT<IT>::type;
    const int c = kClassHash0 + bin;
    const long long nrows = (long long)P.class_count[c];
    if (nrows == 0) return cudaSuccess;
    auto k = numeric_hash_kernel<IT, V, LOG2T, WARPS>;
    constexpr size_t vb = VOps<V>::has_val ? sizeof(V) : 0;
    size_t smem = (size_t)WARPS * (1u << LOG2T) * (sizeof(K) + vb);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    int occ = occupancy_blocks(k, WARPS * 32, smem);
    long long g = grid_for(nrows, WARPS, P.sm_count, occ);
    count_launches(1);
    k<<<(unsigned)g, WARPS * 32, smem, P.stream>>>(
        P.rows + P.class_off[c], nrows, P.A.rowptr, P.A.rowend, (const IT*)P.A.col,
        (const V*)P.A.val, P.B.rowptr, (const IT*)P.B.col, (const V*)P.B.val, rpC, colC, valC,
        &P.cnt->err);
    return cudaGetLastError();
}

template <class IT, class V>
cudaError_t launch_numeric(Plan& P, unsigned char* ws, const int64_t* rpC, void* colC_,
                           void* valC_) {
    IT* colC = (IT*)colC_;
    V* valC = (V*)valC_;
    cudaError_t e;
    if ((e = num_hash_bin<IT, V, 6, 8>(P, 0, rpC, colC, valC)) != cudaSuccess) return e;
    if ((e = num_hash_bin<IT, V, 8, 8>(P, 1, rpC, colC, valC)) != cudaSuccess) return e;
    if ((e = num_hash_bin<IT, V, 10, 8>(P, 2, rpC, colC, valC)) != cudaSuccess) return e;
    if ((e = num_hash_bin<IT, V, 11, 4>(P, 3, rpC, colC, valC)) != cudaSuccess) return e;
    if (P.ndense > 0) {
        e = P.W == kDenseW0 ? launch_numeric_dense<IT, V, kDenseW0, kDenseWarps0>(P, ws, rpC, colC, valC)
                            : launch_numeric_dense<IT, V, kDenseW1, kDenseWarps1>(P, ws, rpC, colC, valC);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class IT, class V, int W, int WARPS>
cudaError_t launch_numeric_dense(Plan& P, unsigned char* ws, const int64_t* rpC, IT* colC, V* valC) {
    WsLayout L = workspace_layout(P);
    auto k = numeric_dense_kernel<IT, V, W, WARPS>;
    constexpr size_t vb = VOps<V>::has_val ? sizeof(V) : 0;
    size_t smem = (size_t)WARPS * (W * vb + W / 8);
    cudaError_t e;
    if ((e = allow_smem(k, smem)) != cudaSuccess) return e;
    unsigned long long* work = &P.cnt->work_counter[1];
    if ((e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), P.stream)) != cudaSuccess)
        return e;
    count_launches(1);
    k<<<(unsigned)P.dense_grid, WARPS * 32, smem, P.stream>>>(
        P.rows + P.class_off[kClassDense0], P.units, P.A.rowptr, P.A.rowend,
        (const IT*)P.A.col, (const V*)P.A.val, P.B.rowptr, (const IT*)P.B.col,
        (const V*)P.B.val, P.n, P.P, (const int32_t*)(ws + L.chunkcnt),
        (const int32_t*)(ws + L.segtab), (const int32_t*)(ws + L.runlen),
        (DenseCursor*)(ws + L.arena), L.arena_stride, rpC, colC, valC, work, &P.cnt->err);
    return cudaGetLastError();
}

template <class IT, class V, int W, int WARPS>
cudaError_t prepare_numeric_dense(Plan& P) {
    auto k = numeric_dense_kernel<IT, V, W, WARPS>;
    constexpr size_t vb = VOps<V>::has_val ? sizeof(V) : 0;
    size_t smem = (size_t)WARPS * (W * vb + W / 8);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    int occ = occupancy_blocks(k, WARPS * 32, smem);
    long long units = P.units.unit_begin[P.units.nclass];
    P.dense_warps_per_block = WARPS;
    P.dense_grid = grid_for(std::max<long long>(units, 1), WARPS, P.sm_count, occ);
    return cudaSuccess;
}

// Grid of the dense numeric kernel (one resident wave; units are grabbed
// dynamically), fixed at plan time so the workspace can size the cursor arena.
template <class IT, class V>
cudaError_t prepare_numeric(Plan& P) {
    return P.W == kDenseW0 ? prepare_numeric_dense<IT, V, kDenseW0, kDenseWarps0>(P)
                           : prepare_numeric_dense<IT, V, kDenseW1, kDenseWarps1>(P);
}

#define SG_INSTANTIATE_IT(IT)                                                                   \
    template cudaError_t launch_analyze<IT>(Plan&);                                            \
    template cudaError_t launch_validate<IT>(const spgemm_csr&, int*, int, cudaStream_t);      \
    template cudaError_t launch_symbolic<IT>(Plan&, unsigned char*, int64_t*);                 \
    template cudaError_t launch_kslice_bounds<IT>(const spgemm_csr&, int, int64_t*, int,       \
                                                  cudaStream_t);                               \
    template cudaError_t prepare_numeric<IT, double>(Plan&);                                   \
    template cudaError_t prepare_numeric<IT, float>(Plan&);                                    \
    template cudaError_t prepare_numeric<IT, int64_t>(Plan&);                                  \
    template cudaError_t prepare_numeric<IT, NoVal>(Plan&);                                    \
    template cudaError_t launch_numeric<IT, double>(Plan&, unsigned char*, const int64_t*,     \
                                                    void*, void*);                             \
    template cudaError_t launch_numeric<IT, float>(Plan&, unsigned char*, const int64_t*,      \
                                                   void*, void*);                              \
    template cudaError_t launch_numeric<IT, int64_t>(Plan&, unsigned char*, const int64_t*,    \
                                                     void*, void*);                            \
    template cudaError_t launch_numeric<IT, NoVal>(Plan&, unsigned char*, const int64_t*,      \
                                                   void*, void*);

}  // namespace sg
