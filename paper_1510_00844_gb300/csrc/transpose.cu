// CSR transpose: A (m x n) -> A^T (n x m), rows of A^T with ascending column
// (= original row) indices.  The paper transposes the B blocks locally during
// redistribution (Alg. 2, the all-to-all of B); here it supplies R^T for the
// Galerkin product R^T A R.
//
// Steps: column counts (atomic histogram) -> exclusive scan = row pointers of
// A^T -> scatter of (row, value) with per-column atomic cursors (arbitrary
// order inside a row) -> per-row sort by the original row index: one warp
// per row up to 1024 entries (bitonic in shared memory), one block per row up
// to 8192, and a rank count (each entry counts the smaller row indices of its
// row) for longer rows.  Original row indices are unique within a row of A^T,
// so the sorted order is unique.
#include <cstdio>

#include "plan.h"

namespace sg {

template <class IT>
__global__ void col_count_kernel(long long m, const int64_t* __restrict__ rp,
                                 const IT* __restrict__ ci, unsigned long long* __restrict__ cnt) {
    const int lane = lane_id();
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < m; i += nwarps)
        for (long long p = rp[i] + lane; p < rp[i + 1]; p += 32)
            atomicAdd(&cnt[(long long)ci[p]], 1ull);
}

template <class IT, class V>
__global__ void scatter_kernel(long long m, const int64_t* __restrict__ rp,
                               const IT* __restrict__ ci, const V* __restrict__ va,
                               const int64_t* __restrict__ rpT,
                               unsigned long long* __restrict__ cursor, IT* __restrict__ ciT,
                               V* __restrict__ vaT) {
    const int lane = lane_id();
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < m; i += nwarps)
        for (long long p = rp[i] + lane; p < rp[i + 1]; p += 32) {
            const long long j = (long long)ci[p];
            const long long pos = rpT[j] + (long long)atomicAdd(&cursor[j], 1ull);
            ciT[pos] = (IT)i;
            if constexpr (VOps<V>::has_val) vaT[pos] = va[p];
        }
}

// Sorts rows of A^T with length in (lo, hi]; WARP_ROWS: one warp per row
// (hi <= 1024), which also lists the longer rows; else one block per listed
// row (hi <= 8192).  Keys are unique.
template <class IT, class V, bool WARP_ROWS, int CAP>
__global__ void sort_rows_kernel(long long n, const int64_t* __restrict__ rpT, int lo, int hi,
                                 IT* __restrict__ ciT, V* __restrict__ vaT,
                                 long long* __restrict__ long_rows, unsigned* long_count) {
    constexpr bool HV = VOps<V>::has_val;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const int w = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int slots = WARP_ROWS ? nwarps : 1;
    const int unit = WARP_ROWS ? w : 0;
    long long* keys = reinterpret_cast<long long*>(smem_raw) + (size_t)unit * CAP;
    V* vals = reinterpret_cast<V*>(smem_raw + (size_t)slots * CAP * sizeof(long long)) +
              (size_t)unit * CAP;
    const long long first = WARP_ROWS ? ((long long)blockIdx.x * nwarps + w) : blockIdx.x;
    const long long step = WARP_ROWS ? (long long)gridDim.x * nwarps : gridDim.x;
    const int t0 = WARP_ROWS ? lane : threadIdx.x;
    const int tstep = WARP_ROWS ? 32 : blockDim.x;
    const long long nitems = WARP_ROWS ? n : (long long)*long_count;
    for (long long it = first; it < nitems; it += step) {
        const long long j = WARP_ROWS ? it : long_rows[it];
        const long long a = rpT[j];
        const int L = (int)(rpT[j + 1] - a);
        if (L > hi && WARP_ROWS && long_rows) {   // handed to the block pass
            if (lane == 0) long_rows[atomicAdd(long_count, 1u)] = j;
            continue;
        }
        if (L <= lo || L > hi) continue;
        int N = 1;
        while (N < L) N <<= 1;
        for (int t = t0; t < N; t += tstep) {
            keys[t] = t < L ? (long long)ciT[a + t] : 0x7fffffffffffffffLL;
            if constexpr (HV)
                if (t < L) vals[t] = vaT[a + t];
        }
        if (WARP_ROWS) __syncwarp(); else __syncthreads();
        for (int k = 2; k <= N; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = t0; i < N; i += tstep) {
                    const int ixj = i ^ jj;
                    if (ixj > i) {
                        const long long ki = keys[i], kj = keys[ixj];
                        const bool up = (i & k) == 0;
                        if ((ki > kj) == up) {
                            keys[i] = kj;
                            keys[ixj] = ki;
                            if constexpr (HV) {
                                V tv = vals[i];
                                vals[i] = vals[ixj];
                                vals[ixj] = tv;
                            }
                        }
                    }
                }
                if (WARP_ROWS) __syncwarp(); else __syncthreads();
            }
        }
        for (int t = t0; t < L; t += tstep) {
            ciT[a + t] = (IT)keys[t];
            if constexpr (HV) vaT[a + t] = vals[t];
        }
        if (WARP_ROWS) __syncwarp(); else __syncthreads();
    }
}

// Rows longer than 8192: each entry's position is the number of smaller keys
// in its row (keys are unique); results go to a scratch copy, then back.
template <class IT, class V>
__global__ void rank_rows_kernel(const long long* __restrict__ long_rows,
                                 const unsigned* long_count, const int64_t* __restrict__ rpT,
                                 int lo, const IT* __restrict__ ciT, const V* __restrict__ vaT,
                                 IT* __restrict__ ciS, V* __restrict__ vaS) {
    const long long nitems = (long long)*long_count;
    for (long long it = blockIdx.x; it < nitems; it += gridDim.x) {
        const long long j = long_rows[it];
        const long long a = rpT[j];
        const long long L = rpT[j + 1] - a;
        if (L <= lo) continue;
        for (long long t = threadIdx.x; t < L; t += blockDim.x) {
            const long long key = (long long)ciT[a + t];
            long long rank = 0;
            for (long long u = 0; u < L; ++u) rank += (long long)ciT[a + u] < key;
            ciS[a + rank] = (IT)key;
            if constexpr (VOps<V>::has_val) vaS[a + rank] = vaT[a + t];
        }
    }
}

template <class IT, class V>
__global__ void copy_back_kernel(const long long* __restrict__ long_rows,
                                 const unsigned* long_count, const int64_t* __restrict__ rpT,
                                 int lo, const IT* __restrict__ ciS, const V* __restrict__ vaS,
                                 IT* __restrict__ ciT, V* __restrict__ vaT) {
    const long long nitems = (long long)*long_count;
    for (long long it = blockIdx.x; it < nitems; it += gridDim.x) {
        const long long j = long_rows[it];
        const long long a = rpT[j];
        const long long L = rpT[j + 1] - a;
        if (L <= lo) continue;
        for (long long t = threadIdx.x; t < L; t += blockDim.x) {
            ciT[a + t] = ciS[a + t];
            if constexpr (VOps<V>::has_val) vaT[a + t] = vaS[a + t];
        }
    }
}

template <class IT, class V>
cudaError_t launch_transpose(const spgemm_csr& A, cudaStream_t s, unsigned char* ws,
                             int64_t* rpT, void* ciT_, void* vaT_) {
    const long long m = A.nrows, n = A.ncols, nnz = A.nnz;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    IT* ciT = (IT*)ciT_;
    V* vaT = (V*)vaT_;
    unsigned long long* cursor = (unsigned long long*)ws;
    int64_t* temp = (int64_t*)(ws + ((size_t)(n + 1) * 8 + 255) / 256 * 256);
    const size_t isz = sizeof(IT), vsz = VOps<V>::has_val ? sizeof(V) : 0;
    unsigned char* after_scratch = ws + ((size_t)(n + 1) * 8 + 255) / 256 * 256 +
                                   (scan_temp_bytes(n + 1) + 255) / 256 * 256 +
                                   ((size_t)nnz * isz + 255) / 256 * 256 +
                                   ((size_t)nnz * vsz + 255) / 256 * 256;
    unsigned* long_count = (unsigned*)after_scratch;
    long long* long_rows = (long long*)(after_scratch + 256);
    cudaError_t e;
    if ((e = cudaMemsetAsync(rpT, 0, (size_t)(n + 1) * sizeof(int64_t), s)) != cudaSuccess) return e;
    auto blocks = [&](long long items, int per) {
        return (unsigned)std::max<long long>(1, std::min<long long>((items + per - 1) / per, (long long)sms * 8));
    };
    if (m > 0) {
        count_launches(1);
        col_count_kernel<IT><<<blocks(m, 8), 256, 0, s>>>(m, A.rowptr, (const IT*)A.col,
                                                         (unsigned long long*)rpT);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = launch_exclusive_scan(rpT, n + 1, temp, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cursor, 0, (size_t)(n + 1) * 8, s)) != cudaSuccess) return e;
    if (m > 0) {
        count_launches(1);
        scatter_kernel<IT, V><<<blocks(m, 8), 256, 0, s>>>(m, A.rowptr, (const IT*)A.col,
                                                          (const V*)A.val, rpT, cursor, ciT, vaT);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (n <= 0 || nnz <= 0) return cudaSuccess;
    if ((e = cudaMemsetAsync(long_count, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    constexpr size_t vb = VOps<V>::has_val ? sizeof(V) : 0;
    {
        auto k = sort_rows_kernel<IT, V, true, 1024>;
        const size_t smem = 4 * 1024 * (8 + vb);
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        count_launches(1);
        k<<<blocks(n, 4), 128, smem, s>>>(n, rpT, 1, 1024, ciT, vaT, long_rows, long_count);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        auto k = sort_rows_kernel<IT, V, false, 8192>;
        const size_t smem = 8192 * (8 + vb);
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        count_launches(1);
        k<<<(unsigned)std::min<long long>(n, (long long)sms * 2), 512, smem, s>>>(
            n, rpT, 1024, 8192, ciT, vaT, long_rows, long_count);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        IT* ciS = (IT*)(ws + ((size_t)(n + 1) * 8 + 255) / 256 * 256 +
                        (scan_temp_bytes(n + 1) + 255) / 256 * 256);
        V* vaS = (V*)((unsigned char*)ciS + ((size_t)nnz * sizeof(IT) + 255) / 256 * 256);
        const unsigned g = (unsigned)std::min<long long>(n, (long long)sms * 4);
        count_launches(2);
        rank_rows_kernel<IT, V><<<g, 256, 0, s>>>(long_rows, long_count, rpT, 8192, ciT, vaT, ciS, vaS);
        copy_back_kernel<IT, V><<<g, 256, 0, s>>>(long_rows, long_count, rpT, 8192, ciS, vaS, ciT, vaT);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sg

extern "C" {

size_t spgemm_transpose_workspace_size(const spgemm_csr* A) {
    if (!A) return 0;
    const size_t n = (size_t)std::max<long long>(0, A->ncols);
    const size_t nnz = (size_t)std::max<long long>(0, A->nnz);
    const size_t isz = A->index_type == SPGEMM_INDEX_I32 ? 4 : 8;
    const size_t vsz = A->value_type == SPGEMM_F32 ? 4 : A->value_type == SPGEMM_BOOL ? 0 : 8;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    return al((n + 1) * 8) + al(sg::scan_temp_bytes((long long)n + 1)) + al(nnz * isz) +
           al(nnz * vsz) + 256 + al((n + 1) * 8);
}

spgemm_status spgemm_transpose(const spgemm_csr* A, void* stream, void* ws, size_t ws_bytes,
                               int64_t* rowptrT, void* colT, void* valT) {
    sg::set_last_error("");
    if (!A || !rowptrT || (A->nnz > 0 && !colT)) {
        sg::set_last_error("NULL argument");
        return SPGEMM_ERR_INVALID_ARG;
    }
    if (A->rowend || A->nrows < 0 || A->ncols < 0 || A->nnz < 0 || !A->rowptr ||
        (A->nnz > 0 && !A->col)) {
        sg::set_last_error("A must be a plain CSR with non-negative sizes");
        return SPGEMM_ERR_INVALID_ARG;
    }
    const bool has_val = A->value_type != SPGEMM_BOOL;
    if (has_val && A->nnz > 0 && (!A->val || !valT)) {
        sg::set_last_error("values are NULL");
        return SPGEMM_ERR_INVALID_ARG;
    }
    if (A->index_type == SPGEMM_INDEX_I32 && A->nrows > 0x7fffffffLL) {
        sg::set_last_error("rows of A exceed int32 column indices of A^T");
        return SPGEMM_ERR_INDEX_OVERFLOW;
    }
    if (!ws || ws_bytes < spgemm_transpose_workspace_size(A) || ((uintptr_t)ws) % 256) {
        sg::set_last_error("transpose workspace missing, too small or not 256-byte aligned");
        return SPGEMM_ERR_OUT_OF_MEMORY;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* w = (unsigned char*)ws;
    const bool i32 = A->index_type == SPGEMM_INDEX_I32;
    cudaError_t e;
    switch (A->value_type) {
        case SPGEMM_F64:
            e = i32 ? sg::launch_transpose<int32_t, double>(*A, s, w, rowptrT, colT, valT)
                    : sg::launch_transpose<int64_t, double>(*A, s, w, rowptrT, colT, valT);
            break;
        case SPGEMM_F32:
            e = i32 ? sg::launch_transpose<int32_t, float>(*A, s, w, rowptrT, colT, valT)
                    : sg::launch_transpose<int64_t, float>(*A, s, w, rowptrT, colT, valT);
            break;
        case SPGEMM_I64:
            e = i32 ? sg::launch_transpose<int32_t, int64_t>(*A, s, w, rowptrT, colT, valT)
                    : sg::launch_transpose<int64_t, int64_t>(*A, s, w, rowptrT, colT, valT);
            break;
        default:
            e = i32 ? sg::launch_transpose<int32_t, sg::NoVal>(*A, s, w, rowptrT, colT, nullptr)
                    : sg::launch_transpose<int64_t, sg::NoVal>(*A, s, w, rowptrT, colT, nullptr);
            break;
    }
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "transpose: CUDA error %d (%s)", (int)e, cudaGetErrorString(e));
        sg::set_last_error(buf);
        return SPGEMM_ERR_CUDA;
    }
    return SPGEMM_OK;
}

}  // extern "C"
