// Masked product (the structural mask that MIS-2 aggregation applies to its
// semiring products, Alg. 3): keep the entries of C whose (i, j) is in the
// pattern of M (complement = 0) or not in it (complement = 1).  The mask is
// applied to the rows of the finished product: one warp per row looks every
// column of C(i,:) up in the sorted row M(i,:) by binary search; pass 1
// counts the kept entries, a scan gives the row pointers, pass 2 copies them
// in order.  The product's own work is not reduced by the mask.
#include <cstdio>

#include "plan.h"

namespace sg {

// Is column j in the sorted range cm[lo, hi)?
template <class IT>
__device__ __forceinline__ bool in_row(const IT* __restrict__ cm, long long lo, long long hi,
                                       long long j) {
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        const long long c = (long long)cm[mid];
        if (c == j) return true;
        if (c < j) lo = mid + 1;
        else hi = mid;
    }
    return false;
}

template <class IT>
__global__ void mask_count_kernel(long long m, const int64_t* __restrict__ rp,
                                  const int64_t* __restrict__ re, const IT* __restrict__ col,
                                  const int64_t* __restrict__ mrp, const int64_t* __restrict__ mre,
                                  const IT* __restrict__ mcol, int complement,
                                  int64_t* __restrict__ cnt) {
    const int lane = lane_id();
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < m; i += nwarps) {
        const long long a = rp[i], b = re ? re[i] : rp[i + 1];
        const long long ma = mrp[i], mb = mre ? mre[i] : mrp[i + 1];
        long long c = 0;
        for (long long q = a + lane; q < b; q += 32)
            c += in_row(mcol, ma, mb, (long long)col[q]) != (complement != 0);
        c = warp_sum(c);
        if (lane == 0) cnt[i] = c;
    }
}

template <class IT, class V>
__global__ void mask_fill_kernel(long long m, const int64_t* __restrict__ rp,
                                 const int64_t* __restrict__ re, const IT* __restrict__ col,
                                 const V* __restrict__ val, const int64_t* __restrict__ mrp,
                                 const int64_t* __restrict__ mre, const IT* __restrict__ mcol,
                                 int complement, const int64_t* __restrict__ rpo,
                                 IT* __restrict__ colo, V* __restrict__ valo) {
    constexpr bool HV = VOps<V>::has_val;
    const int lane = lane_id();
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < m; i += nwarps) {
        const long long a = rp[i], b = re ? re[i] : rp[i + 1];
        const long long ma = mrp[i], mb = mre ? mre[i] : mrp[i + 1];
        long long out = rpo[i];
        for (long long q0 = a; q0 < b; q0 += 32) {
            const long long q = q0 + lane;
            const bool keep =
                q < b && (in_row(mcol, ma, mb, (long long)col[q]) != (complement != 0));
            const unsigned msk = __ballot_sync(kFull, keep);
            if (keep) {
                const long long pos = out + __popc(msk & lanemask_lt());
                colo[pos] = col[q];
                if constexpr (HV) valo[pos] = val[q];
            }
            out += __popc(msk);
        }
    }
}

}  // namespace sg

namespace {

spgemm_status kfail(spgemm_status st, const char* msg) {
    sg::set_last_error(msg);
    return st;
}

spgemm_status kcheck(const spgemm_csr* C, const spgemm_csr* M) {
    if (!C || !M || !C->rowptr || !M->rowptr || C->nrows < 0 ||
        (C->nnz > 0 && !C->col) || (M->nnz > 0 && !M->col))
        return kfail(SPGEMM_ERR_INVALID_ARG, "mask: NULL or malformed matrix");
    if (M->nrows != C->nrows || M->ncols != C->ncols)
        return kfail(SPGEMM_ERR_INVALID_ARG, "mask: M and C differ in shape");
    if (M->index_type != C->index_type)
        return kfail(SPGEMM_ERR_INVALID_ARG, "mask: M and C differ in index type");
    if (C->value_type != SPGEMM_BOOL && C->nnz > 0 && !C->val)
        return kfail(SPGEMM_ERR_INVALID_ARG, "mask: C has no values");
    return SPGEMM_OK;
}

unsigned grid_rows(long long m) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (unsigned)std::max<long long>(1, std::min<long long>((m + 7) / 8, (long long)sms * 8));
}

}  // namespace

extern "C" {

size_t spgemm_mask_workspace_size(int64_t m) {
    if (m < 0) m = 0;
    return sg::scan_temp_bytes(m + 1);
}

spgemm_status spgemm_mask_count(const spgemm_csr* C, const spgemm_csr* M, int32_t complement,
                                void* stream, void* ws, size_t ws_bytes, int64_t* rowptrP,
                                int64_t* nnz_host) {
    sg::set_last_error("");
    spgemm_status st = kcheck(C, M);
    if (st != SPGEMM_OK) return st;
    const long long m = C->nrows;
    if (!rowptrP || !nnz_host || !ws || ws_bytes < spgemm_mask_workspace_size(m))
        return kfail(SPGEMM_ERR_INVALID_ARG, "mask: outputs or workspace missing");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(rowptrP + m, 0, 8, s);
    if (e == cudaSuccess && m > 0) {
        sg::count_launches(1);
        if (C->index_type == SPGEMM_INDEX_I32)
            sg::mask_count_kernel<int32_t><<<grid_rows(m), 256, 0, s>>>(
                m, C->rowptr, C->rowend, (const int32_t*)C->col, M->rowptr, M->rowend,
                (const int32_t*)M->col, complement, rowptrP);
        else
            sg::mask_count_kernel<int64_t><<<grid_rows(m), 256, 0, s>>>(
                m, C->rowptr, C->rowend, (const int64_t*)C->col, M->rowptr, M->rowend,
                (const int64_t*)M->col, complement, rowptrP);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = sg::launch_exclusive_scan(rowptrP, m + 1, (int64_t*)ws, s);
    int64_t total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, rowptrP + m, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return kfail(SPGEMM_ERR_CUDA, cudaGetErrorString(e));
    *nnz_host = total;
    return SPGEMM_OK;
}

spgemm_status spgemm_mask_fill(const spgemm_csr* C, const spgemm_csr* M, int32_t complement,
                               void* stream, const int64_t* rowptrP, void* colP, void* valP) {
    sg::set_last_error("");
    spgemm_status st = kcheck(C, M);
    if (st != SPGEMM_OK) return st;
    const long long m = C->nrows;
    if (!rowptrP) return kfail(SPGEMM_ERR_INVALID_ARG, "mask: rowptrP is NULL");
    if (m == 0) return SPGEMM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int vt = C->value_type;
    const bool i32 = C->index_type == SPGEMM_INDEX_I32;
    cudaError_t e = sg::with_value_type(vt, [&](auto tag) -> cudaError_t {
        using V = decltype(tag);
        sg::count_launches(1);
        if (i32)
            sg::mask_fill_kernel<int32_t, V><<<grid_rows(m), 256, 0, s>>>(
                m, C->rowptr, C->rowend, (const int32_t*)C->col, (const V*)C->val, M->rowptr,
                M->rowend, (const int32_t*)M->col, complement, rowptrP, (int32_t*)colP, (V*)valP);
        else
            sg::mask_fill_kernel<int64_t, V><<<grid_rows(m), 256, 0, s>>>(
                m, C->rowptr, C->rowend, (const int64_t*)C->col, (const V*)C->val, M->rowptr,
                M->rowend, (const int64_t*)M->col, complement, rowptrP, (int64_t*)colP, (V*)valP);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return kfail(SPGEMM_ERR_CUDA, cudaGetErrorString(e));
    return SPGEMM_OK;
}

}  // extern "C"
