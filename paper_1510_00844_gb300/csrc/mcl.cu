// Markov-clustering epilogue on the expansion product (the paper squares
// matrices to represent MCL expansion, Sec. 5.3): on M^T stored in CSR (rows
// of M^T are the columns of M), drop every entry below `threshold` and divide
// each row by the sum of its kept entries, so M stays column-stochastic.
// Input may be a view (rowend); output is a plain CSR of float64 values.
// Pass 1 (one warp per row): kept count and kept sum; scan; pass 2: the kept
// entries, in order, divided by the row sum.  The sum of a row is a warp
// reduction over its kept entries in a fixed order, so results repeat
// exactly from run to run.
#include <cstdio>

#include "plan.h"

namespace sg {

template <class IT>
__global__ void mcl_count_kernel(long long m, const int64_t* __restrict__ rp,
                                 const int64_t* __restrict__ re, const double* __restrict__ val,
                                 double thr, int64_t* __restrict__ cnt, double* __restrict__ sums) {
    const int lane = lane_id();
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < m; i += nwarps) {
        const long long a = rp[i], b = re ? re[i] : rp[i + 1];
        long long c = 0;
        double s = 0.0;
        for (long long q = a + lane; q < b; q += 32) {
            const double v = val[q];
            if (v >= thr) {
                ++c;
                s = __dadd_rn(s, v);
            }
        }
        c = warp_sum(c);
#pragma unroll
        for (int d = 16; d; d >>= 1) s = __dadd_rn(s, __shfl_xor_sync(kFull, s, d));
        if (lane == 0) {
            cnt[i] = c;
            sums[i] = s;
        }
    }
}

template <class IT>
__global__ void mcl_fill_kernel(long long m, const int64_t* __restrict__ rp,
                                const int64_t* __restrict__ re, const IT* __restrict__ col,
                                const double* __restrict__ val, double thr,
                                const double* __restrict__ sums, const int64_t* __restrict__ rpo,
                                IT* __restrict__ colo, double* __restrict__ valo) {
    const int lane = lane_id();
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < m; i += nwarps) {
        const long long a = rp[i], b = re ? re[i] : rp[i + 1];
        long long out = rpo[i];
        const double s = sums[i];
        for (long long q0 = a; q0 < b; q0 += 32) {
            const long long q = q0 + lane;
            const bool keep = q < b && val[q] >= thr;
            const unsigned msk = __ballot_sync(kFull, keep);
            if (keep) {
                const long long pos = out + __popc(msk & lanemask_lt());
                colo[pos] = col[q];
                valo[pos] = __ddiv_rn(val[q], s);
            }
            out += __popc(msk);
        }
    }
}

}  // namespace sg

namespace {

spgemm_status mfail(spgemm_status st, const char* msg) {
    sg::set_last_error(msg);
    return st;
}

spgemm_status mcheck(const spgemm_csr* C) {
    if (!C || !C->rowptr || C->nrows < 0 || (C->nnz > 0 && (!C->col || !C->val)))
        return mfail(SPGEMM_ERR_INVALID_ARG, "mcl: NULL or malformed matrix");
    if (C->value_type != SPGEMM_F64) return mfail(SPGEMM_ERR_NOT_SUPPORTED, "mcl: float64 values only");
    return SPGEMM_OK;
}

size_t al(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" {

size_t spgemm_mcl_workspace_size(int64_t m) {
    if (m < 0) m = 0;
    return al((size_t)m * 8) + al(sg::scan_temp_bytes(m + 1));
}

spgemm_status spgemm_mcl_prune_count(const spgemm_csr* C, double threshold, void* stream,
                                     void* ws, size_t ws_bytes, int64_t* rowptrP,
                                     int64_t* nnz_host) {
    sg::set_last_error("");
    spgemm_status st = mcheck(C);
    if (st != SPGEMM_OK) return st;
    const long long m = C->nrows;
    if (!rowptrP || !nnz_host || !ws || ws_bytes < spgemm_mcl_workspace_size(m))
        return mfail(SPGEMM_ERR_INVALID_ARG, "mcl: outputs or workspace missing");
    cudaStream_t s = (cudaStream_t)stream;
    double* sums = (double*)ws;
    int64_t* temp = (int64_t*)((unsigned char*)ws + al((size_t)m * 8));
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMemsetAsync(rowptrP + m, 0, 8, s);
    if (e == cudaSuccess && m > 0) {
        const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>((m + 7) / 8, (long long)sms * 8));
        sg::count_launches(1);
        if (C->index_type == SPGEMM_INDEX_I32)
            sg::mcl_count_kernel<int32_t><<<g, 256, 0, s>>>(m, C->rowptr, C->rowend, (const double*)C->val,
                                                            threshold, rowptrP, sums);
        else
            sg::mcl_count_kernel<int64_t><<<g, 256, 0, s>>>(m, C->rowptr, C->rowend, (const double*)C->val,
                                                            threshold, rowptrP, sums);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = sg::launch_exclusive_scan(rowptrP, m + 1, temp, s);
    int64_t total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, rowptrP + m, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return mfail(SPGEMM_ERR_CUDA, cudaGetErrorString(e));
    *nnz_host = total;
    return SPGEMM_OK;
}

spgemm_status spgemm_mcl_prune_fill(const spgemm_csr* C, double threshold, void* stream, void* ws,
                                    size_t ws_bytes, const int64_t* rowptrP, void* colP,
                                    double* valP) {
    sg::set_last_error("");
    spgemm_status st = mcheck(C);
    if (st != SPGEMM_OK) return st;
    const long long m = C->nrows;
    if (!rowptrP || !ws || ws_bytes < spgemm_mcl_workspace_size(m))
        return mfail(SPGEMM_ERR_INVALID_ARG, "mcl: outputs or workspace missing");
    if (m == 0) return SPGEMM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>((m + 7) / 8, (long long)sms * 8));
    sg::count_launches(1);
    if (C->index_type == SPGEMM_INDEX_I32)
        sg::mcl_fill_kernel<int32_t><<<g, 256, 0, s>>>(m, C->rowptr, C->rowend, (const int32_t*)C->col,
                                                       (const double*)C->val, threshold, (const double*)ws,
                                                       rowptrP, (int32_t*)colP, valP);
    else
        sg::mcl_fill_kernel<int64_t><<<g, 256, 0, s>>>(m, C->rowptr, C->rowend, (const int64_t*)C->col,
                                                       (const double*)C->val, threshold, (const double*)ws,
                                                       rowptrP, (int64_t*)colP, valP);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mfail(SPGEMM_ERR_CUDA, cudaGetErrorString(e));
    return SPGEMM_OK;
}

}  // extern "C"
