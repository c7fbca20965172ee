// Doubly compressed rows (the row-wise form of the DCSC structure of Sec. 3:
// only rows with at least one entry are represented, with their ids).  A
// k-slice or a row panel of a sparse matrix has many empty rows; a DCSR view
// lists its nonempty rows once, so the product's work no longer depends on
// the number of rows.  The view shares A's column and value arrays; the
// product of the view has the same column and value arrays as the product of
// the full matrix (rows stay in order), and only its row pointers need to be
// expanded back to all rows.
#include <cstdio>

#include "plan.h"

namespace sg {

__global__ void nonempty_flags_kernel(long long m, const int64_t* __restrict__ rp,
                                      const int64_t* __restrict__ re, int64_t* __restrict__ flag) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x)
        flag[i] = (re ? re[i] : rp[i + 1]) > rp[i] ? 1 : 0;
}

__global__ void dcsr_scatter_kernel(long long m, const int64_t* __restrict__ rp,
                                    const int64_t* __restrict__ re, const int64_t* __restrict__ pos,
                                    int64_t* __restrict__ rowids, int64_t* __restrict__ vrp,
                                    int64_t* __restrict__ vre) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x) {
        const long long e = re ? re[i] : rp[i + 1];
        if (e > rp[i]) {
            const long long t = pos[i];
            rowids[t] = i;
            vrp[t] = rp[i];
            vre[t] = e;
        }
    }
}

// full[i] = rowptr_c[number of listed rows with id < i], i = 0..m
__global__ void dcsr_expand_kernel(long long m, long long nzr, const int64_t* __restrict__ rowids,
                                   const int64_t* __restrict__ rowptr_c,
                                   int64_t* __restrict__ full) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= m;
         i += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = nzr;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (rowids[mid] < i) lo = mid + 1;
            else hi = mid;
        }
        full[i] = rowptr_c[lo];
    }
}

}  // namespace sg

namespace {

spgemm_status dfail(spgemm_status st, const char* msg) {
    sg::set_last_error(msg);
    return st;
}

unsigned grid1d(long long work) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (unsigned)std::max<long long>(1, std::min<long long>((work + 255) / 256, (long long)sms * 8));
}

}  // namespace

extern "C" {

size_t spgemm_dcsr_workspace_size(int64_t m) {
    if (m < 0) m = 0;
    const size_t a = ((size_t)(m + 1) * 8 + 255) / 256 * 256;
    return a + sg::scan_temp_bytes(m + 1);
}

spgemm_status spgemm_dcsr_view(const spgemm_csr* A, void* stream, void* ws, size_t ws_bytes,
                               int64_t* rowids, int64_t* rowptr_v, int64_t* rowend_v,
                               int64_t* nzr_host) {
    sg::set_last_error("");
    if (!A || !A->rowptr || A->nrows < 0 || !nzr_host)
        return dfail(SPGEMM_ERR_INVALID_ARG, "dcsr: NULL or malformed matrix");
    const long long m = A->nrows;
    if (m > 0 && (!rowids || !rowptr_v || !rowend_v))
        return dfail(SPGEMM_ERR_INVALID_ARG, "dcsr: NULL output");
    if (!ws || ws_bytes < spgemm_dcsr_workspace_size(m))
        return dfail(SPGEMM_ERR_INVALID_ARG, "dcsr: workspace missing or too small");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t* pos = (int64_t*)ws;
    int64_t* temp = (int64_t*)((unsigned char*)ws + ((size_t)(m + 1) * 8 + 255) / 256 * 256);
    cudaError_t e = cudaMemsetAsync(pos + m, 0, 8, s);
    if (e == cudaSuccess && m > 0) {
        sg::count_launches(1);
        sg::nonempty_flags_kernel<<<grid1d(m), 256, 0, s>>>(m, A->rowptr, A->rowend, pos);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = sg::launch_exclusive_scan(pos, m + 1, temp, s);
    if (e == cudaSuccess && m > 0) {
        sg::count_launches(1);
        sg::dcsr_scatter_kernel<<<grid1d(m), 256, 0, s>>>(m, A->rowptr, A->rowend, pos, rowids,
                                                          rowptr_v, rowend_v);
        e = cudaGetLastError();
    }
    int64_t nzr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nzr, pos + m, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return dfail(SPGEMM_ERR_CUDA, cudaGetErrorString(e));
    *nzr_host = nzr;
    return SPGEMM_OK;
}

spgemm_status spgemm_dcsr_expand(int64_t m, int64_t nzr, const int64_t* rowids,
                                 const int64_t* rowptr_c, void* stream, int64_t* rowptr_full) {
    sg::set_last_error("");
    if (m < 0 || nzr < 0 || nzr > m || !rowptr_c || !rowptr_full || (nzr > 0 && !rowids))
        return dfail(SPGEMM_ERR_INVALID_ARG, "dcsr: bad expand arguments");
    cudaStream_t s = (cudaStream_t)stream;
    sg::count_launches(1);
    sg::dcsr_expand_kernel<<<grid1d(m + 1), 256, 0, s>>>(m, nzr, rowids, rowptr_c, rowptr_full);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return dfail(SPGEMM_ERR_CUDA, cudaGetErrorString(e));
    return SPGEMM_OK;
}

}  // extern "C"
