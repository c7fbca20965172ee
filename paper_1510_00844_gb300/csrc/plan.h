// Host-side plan object and launcher declarations (internal).
#pragma once

#include <algorithm>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/spgemm.h"
#include "kernels.cuh"

struct spgemm_plan_s {
    spgemm_csr A{}, B{};
    spgemm_opts opts{};
    cudaStream_t stream = nullptr;
    int it = 0;              // index type
    int vt = 0;              // value type used by the kernels (BOOL when pattern only)
    long long m = 0, l = 0, n = 0;
    long long max_dense_n = 0;
    // plan workspace
    unsigned char* pws = nullptr;
    size_t pws_bytes = 0;
    sg::DevCounters* cnt = nullptr;
    int64_t* flops = nullptr;
    int32_t* rows = nullptr;
    // host copies of the row analysis
    unsigned long long class_count[sg::kNumClasses] = {};
    long long class_off[sg::kNumClasses + 1] = {};
    long long total_flops = 0, max_flops = 0;
    long long ndense = 0;
    int W = 2048;            // dense chunk width (columns)
    int P = 1;               // chunks per dense row
    long long max_dense_len = 0;  // longest A row among dense rows
    long long dense_grid = 0;     // blocks of the dense numeric kernel
    int dense_warps_per_block = 4;
    sg::DenseUnits units{};
    long long nnz_c = -1;
    int sm_count = 1;
    int smem_optin = 0;
};
using Plan = spgemm_plan_s;

namespace sg {

// Process-wide count of kernels this library has launched.
void count_launches(long long k);
// Message returned by spgemm_last_error() on this thread.
void set_last_error(const char* msg);

struct WsLayout {
    size_t chunkcnt = 0, segtab = 0, runlen = 0, arena = 0, scan = 0, total = 0;
    long long arena_stride = 0;
};
void build_dense_units(Plan& P);
WsLayout workspace_layout(const Plan& P);

size_t scan_temp_bytes(long long N);
cudaError_t launch_exclusive_scan(int64_t* x, long long N, int64_t* temp, cudaStream_t s);
cudaError_t launch_binning(Plan& P);
cudaError_t launch_zero_rows(const int32_t* rows, long long nrows, int64_t* rowcnt, int sm_count,
                             cudaStream_t s);

// Template launchers (instantiated per index type / value type).
template <class IT>
cudaError_t launch_analyze(Plan& P);
template <class IT>
cudaError_t launch_validate(const spgemm_csr& M, int* err, int sm_count, cudaStream_t s);
template <class IT>
cudaError_t launch_symbolic(Plan& P, unsigned char* ws, int64_t* rowcnt);
template <class IT, class V>
cudaError_t prepare_numeric(Plan& P);
template <class IT, class V>
cudaError_t launch_numeric(Plan& P, unsigned char* ws, const int64_t* rpC, void* colC, void* valC);
cudaError_t launch_merge(int c, const spgemm_csr* parts, int vt, long long m, long long n,
                         int sm_count, cudaStream_t s, bool numeric, int64_t* rowcnt,
                         const int64_t* rpC, void* colC, void* valC, int* err);
template <class IT>
cudaError_t launch_kslice_bounds(const spgemm_csr& A, int c, int64_t* bounds, int sm_count,
                                 cudaStream_t s);

}  // namespace sg
