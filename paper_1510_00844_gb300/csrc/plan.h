// Host-side plan object and launcher declarations (internal).
#pragma once

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/spgemm.h"
#include "kernels.cuh"

// A plan covers a batch of products C_p = A_p . B_p (a single product is a
// batch of one).  Rows of all products are numbered globally; the outputs
// are the concatenation of the products' rows.
struct spgemm_plan_s {
    spgemm_opts opts{};
    cudaStream_t stream = nullptr;
    int it = 0;              // index type
    int vt = 0;              // value type used by the kernels (BOOL when pattern only)
    int nprod = 0;
    std::vector<sg::ProdDesc> descs;   // host copy
    long long R = 0;         // total rows of the batch
    long long LB = 0;        // total B rows of the batch
    long long max_n = 0;     // largest n of the batch
    long long max_dense_n = 0;
    int dense_min = 1024;    // rows with more products than this are dense
    int hash_shift = 0;      // hash rows are binned by flops << hash_shift
    int seg_log2 = 16;       // dense work units of about 2^seg_log2 products
    bool device_sized = false;  // no host readback: sizes are upper bounds
    // plan workspace
    unsigned char* pws = nullptr;
    size_t pws_bytes = 0;
    sg::DevCounters* cnt = nullptr;
    sg::ProdDesc* d_descs = nullptr;
    long long* rb = nullptr;       // row base prefix [nprod+1]
    long long* bb = nullptr;       // B-row base prefix [nprod+1]
    int64_t* flops = nullptr;
    unsigned char* cls = nullptr;
    int32_t* rows = nullptr;
    int64_t* cap = nullptr;          // predicted (learned plans) or flops bound per row
    const float* prm = nullptr;      // row-size predictor parameters (learned plans)
    float margin = 0.f;              // log2 safety margin added to the prediction
    int64_t* unit_cnt = nullptr;     // slot-mode dense numeric: entries per work unit
    // host copies of the row analysis (host-synced plans)
    unsigned long long class_count[sg::kNumClasses] = {};
    long long class_off[sg::kNumClasses + 1] = {};
    long long total_flops = 0, max_flops = 0;
    long long ndense = 0;
    int W = 1024;            // dense chunk width (columns)
    long long max_dense_len = 0;  // cursor arena slot (entries)
    long long dense_grid = 0;     // blocks of the dense numeric kernel
    int dense_warps_per_block = 8;
    long long chunk_total = 0, seg_total = 0, run_total = 0;
    long long nnz_c = -1;
    int sm_count = 1;
    int smem_optin = 0;
};
using Plan = spgemm_plan_s;

namespace sg {

// Value kinds of the kernels: the storage types of spgemm_value_type (BOOL
// when only the pattern is computed) and the min semirings on double and
// int64 storage.
constexpr int kVtMinPlusF64 = 16, kVtMinPlusI64 = 17, kVtMinSelF64 = 18, kVtMinSelI64 = 19;

inline size_t vt_bytes(int vt) {
    return vt == SPGEMM_F32 ? 4 : vt == SPGEMM_BOOL ? 0 : 8;
}

// Calls f(V{}) with the value type of kind vt.
template <class F>
decltype(auto) with_value_type(int vt, F&& f) {
    switch (vt) {
        case SPGEMM_F64: return f(double{});
        case SPGEMM_F32: return f(float{});
        case SPGEMM_I64: return f(int64_t{});
        case kVtMinPlusF64: return f(MinPlus<double>{});
        case kVtMinPlusI64: return f(MinPlus<int64_t>{});
        case kVtMinSelF64: return f(MinSel<double>{});
        case kVtMinSelI64: return f(MinSel<int64_t>{});
        default: return f(NoVal{});
    }
}

// Process-wide count of kernels this library has launched.
void count_launches(long long k);
// Message returned by spgemm_last_error() on this thread.
void set_last_error(const char* msg);

struct WsLayout {
    size_t chunkcnt = 0, segtab = 0, runlen = 0, nextrun = 0, arena = 0, scan = 0, total = 0;
    long long arena_stride = 0;
};
WsLayout workspace_layout(const Plan& P);
size_t plan_workspace_bytes(int nprod, long long R);

spgemm_status make_plan(int32_t count, const spgemm_csr* A, const spgemm_csr* B,
                        const spgemm_opts* opts, void* stream, void* plan_ws, size_t plan_ws_bytes,
                        bool device_sized, spgemm_plan_t* plan_out, const float* sizer_params,
                        float sizer_margin);
spgemm_status check_ws(spgemm_plan_t P, void* ws, size_t ws_bytes);
// Checks of the merge arguments (count of parts, shapes, index and value
// types, semiring); *vt_out = the value kind the merge kernels use.
spgemm_status check_merge_parts(int32_t c, const spgemm_csr* parts, const spgemm_opts* opts,
                                int* vt_out);
cudaError_t run_numeric(Plan* P, unsigned char* w, const int64_t* rowptrC, long long cap,
                        void* colC, void* valC);

size_t scan_temp_bytes(long long N);
cudaError_t launch_exclusive_scan(int64_t* x, long long N, int64_t* temp, cudaStream_t s);
cudaError_t launch_binning(Plan& P);
cudaError_t launch_class_offsets(Plan& P);
cudaError_t launch_zero_rows(const Plan& P, int64_t* rowcnt);
cudaError_t launch_product_rowptr(const Plan& P, const int64_t* g, int64_t* out);

// Template launchers (instantiated per index type / value type).
template <class IT>
cudaError_t launch_analyze(Plan& P);
template <class IT>
cudaError_t launch_row_features(Plan& P, float* X);
template <class IT>
cudaError_t launch_validate(const spgemm_csr& M, int* err, int sm_count, cudaStream_t s);
template <class IT>
cudaError_t launch_symbolic(Plan& P, unsigned char* ws, int64_t* rowcnt);
template <class IT>
cudaError_t launch_dense_tables(Plan& P, unsigned char* ws);
template <class IT, class V>
cudaError_t launch_dense_slot_pack(Plan& P, const int64_t* rpC, void* colC, void* valC,
                                   int64_t* rowend);
long long dense_unit_count(const Plan& P);
template <class IT, class V>
cudaError_t prepare_numeric(Plan& P);
template <class IT, class V>
cudaError_t launch_numeric(Plan& P, unsigned char* ws, const int64_t* rpC, long long cap,
                           void* colC, void* valC, int64_t* rowend = nullptr,
                           int32_t* overflow = nullptr, unsigned* overflow_count = nullptr);
cudaError_t launch_merge(int c, const spgemm_csr* parts, int vt, long long m, long long n,
                         int sm_count, cudaStream_t s, bool numeric, int64_t* rowcnt,
                         const int64_t* rpC, void* colC, void* valC, int* err,
                         unsigned long long* work,   // work: zeroed row counter
                         bool staged = false);       // numeric: stage lists by bulk copies
template <class IT>
cudaError_t launch_kslice_bounds(const spgemm_csr& A, int c, int64_t* bounds, int sm_count,
                                 cudaStream_t s);

}  // namespace sg
