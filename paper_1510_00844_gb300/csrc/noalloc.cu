// spgemm_merge_symbolic_static: the row-count step of the k-slice merge
// (same result as spgemm_merge_symbolic) for callers that may not allocate
// device memory and cannot hand the library a workspace -- for example code
// that runs under a fixed device-memory budget reserved at start-up, or a
// plug-in interface that passes only inputs and outputs.  Its scratch (the
// device error word and the scan's per-tile partial sums) lives in one
// file-scope device array of fixed size instead of a caller workspace, so the
// call allocates nothing.
//
// Limits and sharing:
// * at most kStaticMaxRows rows (2^24); larger inputs are rejected;
// * every call on a device uses the same array, which keeps the last call's
//   contents (the error word is cleared at the start of each call); calls
//   that overlap on the GPU (other threads, other streams) race on it;
// * the array's device address is looked up by the first call made on a
//   device, with that device current, and again whenever the device's
//   context has changed since (after a device reset, say); make that first
//   call before any stream capture.
#include <cstdio>
#include <mutex>

#include <cuda.h>

#include "plan.h"

namespace {

constexpr long long kStaticMaxRows = 1LL << 24;
constexpr size_t kCountersBytes = (sizeof(sg::DevCounters) + 255) / 256 * 256;
constexpr size_t kPartialsBytes =
    ((kStaticMaxRows + sg::kScanTile) / sg::kScanTile) * sizeof(int64_t);
constexpr size_t kScratchBytes = kCountersBytes + (kPartialsBytes + 255) / 256 * 256;

// Host code must not use this name as a device address: it is a host-side
// stand-in.  The address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // context the address belongs to

spgemm_status static_fail(spgemm_status st, const char* msg) {
    sg::set_last_error(msg);
    return st;
}

// Unique id of the calling thread's current context (ids are never reused
// within a process, so a reset device's new context has a new one); 0 when
// there is no current context or the driver entry points are unavailable.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = (GetId)f;
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array on the current device: looked up once
// per device and context, and on every call when the context id is unknown.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long ctx = current_context_id();
    if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
        // the lookup made the device's context current if none was
        g_scratch_ctx[dev] = ctx ? ctx : current_context_id();
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" {

spgemm_status spgemm_merge_symbolic_static(int32_t c, const spgemm_csr* parts,
                                           const spgemm_opts* opts, void* stream,
                                           int64_t* rowptrC, int64_t* nnz_c) {
    sg::set_last_error("");
    // the same argument checks as spgemm_merge_symbolic
    int vt = 0;
    spgemm_status st = sg::check_merge_parts(c, parts, opts, &vt);
    if (st != SPGEMM_OK) return st;
    if (!rowptrC || !nnz_c) return static_fail(SPGEMM_ERR_INVALID_ARG, "NULL output");
    const long long m = parts[0].nrows, n = parts[0].ncols;
    if (m > kStaticMaxRows)
        return static_fail(SPGEMM_ERR_INVALID_ARG,
                           "row count outside the static scratch limit (at most 16777216 rows)");
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return static_fail(SPGEMM_ERR_CUDA, cudaGetErrorString(e));
    unsigned char* w = (unsigned char*)base;
    sg::DevCounters* cnt = (sg::DevCounters*)w;
    int64_t* partials = (int64_t*)(w + kCountersBytes);
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the error word must start at zero; the partials are overwritten
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(sg::DevCounters), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(rowptrC + m, 0, sizeof(int64_t), s)) != cudaSuccess)
        return static_fail(SPGEMM_ERR_CUDA, cudaGetErrorString(e));
    e = sg::launch_merge(c, parts, vt, m, n, sms, s, false, rowptrC, nullptr, nullptr, nullptr,
                         &cnt->err, &cnt->work_counter[0]);
    if (e == cudaSuccess) e = sg::launch_exclusive_scan(rowptrC, m + 1, partials, s);
    int64_t total = 0;
    int herr = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, rowptrC + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&herr, &cnt->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return static_fail(SPGEMM_ERR_CUDA, cudaGetErrorString(e));
    if (herr) return static_fail(SPGEMM_ERR_INTERNAL, "device check failed in the merge count");
    *nnz_c = total;
    return SPGEMM_OK;
}

}  // extern "C"
