// C ABI of the persistent chain executor (declared in include/spgemm.h):
// many device-sized products, independent or each reading the previous
// one's output, run in one kernel launch (chain.cuh).
#include <algorithm>
#include <cstdio>
#include <vector>

#include "chain.h"

struct spgemm_chain_s {
    int it = 0, vt = 0, nsteps = 0, max_words = 1, sm_count = 1, threads = 768;
    sg::ChainSync* sync = nullptr;          // in the caller's chain workspace
    sg::ChainProduct* steps = nullptr;
    int grid = 0;
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

spgemm_status chain_fail(spgemm_status st, const char* msg) {
    sg::set_last_error(msg);
    return st;
}

spgemm_status chain_cuda_fail(cudaError_t e, const char* where) {
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    sg::set_last_error(buf);
    return SPGEMM_ERR_CUDA;
}

bool chain_value_kind(int vt) {
    return vt == SPGEMM_F64 || vt == SPGEMM_F32 || vt == SPGEMM_I64 || vt == SPGEMM_BOOL;
}

template <class F>
cudaError_t with_chain_types(int it, int vt, F&& f) {
    const bool i32 = it == SPGEMM_INDEX_I32;
    switch (vt) {
        case SPGEMM_F64: return i32 ? f(int32_t{}, double{}) : f(int64_t{}, double{});
        case SPGEMM_F32: return i32 ? f(int32_t{}, float{}) : f(int64_t{}, float{});
        case SPGEMM_I64: return i32 ? f(int32_t{}, int64_t{}) : f(int64_t{}, int64_t{});
        default: return i32 ? f(int32_t{}, sg::NoVal{}) : f(int64_t{}, sg::NoVal{});
    }
}

}  // namespace

extern "C" {

size_t spgemm_chain_workspace_size(int32_t nsteps) {
    if (nsteps < 0) nsteps = 0;
    return align_up(sizeof(sg::ChainSync)) + align_up((size_t)nsteps * sizeof(sg::ChainProduct));
}

spgemm_status spgemm_chain_create(int32_t nsteps, const spgemm_chain_step* steps,
                                  const spgemm_chain_opts* opts, void* chain_ws,
                                  size_t chain_ws_bytes, spgemm_chain_t* chain_out) {
    sg::set_last_error("");
    if (nsteps < 1 || !steps || !chain_out)
        return chain_fail(SPGEMM_ERR_INVALID_ARG, "need at least one step and a chain handle");
    const size_t need = spgemm_chain_workspace_size(nsteps);
    if (!chain_ws || chain_ws_bytes < need)
        return chain_fail(SPGEMM_ERR_OUT_OF_MEMORY, "chain workspace too small");
    if (((uintptr_t)chain_ws) % kAlign)
        return chain_fail(SPGEMM_ERR_INVALID_ARG, "chain workspace not 256-byte aligned");
    spgemm_chain_opts o{};
    if (opts) o = *opts;
    if (o.timeout_s < 0) return chain_fail(SPGEMM_ERR_INVALID_ARG, "negative timeout");
    if (o.block_threads != 0 && o.block_threads != sg::kChainThreads &&
        o.block_threads != sg::kChainThreadsWide)
        return chain_fail(SPGEMM_ERR_INVALID_ARG, "block_threads must be 0, 768 or 1024");
    const spgemm_plan_t P0 = steps[0].plan;
    if (!P0) return chain_fail(SPGEMM_ERR_INVALID_ARG, "step 0 has no plan");
    if (!chain_value_kind(P0->vt))
        return chain_fail(SPGEMM_ERR_NOT_SUPPORTED,
                          "chains take float64, float32, int64 or Boolean products");
    std::vector<sg::ChainProduct> host((size_t)nsteps);
    long long max_words = 1;
    for (int p = 0; p < nsteps; ++p) {
        const spgemm_chain_step& st = steps[p];
        const spgemm_plan_t P = st.plan;
        if (!P || !P->device_sized)
            return chain_fail(SPGEMM_ERR_INVALID_ARG, "chain steps need plans from spgemm_plan_device");
        if (P->it != P0->it || P->vt != P0->vt)
            return chain_fail(SPGEMM_ERR_INVALID_ARG, "all steps of a chain use one index and value type");
        if (!st.rowptrC || st.capacity < 0 || (st.capacity > 0 && !st.colC) ||
            (st.capacity > 0 && P->vt != SPGEMM_BOOL && !st.valC))
            return chain_fail(SPGEMM_ERR_INVALID_ARG, "a step misses its output arrays");
        if (sg::check_ws(P, st.ws, st.ws_bytes) != SPGEMM_OK) return SPGEMM_ERR_OUT_OF_MEMORY;
        const sg::WsLayout L = sg::workspace_layout(*P);
        unsigned char* w = (unsigned char*)st.ws;
        sg::ChainProduct& c = host[(size_t)p];
        c.D = P->d_descs;
        c.rb = P->rb;
        c.bb = P->bb;
        c.cnt = P->cnt;
        c.flops = P->flops;
        c.cls = P->cls;
        c.rows = P->rows;
        c.cap = P->cap;
        c.prm = P->prm;
        c.margin = P->margin;
        c.chunkcnt = (int32_t*)(w + L.chunkcnt);
        c.segtab = (int32_t*)(w + L.segtab);
        c.runlen = (int32_t*)(w + L.runlen);
        c.nextrun = (int2*)(w + L.nextrun);
        c.arena = (sg::DenseCursor*)(w + L.arena);
        c.arena_stride = L.arena_stride;
        c.scan = (int64_t*)(w + L.scan);
        c.rowptrC = st.rowptrC;
        c.colC = st.colC;
        c.valC = st.valC;
        c.capacity = st.capacity;
        c.R = P->R;
        c.LB = P->LB;
        c.nprod = P->nprod;
        c.W = P->W;
        c.dense_min = P->dense_min;
        c.hash_shift = P->hash_shift;
        c.seg_log2 = P->seg_log2;
        c.max_dense_n = P->max_dense_n;
        max_words = std::max(max_words, (std::min(P->max_n, P->max_dense_n) + 31) / 32);
        // the dense stages use 8 warps per persistent block; their cursor
        // arena slots must exist in the plan's workspace
        const int dense_warps = P->W == sg::kDenseW0 ? sg::kChainDense0 : sg::kChainDense1;
        if (P->dense_grid * P->dense_warps_per_block < (long long)P->sm_count * dense_warps)
            return chain_fail(SPGEMM_ERR_NOT_SUPPORTED, "plan's dense arena too small for a chain");
    }
    // the dense symbolic bitmap shares the persistent block's shared memory
    // with the other stages; wider products fall back to the TooWide report
    int optin = 48 * 1024, dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long words_cap = (long long)(optin - 16 * 1024) / 4;
    if (max_words > words_cap) {
        max_words = words_cap;
        for (auto& c : host) c.max_dense_n = std::min(c.max_dense_n, 32 * words_cap);
    }
    for (auto& c : host) c.max_words = (int)max_words;
    spgemm_chain_t C = new spgemm_chain_s();
    C->it = P0->it;
    C->vt = P0->vt;
    C->nsteps = nsteps;
    C->max_words = (int)max_words;
    C->sm_count = sms;
    C->threads = o.block_threads ? o.block_threads : sg::kChainThreads;
    unsigned char* base = (unsigned char*)chain_ws;
    C->sync = (sg::ChainSync*)base;
    C->steps = (sg::ChainProduct*)(base + align_up(sizeof(sg::ChainSync)));
    sg::ChainSync hs{};
    const double t = o.timeout_s > 0 ? o.timeout_s : 10.0;
    hs.timeout_ns = (unsigned long long)(t * 1e9);
    hs.withhold = o.withhold_stage;
    hs.nsteps = nsteps;
    hs.stamps = reinterpret_cast<unsigned long long*>(o.stage_ns);
    cudaError_t e = cudaMemcpy(C->sync, &hs, sizeof(hs), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(C->steps, host.data(), host.size() * sizeof(sg::ChainProduct),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete C;
        return chain_cuda_fail(e, "chain: table upload");
    }
    *chain_out = C;
    return SPGEMM_OK;
}

spgemm_status spgemm_chain_launch(spgemm_chain_t C, void* stream) {
    if (!C) return chain_fail(SPGEMM_ERR_INVALID_ARG, "NULL chain");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = with_chain_types(C->it, C->vt, [&](auto itag, auto vtag) -> cudaError_t {
        using IT = decltype(itag);
        using V = decltype(vtag);
        if (C->threads == sg::kChainThreadsWide)
            return sg::launch_chain<IT, V, sg::kChainThreadsWide>(C->steps, C->sync, C->max_words,
                                                                  C->sm_count, s, &C->grid);
        return sg::launch_chain<IT, V, sg::kChainThreads>(C->steps, C->sync, C->max_words,
                                                          C->sm_count, s, &C->grid);
    });
    if (e != cudaSuccess) return chain_cuda_fail(e, "chain launch");
    return SPGEMM_OK;
}

spgemm_status spgemm_chain_check(spgemm_chain_t C, void* stream) {
    if (!C) return chain_fail(SPGEMM_ERR_INVALID_ARG, "NULL chain");
    int status = 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&status, &C->sync->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return chain_cuda_fail(e, "chain check");
    if (status == sg::kDevTimeout)
        return chain_fail(SPGEMM_ERR_TIMEOUT, "a chain stage waited longer than the timeout");
    if (status) return chain_fail(SPGEMM_ERR_INTERNAL, "chain status word set");
    return SPGEMM_OK;
}

int32_t spgemm_chain_grid(spgemm_chain_t C) { return C ? C->grid : 0; }

void spgemm_chain_destroy(spgemm_chain_t C) { delete C; }

}  // extern "C"
