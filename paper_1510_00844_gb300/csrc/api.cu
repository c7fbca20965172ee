// C ABI of the library (declared in include/spgemm.h): argument checks,
// plan bookkeeping, dispatch on index/value type, error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <new>

#include "plan.h"

namespace {

thread_local std::string g_last_error;

spgemm_status fail(spgemm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

spgemm_status cuda_fail(cudaError_t e, const char* where) {
    return fail(SPGEMM_ERR_CUDA, "%s: CUDA error %d (%s)", where, (int)e, cudaGetErrorString(e));
}

#define SG_CUDA(call, where)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);   \
    } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool valid_value_type(int32_t v) { return v >= SPGEMM_F64 && v <= SPGEMM_BOOL; }
bool valid_index_type(int32_t t) { return t == SPGEMM_INDEX_I32 || t == SPGEMM_INDEX_I64; }

spgemm_status check_csr(const spgemm_csr* M, const char* name, bool need_vals) {
    if (!M) return fail(SPGEMM_ERR_INVALID_ARG, "%s is NULL", name);
    if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0)
        return fail(SPGEMM_ERR_INVALID_ARG, "%s has a negative size", name);
    if (!valid_index_type(M->index_type))
        return fail(SPGEMM_ERR_INVALID_ARG, "%s.index_type invalid", name);
    if (!valid_value_type(M->value_type))
        return fail(SPGEMM_ERR_INVALID_ARG, "%s.value_type invalid", name);
    if (!M->rowptr) return fail(SPGEMM_ERR_INVALID_ARG, "%s.rowptr is NULL", name);
    if (M->nnz > 0 && !M->col) return fail(SPGEMM_ERR_INVALID_ARG, "%s.col is NULL", name);
    if (need_vals && M->nnz > 0 && !M->val)
        return fail(SPGEMM_ERR_INVALID_ARG, "%s.val is NULL", name);
    if (M->index_type == SPGEMM_INDEX_I32 && (M->ncols > 0x7fffffffLL || M->nrows > 0x7fffffffLL))
        return fail(SPGEMM_ERR_INDEX_OVERFLOW, "%s dimensions exceed int32 indices", name);
    if (M->nrows > 0x7fffffffLL)
        return fail(SPGEMM_ERR_NOT_SUPPORTED, "%s has more than 2^31-1 rows", name);
    return SPGEMM_OK;
}

// value type the kernels use: BOOL for the (or, and) semiring
int kernel_value_type(const spgemm_csr* A, const spgemm_opts* o) {
    if ((o && o->semiring == SPGEMM_OR_AND) || A->value_type == SPGEMM_BOOL) return SPGEMM_BOOL;
    if (o && o->semiring == SPGEMM_MIN_PLUS)
        return A->value_type == SPGEMM_I64 ? sg::kVtMinPlusI64 : sg::kVtMinPlusF64;
    if (o && o->semiring == SPGEMM_MIN_SELECT2ND)
        return A->value_type == SPGEMM_I64 ? sg::kVtMinSelI64 : sg::kVtMinSelF64;
    return A->value_type;
}

// The min semirings run on float64 and int64 values only.
spgemm_status check_semiring(const spgemm_opts& o, const spgemm_csr* A) {
    if (o.semiring < SPGEMM_PLUS_TIMES || o.semiring > SPGEMM_MIN_SELECT2ND)
        return fail(SPGEMM_ERR_INVALID_ARG, "unknown semiring %d", o.semiring);
    if ((o.semiring == SPGEMM_MIN_PLUS || o.semiring == SPGEMM_MIN_SELECT2ND) && A &&
        A->value_type != SPGEMM_F64 && A->value_type != SPGEMM_I64)
        return fail(SPGEMM_ERR_NOT_SUPPORTED, "the min semirings need float64 or int64 values");
    return SPGEMM_OK;
}

int device_sm_count(int* smem_optin) {
    int dev = 0, sms = 1, optin = 48 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    if (smem_optin) *smem_optin = optin;
    return sms;
}

}  // namespace

namespace sg {

// Work units of the dense numeric kernel: each dense row of class t is cut
// into dense_class_segments(t) segments.
long long dense_unit_count(const Plan& P) {
    long long u = 0;
    for (int t = 0; t < kMaxDenseClasses; ++t)
        u += (long long)P.class_count[kClassDense0 + t] * dense_class_segments(t, P.seg_log2);
    return u;
}


static std::atomic<long long> g_launches{0};
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void set_last_error(const char* msg) { g_last_error = msg; }

WsLayout workspace_layout(const Plan& P) {
    WsLayout L;
    const bool dense = P.device_sized || P.ndense > 0;
    size_t off = 0;
    L.chunkcnt = off;
    if (dense) off += align_up((size_t)P.chunk_total * sizeof(int32_t));
    L.segtab = off;
    if (dense) off += align_up((size_t)P.seg_total * sizeof(int32_t));
    L.runlen = off;
    if (dense) off += align_up((size_t)P.run_total * sizeof(int32_t));
    L.nextrun = off;
    if (dense) off += align_up((size_t)P.run_total * sizeof(int2));
    L.arena = off;
    L.arena_stride = std::max<long long>(1, P.max_dense_len);
    if (dense)
        off += align_up((size_t)P.dense_grid * P.dense_warps_per_block * (size_t)L.arena_stride *
                        sizeof(DenseCursor));
    L.scan = off;
    off += align_up(scan_temp_bytes(P.R + 1));
    L.total = off;
    return L;
}

size_t plan_workspace_bytes(int nprod, long long R) {
    if (R < 0) R = 0;
    return align_up(sizeof(DevCounters)) + align_up((size_t)nprod * sizeof(ProdDesc)) +
           2 * align_up((size_t)(nprod + 1) * sizeof(long long)) +
           align_up((size_t)R * sizeof(int64_t)) + align_up((size_t)R) +
           align_up((size_t)R * sizeof(int32_t)) + align_up((size_t)R * sizeof(int64_t));
}

}  // namespace sg

namespace sg {

// Checks and records a batch of products; shared by spgemm_plan,
// spgemm_batch_plan and spgemm_plan_device.
spgemm_status make_plan(int32_t count, const spgemm_csr* A, const spgemm_csr* B,
                        const spgemm_opts* opts, void* stream, void* plan_ws, size_t plan_ws_bytes,
                        bool device_sized, spgemm_plan_t* plan_out, const float* sizer_params,
                        float sizer_margin) {
    g_last_error.clear();
    if (!plan_out) return fail(SPGEMM_ERR_INVALID_ARG, "plan output pointer is NULL");
    *plan_out = nullptr;
    if (count < 1) return fail(SPGEMM_ERR_INVALID_ARG, "a batch needs at least one product");
    spgemm_opts o{};
    if (opts) o = *opts;
    if (!A || !B) return fail(SPGEMM_ERR_INVALID_ARG, "A or B is NULL");
    if (spgemm_status st0 = check_semiring(o, &A[0]); st0 != SPGEMM_OK) return st0;
    if (o.dense_chunk != 0 && o.dense_chunk != sg::kDenseW0 && o.dense_chunk != sg::kDenseW1)
        return fail(SPGEMM_ERR_INVALID_ARG, "dense_chunk must be 0, %d or %d", sg::kDenseW0,
                    sg::kDenseW1);
    if (o.dense_min_flops != 0 && (o.dense_min_flops < 32 || o.dense_min_flops > 1024))
        return fail(SPGEMM_ERR_INVALID_ARG, "dense_min_flops must be 0 or in [32, 1024]");
    if (o.max_row_nnz < 0) return fail(SPGEMM_ERR_INVALID_ARG, "max_row_nnz must be >= 0");
    if (o.hash_shift < 0 || o.hash_shift > 2)
        return fail(SPGEMM_ERR_INVALID_ARG, "hash_shift must be in [0, 2]");
    if (o.seg_log2 != 0 && (o.seg_log2 < 10 || o.seg_log2 > 22))
        return fail(SPGEMM_ERR_INVALID_ARG, "seg_log2 must be 0 or in [10, 22]");
    if (!A || !B) return fail(SPGEMM_ERR_INVALID_ARG, "A or B is NULL");
    const int vt = kernel_value_type(&A[0], &o);
    const bool need_vals = vt != SPGEMM_BOOL;
    long long R = 0;
    for (int p = 0; p < count; ++p) {
        spgemm_status st;
        if ((st = check_csr(&A[p], "A", need_vals)) != SPGEMM_OK) return st;
        if ((st = check_csr(&B[p], "B", need_vals)) != SPGEMM_OK) return st;
        if (A[p].ncols != B[p].nrows)
            return fail(SPGEMM_ERR_INVALID_ARG,
                        "product %d: inner dimensions differ: A is %lld x %lld, B is %lld x %lld", p,
                        (long long)A[p].nrows, (long long)A[p].ncols, (long long)B[p].nrows,
                        (long long)B[p].ncols);
        if (A[p].index_type != A[0].index_type || B[p].index_type != A[0].index_type)
            return fail(SPGEMM_ERR_INVALID_ARG, "product %d: index types differ", p);
        if (need_vals && (A[p].value_type != A[0].value_type || B[p].value_type != A[0].value_type))
            return fail(SPGEMM_ERR_INVALID_ARG, "product %d: value types differ", p);
        if (B[p].rowend)
            return fail(SPGEMM_ERR_INVALID_ARG, "product %d: B must be a plain CSR (rowend NULL)", p);
        R += A[p].nrows;
    }
    if (R > 0x7fffffffLL)
        return fail(SPGEMM_ERR_NOT_SUPPORTED, "a batch may have at most 2^31-1 rows in total");
    const size_t need = sg::plan_workspace_bytes(count, R);
    if (!plan_ws || plan_ws_bytes < need)
        return fail(SPGEMM_ERR_OUT_OF_MEMORY, "plan workspace %zu bytes < %zu required",
                    plan_ws_bytes, need);
    if (((uintptr_t)plan_ws) % kAlign)
        return fail(SPGEMM_ERR_INVALID_ARG, "plan workspace not %zu-byte aligned", kAlign);

    Plan* P = new (std::nothrow) Plan();
    if (!P) return fail(SPGEMM_ERR_OUT_OF_MEMORY, "host allocation of the plan failed");
    auto bail = [&](spgemm_status s) {
        delete P;
        return s;
    };
    P->opts = o;
    P->stream = (cudaStream_t)stream;
    P->it = A[0].index_type;
    P->vt = vt;
    P->nprod = count;
    P->R = R;
    P->device_sized = device_sized;
    P->prm = sizer_params;
    P->margin = sizer_margin;
    P->dense_min = o.dense_min_flops ? o.dense_min_flops : 1024;
    P->hash_shift = o.hash_shift;
    P->seg_log2 = o.seg_log2 ? o.seg_log2 : 16;  // host-synced plans refine it below
    P->sm_count = device_sm_count(&P->smem_optin);
    // the dense symbolic bitmap (n bits) must fit the per-block shared memory
    P->max_dense_n = (long long)(P->smem_optin - 1024) * 8;
    {
        // 8-byte values: 1024-column chunks (eight warps per block) up to
        // 2^18 columns, 2048 beyond (fewer chunks per row; measured faster on
        // R-MAT 20, slower on R-MAT 18); 4-byte values and patterns: 2048
        long long widest = 0;
        for (int p = 0; p < count; ++p) widest = std::max<long long>(widest, B[p].ncols);
        const size_t vbytes = sg::vt_bytes(vt);
        int cfg = (vbytes == 8 && widest <= (1LL << 18)) ? 0 : 1;
        if (o.dense_chunk == sg::kDenseW0) cfg = 0;
        if (o.dense_chunk == sg::kDenseW1) cfg = 1;
        P->W = cfg == 0 ? sg::kDenseW0 : sg::kDenseW1;
    }
    P->descs.resize(count);
    std::vector<long long> rb(count + 1), bb(count + 1);
    long long rbase = 0, bbase = 0, chunk = 0, seg = 0, run = 0;
    for (int p = 0; p < count; ++p) {
        sg::ProdDesc& d = P->descs[p];
        d = sg::ProdDesc{};
        d.m = A[p].nrows;
        d.l = A[p].ncols;
        d.n = B[p].ncols;
        d.row_base = rbase;
        d.brow_base = bbase;
        d.rpA = A[p].rowptr;
        d.reA = A[p].rowend;
        d.ciA = A[p].col;
        d.vA = need_vals ? A[p].val : nullptr;
        d.rpB = B[p].rowptr;
        d.ciB = B[p].col;
        d.vB = need_vals ? B[p].val : nullptr;
        d.nnzB = B[p].nnz;
        d.P = (int)std::max<long long>(1, (d.n + P->W - 1) / P->W);
        d.chunk_base = chunk;
        d.seg_base = seg;
        d.run_base = run;
        rb[p] = rbase;
        bb[p] = bbase;
        rbase += d.m;
        bbase += d.l;
        chunk += d.m * d.P;
        seg += d.l * (sg::kSegGrid + 1);
        run += d.nnzB;
        P->max_n = std::max(P->max_n, d.n);
    }
    rb[count] = rbase;
    bb[count] = bbase;
    P->LB = bbase;
    P->chunk_total = chunk;
    P->seg_total = seg;
    P->run_total = run;
    // plan workspace layout
    P->pws = (unsigned char*)plan_ws;
    P->pws_bytes = plan_ws_bytes;
    size_t off = 0;
    P->cnt = (sg::DevCounters*)(P->pws + off);
    off += align_up(sizeof(sg::DevCounters));
    P->d_descs = (sg::ProdDesc*)(P->pws + off);
    off += align_up((size_t)count * sizeof(sg::ProdDesc));
    P->rb = (long long*)(P->pws + off);
    off += align_up((size_t)(count + 1) * sizeof(long long));
    P->bb = (long long*)(P->pws + off);
    off += align_up((size_t)(count + 1) * sizeof(long long));
    P->flops = (int64_t*)(P->pws + off);
    off += align_up((size_t)R * sizeof(int64_t));
    P->cls = P->pws + off;
    off += align_up((size_t)R);
    P->rows = (int32_t*)(P->pws + off);
    off += align_up((size_t)R * sizeof(int32_t));
    P->cap = (int64_t*)(P->pws + off);

    cudaStream_t s = P->stream;
    cudaError_t e = cudaMemcpyAsync(P->d_descs, P->descs.data(), count * sizeof(sg::ProdDesc),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->rb, rb.data(), (count + 1) * sizeof(long long),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->bb, bb.data(), (count + 1) * sizeof(long long),
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "plan: descriptor upload"));

    auto prepare = [&]() -> cudaError_t {
        const bool i32 = P->it == SPGEMM_INDEX_I32;
        return sg::with_value_type(P->vt, [&](auto tag) -> cudaError_t {
            using V = decltype(tag);
            return i32 ? sg::prepare_numeric<int32_t, V>(*P) : sg::prepare_numeric<int64_t, V>(*P);
        });
    };

    if (device_sized) {
        // sizes are upper bounds; the row analysis runs inside spgemm_execute
        P->max_dense_len = o.max_row_nnz ? o.max_row_nnz : 65536;
        e = prepare();
        if (e != cudaSuccess) return bail(cuda_fail(e, "plan: numeric setup"));
        e = cudaStreamSynchronize(s);  // the descriptor upload reads host buffers
        if (e != cudaSuccess) return bail(cuda_fail(e, "plan: sync"));
        *plan_out = P;
        return SPGEMM_OK;
    }

    e = cudaMemsetAsync(P->cnt, 0, sizeof(sg::DevCounters), s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "plan: memset"));
    if (o.checked) {
        int* err = &P->cnt->err;
        for (int p = 0; p < count && e == cudaSuccess; ++p) {
            e = P->it == SPGEMM_INDEX_I32 ? sg::launch_validate<int32_t>(A[p], err, P->sm_count, s)
                                          : sg::launch_validate<int64_t>(A[p], err, P->sm_count, s);
            if (e == cudaSuccess)
                e = P->it == SPGEMM_INDEX_I32 ? sg::launch_validate<int32_t>(B[p], err, P->sm_count, s)
                                              : sg::launch_validate<int64_t>(B[p], err, P->sm_count, s);
        }
        if (e != cudaSuccess) return bail(cuda_fail(e, "plan: validate"));
        int herr = 0;
        e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bail(cuda_fail(e, "plan: validate readback"));
        if (herr != 0)
            return bail(fail(SPGEMM_ERR_INVALID_CSR, "invalid CSR input (%s)",
                             herr == sg::kDevBadRowptr
                                 ? "row pointers not monotone or out of range"
                                 : "column index out of range, unsorted or duplicated"));
    }
    e = P->it == SPGEMM_INDEX_I32 ? sg::launch_analyze<int32_t>(*P) : sg::launch_analyze<int64_t>(*P);
    if (e != cudaSuccess) return bail(cuda_fail(e, "plan: analyze"));
    e = sg::launch_binning(*P);
    if (e != cudaSuccess) return bail(cuda_fail(e, "plan: binning"));
    sg::DevCounters h;
    e = cudaMemcpyAsync(&h, P->cnt, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "plan: readback"));
    if (h.unsupported)
        return bail(fail(SPGEMM_ERR_NOT_SUPPORTED,
                         "rows with more than %d products need n <= %lld columns (n = %lld)",
                         P->dense_min, P->max_dense_n, P->max_n));
    long long acc = 0;
    for (int c = 0; c < sg::kNumClasses; ++c) {
        P->class_count[c] = h.class_count[c];
        P->class_off[c] = acc;
        acc += (long long)h.class_count[c];
    }
    P->class_off[sg::kNumClasses] = acc;
    P->total_flops = (long long)h.total_flops;
    P->max_flops = (long long)h.max_flops;
    P->ndense = acc - P->class_off[sg::kClassDense0];
    P->max_dense_len = (long long)h.max_dense_len;
    e = prepare();
    if (e != cudaSuccess) return bail(cuda_fail(e, "plan: numeric setup"));
    if (!o.seg_log2 && P->ndense > 0) {
        // dense work units of about total_flops / (4 x resident dense warps)
        // products: few, long units on big products, enough of them on small
        const double warps = (double)std::max<long long>(1, P->dense_grid * P->dense_warps_per_block);
        const double per = (double)std::max<long long>(1, P->total_flops) / (4.0 * warps);
        P->seg_log2 = std::min(20, std::max(14, (int)std::floor(std::log2(per))));
        if (P->seg_log2 != 16) {
            e = sg::launch_class_offsets(*P);
            if (e != cudaSuccess) return bail(cuda_fail(e, "plan: work units"));
        }
    }
    *plan_out = P;
    return SPGEMM_OK;
}

spgemm_status check_ws(spgemm_plan_t P, void* ws, size_t ws_bytes) {
    size_t need = sg::workspace_layout(*P).total;
    if (need > 0 && (!ws || ws_bytes < need))
        return fail(SPGEMM_ERR_OUT_OF_MEMORY, "workspace %zu bytes < %zu required", ws_bytes, need);
    if (ws && ((uintptr_t)ws) % kAlign)
        return fail(SPGEMM_ERR_INVALID_ARG, "workspace not %zu-byte aligned", kAlign);
    return SPGEMM_OK;
}

cudaError_t run_numeric(Plan* P, unsigned char* w, const int64_t* rowptrC, long long cap,
                        void* colC, void* valC) {
    const bool i32 = P->it == SPGEMM_INDEX_I32;
    return sg::with_value_type(P->vt, [&](auto tag) -> cudaError_t {
        using V = decltype(tag);
        void* vals = VOps<V>::has_val ? valC : nullptr;
        return i32 ? sg::launch_numeric<int32_t, V>(*P, w, rowptrC, cap, colC, vals)
                   : sg::launch_numeric<int64_t, V>(*P, w, rowptrC, cap, colC, vals);
    });
}

}  // namespace sg

using sg::make_plan;
using sg::check_ws;
using sg::run_numeric;

namespace sg {
// The argument checks of the merge entry points (shared with the
// allocation-free count in noalloc.cu).
spgemm_status check_merge_parts(int32_t c, const spgemm_csr* parts, const spgemm_opts* opts,
                                int* vt_out) {
    if (c < 1 || c > 32) return fail(SPGEMM_ERR_INVALID_ARG, "merge needs 1 <= c <= 32 parts (c = %d)", c);
    if (!parts) return fail(SPGEMM_ERR_INVALID_ARG, "parts is NULL");
    spgemm_opts o{};
    if (opts) o = *opts;
    if (spgemm_status st0 = check_semiring(o, &parts[0]); st0 != SPGEMM_OK) return st0;
    const int vt = kernel_value_type(&parts[0], &o);
    for (int s = 0; s < c; ++s) {
        spgemm_status st = check_csr(&parts[s], "part", vt != SPGEMM_BOOL);
        if (st != SPGEMM_OK) return st;
        if (parts[s].nrows != parts[0].nrows || parts[s].ncols != parts[0].ncols)
            return fail(SPGEMM_ERR_INVALID_ARG, "part %d shape differs from part 0", s);
        if (parts[s].index_type != parts[0].index_type)
            return fail(SPGEMM_ERR_INVALID_ARG, "part %d index type differs", s);
        if (vt != SPGEMM_BOOL && parts[s].value_type != parts[0].value_type)
            return fail(SPGEMM_ERR_INVALID_ARG, "part %d value type differs", s);
    }
    *vt_out = vt;
    return SPGEMM_OK;
}
}  // namespace sg

extern "C" {

int64_t spgemm_kernel_launches(void) { return sg::g_launches.load(); }

const char* spgemm_version(void) { return "gb300-spgemm 0.2 (sm_103a)"; }

const char* spgemm_last_error(void) { return g_last_error.c_str(); }

size_t spgemm_plan_workspace_size(int64_t m) { return sg::plan_workspace_bytes(1, m); }

size_t spgemm_batch_plan_workspace_size(int32_t count, const spgemm_csr* A) {
    long long R = 0;
    if (A)
        for (int p = 0; p < count; ++p) R += std::max<long long>(0, A[p].nrows);
    return sg::plan_workspace_bytes(std::max(count, 1), R);
}

spgemm_status spgemm_plan(const spgemm_csr* A, const spgemm_csr* B, const spgemm_opts* opts,
                          void* stream, void* plan_ws, size_t plan_ws_bytes,
                          spgemm_plan_t* plan_out) {
    return make_plan(1, A, B, opts, stream, plan_ws, plan_ws_bytes, false, plan_out, nullptr, 0.f);
}

spgemm_status spgemm_batch_plan(int32_t count, const spgemm_csr* A, const spgemm_csr* B,
                                const spgemm_opts* opts, void* stream, void* plan_ws,
                                size_t plan_ws_bytes, spgemm_plan_t* plan_out) {
    return make_plan(count, A, B, opts, stream, plan_ws, plan_ws_bytes, false, plan_out, nullptr,
                     0.f);
}

spgemm_status spgemm_plan_device(int32_t count, const spgemm_csr* A, const spgemm_csr* B,
                                 const spgemm_opts* opts, void* stream, void* plan_ws,
                                 size_t plan_ws_bytes, spgemm_plan_t* plan_out) {
    return make_plan(count, A, B, opts, stream, plan_ws, plan_ws_bytes, true, plan_out, nullptr,
                     0.f);
}

spgemm_status spgemm_plan_info(spgemm_plan_t P, spgemm_info* info) {
    if (!P || !info) return fail(SPGEMM_ERR_INVALID_ARG, "NULL argument");
    info->m = P->R;
    info->l = P->nprod == 1 ? P->descs[0].l : P->LB;
    info->n = P->max_n;
    info->flops = P->total_flops;
    info->max_row_flops = P->max_flops;
    info->rows_empty = (int64_t)P->class_count[sg::kClassEmpty];
    long long h = 0;
    for (int b = 0; b < sg::kNumHashBins; ++b) h += (long long)P->class_count[sg::kClassHash0 + b];
    info->rows_hash = h;
    info->rows_dense = P->ndense;
    info->chunk_width = P->W;
    info->chunks_per_row = P->nprod == 1 ? P->descs[0].P : 0;
    info->nnz_c = P->nnz_c;
    return SPGEMM_OK;
}

spgemm_status spgemm_workspace_size(spgemm_plan_t P, size_t* bytes) {
    if (!P || !bytes) return fail(SPGEMM_ERR_INVALID_ARG, "NULL argument");
    *bytes = sg::workspace_layout(*P).total;
    return SPGEMM_OK;
}

spgemm_status spgemm_symbolic(spgemm_plan_t P, void* ws, size_t ws_bytes, int64_t* rowptrC,
                              int64_t* nnz_c) {
    g_last_error.clear();
    if (!P || !rowptrC || !nnz_c) return fail(SPGEMM_ERR_INVALID_ARG, "NULL argument");
    if (P->device_sized)
        return fail(SPGEMM_ERR_INVALID_ARG, "device-sized plans run through spgemm_execute");
    spgemm_status st = check_ws(P, ws, ws_bytes);
    if (st != SPGEMM_OK) return st;
    cudaStream_t s = P->stream;
    unsigned char* w = (unsigned char*)ws;
    SG_CUDA(cudaMemsetAsync(rowptrC + P->R, 0, sizeof(int64_t), s), "symbolic: memset");
    cudaError_t e = P->it == SPGEMM_INDEX_I32 ? sg::launch_symbolic<int32_t>(*P, w, rowptrC)
                                              : sg::launch_symbolic<int64_t>(*P, w, rowptrC);
    if (e != cudaSuccess) return cuda_fail(e, "symbolic");
    sg::WsLayout L = sg::workspace_layout(*P);
    e = sg::launch_exclusive_scan(rowptrC, P->R + 1, (int64_t*)(w + L.scan), s);
    if (e != cudaSuccess) return cuda_fail(e, "symbolic: scan");
    int64_t total = 0;
    int herr = 0;
    SG_CUDA(cudaMemcpyAsync(&total, rowptrC + P->R, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
            "symbolic: readback");
    SG_CUDA(cudaMemcpyAsync(&herr, &P->cnt->err, sizeof(int), cudaMemcpyDeviceToHost, s),
            "symbolic: readback");
    SG_CUDA(cudaStreamSynchronize(s), "symbolic: sync");
    if (herr) return fail(SPGEMM_ERR_INTERNAL, "device check failed in symbolic phase (code %d)", herr);
    P->nnz_c = total;
    *nnz_c = total;
    return SPGEMM_OK;
}

spgemm_status spgemm_numeric(spgemm_plan_t P, void* ws, size_t ws_bytes, const int64_t* rowptrC,
                             void* colC, void* valC) {
    g_last_error.clear();
    if (!P || !rowptrC) return fail(SPGEMM_ERR_INVALID_ARG, "NULL argument");
    if (P->device_sized)
        return fail(SPGEMM_ERR_INVALID_ARG, "device-sized plans run through spgemm_execute");
    if (P->nnz_c < 0) return fail(SPGEMM_ERR_INVALID_ARG, "spgemm_symbolic has not run on this plan");
    if (P->nnz_c > 0 && !colC) return fail(SPGEMM_ERR_INVALID_ARG, "colC is NULL");
    if (P->nnz_c > 0 && P->vt != SPGEMM_BOOL && !valC)
        return fail(SPGEMM_ERR_INVALID_ARG, "valC is NULL");
    spgemm_status st = check_ws(P, ws, ws_bytes);
    if (st != SPGEMM_OK) return st;
    cudaError_t e = run_numeric(P, (unsigned char*)ws, rowptrC, P->nnz_c, colC, valC);
    if (e != cudaSuccess) return cuda_fail(e, "numeric");
    return SPGEMM_OK;
}

spgemm_status spgemm_execute(spgemm_plan_t P, void* ws, size_t ws_bytes, int64_t* rowptrC,
                             int64_t capacity, void* colC, void* valC) {
    g_last_error.clear();
    if (!P || !rowptrC) return fail(SPGEMM_ERR_INVALID_ARG, "NULL argument");
    if (!P->device_sized)
        return fail(SPGEMM_ERR_INVALID_ARG, "spgemm_execute needs a plan from spgemm_plan_device");
    if (capacity < 0) return fail(SPGEMM_ERR_INVALID_ARG, "negative capacity");
    if (capacity > 0 && !colC) return fail(SPGEMM_ERR_INVALID_ARG, "colC is NULL");
    if (capacity > 0 && P->vt != SPGEMM_BOOL && !valC)
        return fail(SPGEMM_ERR_INVALID_ARG, "valC is NULL");
    spgemm_status st = check_ws(P, ws, ws_bytes);
    if (st != SPGEMM_OK) return st;
    cudaStream_t s = P->stream;
    unsigned char* w = (unsigned char*)ws;
    SG_CUDA(cudaMemsetAsync(P->cnt, 0, sizeof(sg::DevCounters), s), "execute: memset");
    cudaError_t e = P->it == SPGEMM_INDEX_I32 ? sg::launch_analyze<int32_t>(*P) : sg::launch_analyze<int64_t>(*P);
    if (e == cudaSuccess) e = sg::launch_binning(*P);
    if (e == cudaSuccess) e = cudaMemsetAsync(rowptrC + P->R, 0, sizeof(int64_t), s);
    if (e == cudaSuccess)
        e = P->it == SPGEMM_INDEX_I32 ? sg::launch_symbolic<int32_t>(*P, w, rowptrC)
                                      : sg::launch_symbolic<int64_t>(*P, w, rowptrC);
    sg::WsLayout L = sg::workspace_layout(*P);
    if (e == cudaSuccess) e = sg::launch_exclusive_scan(rowptrC, P->R + 1, (int64_t*)(w + L.scan), s);
    if (e == cudaSuccess) e = run_numeric(P, w, rowptrC, capacity, colC, valC);
    if (e != cudaSuccess) return cuda_fail(e, "execute");
    return SPGEMM_OK;
}

spgemm_status spgemm_batch_rowptrs(spgemm_plan_t P, const int64_t* rowptrC, int64_t* out) {
    if (!P || !rowptrC || !out) return fail(SPGEMM_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = sg::launch_product_rowptr(*P, rowptrC, out);
    if (e != cudaSuccess) return cuda_fail(e, "batch rowptrs");
    return SPGEMM_OK;
}

spgemm_status spgemm_check(spgemm_plan_t P) {
    if (!P) return fail(SPGEMM_ERR_INVALID_ARG, "NULL plan");
    int herr = 0;
    SG_CUDA(cudaMemcpyAsync(&herr, &P->cnt->err, sizeof(int), cudaMemcpyDeviceToHost, P->stream),
            "check: readback");
    SG_CUDA(cudaStreamSynchronize(P->stream), "check: sync");
    if (herr == sg::kDevCapacity) return fail(SPGEMM_ERR_OUT_OF_MEMORY, "C did not fit the output capacity");
    if (herr == sg::kDevArena)
        return fail(SPGEMM_ERR_NOT_SUPPORTED, "a dense row of A is longer than max_row_nnz");
    if (herr == sg::kDevTooWide)
        return fail(SPGEMM_ERR_NOT_SUPPORTED,
                    "a row with more than dense_min_flops products in a product with more "
                    "columns than the shared-memory bitmap holds");
    if (herr) return fail(SPGEMM_ERR_INTERNAL, "device check failed (code %d)", herr);
    return SPGEMM_OK;
}

void spgemm_plan_destroy(spgemm_plan_t P) { delete P; }

spgemm_status spgemm_kslice_bounds(const spgemm_csr* A, int32_t c, void* stream, int64_t* bounds) {
    g_last_error.clear();
    spgemm_status st = check_csr(A, "A", false);
    if (st != SPGEMM_OK) return st;
    if (c < 1) return fail(SPGEMM_ERR_INVALID_ARG, "slice count must be >= 1");
    if (A->rowend) return fail(SPGEMM_ERR_INVALID_ARG, "A must be a plain CSR (rowend NULL)");
    if (!bounds && A->nrows > 0) return fail(SPGEMM_ERR_INVALID_ARG, "bounds is NULL");
    int sms = device_sm_count(nullptr);
    cudaError_t e = A->index_type == SPGEMM_INDEX_I32
                        ? sg::launch_kslice_bounds<int32_t>(*A, c, bounds, sms, (cudaStream_t)stream)
                        : sg::launch_kslice_bounds<int64_t>(*A, c, bounds, sms, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "kslice_bounds");
    return SPGEMM_OK;
}

size_t spgemm_merge_workspace_size(int32_t c, int64_t m, int64_t n) {
    (void)c;
    (void)n;
    if (m < 0) m = 0;
    return align_up(sizeof(sg::DevCounters)) + align_up(sg::scan_temp_bytes(m + 1));
}


spgemm_status spgemm_merge_symbolic(int32_t c, const spgemm_csr* parts, const spgemm_opts* opts,
                                    void* stream, void* ws, size_t ws_bytes, int64_t* rowptrC,
                                    int64_t* nnz_c) {
    g_last_error.clear();
    int vt = 0;
    spgemm_status st = sg::check_merge_parts(c, parts, opts, &vt);
    if (st != SPGEMM_OK) return st;
    if (!rowptrC || !nnz_c) return fail(SPGEMM_ERR_INVALID_ARG, "NULL output");
    const long long m = parts[0].nrows, n = parts[0].ncols;
    const size_t need = spgemm_merge_workspace_size(c, m, n);
    if (!ws || ws_bytes < need)
        return fail(SPGEMM_ERR_OUT_OF_MEMORY, "merge workspace %zu bytes < %zu required", ws_bytes, need);
    if (((uintptr_t)ws) % kAlign) return fail(SPGEMM_ERR_INVALID_ARG, "workspace not aligned");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* w = (unsigned char*)ws;
    sg::DevCounters* cnt = (sg::DevCounters*)w;
    int64_t* temp = (int64_t*)(w + align_up(sizeof(sg::DevCounters)));
    int sms = device_sm_count(nullptr);
    SG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(sg::DevCounters), s), "merge: memset");
    SG_CUDA(cudaMemsetAsync(rowptrC + m, 0, sizeof(int64_t), s), "merge: memset");
    cudaError_t e = sg::launch_merge(c, parts, vt, m, n, sms, s, false, rowptrC, nullptr, nullptr,
                                     nullptr, &cnt->err, &cnt->work_counter[0]);
    if (e != cudaSuccess) return cuda_fail(e, "merge symbolic");
    e = sg::launch_exclusive_scan(rowptrC, m + 1, temp, s);
    if (e != cudaSuccess) return cuda_fail(e, "merge symbolic: scan");
    int64_t total = 0;
    SG_CUDA(cudaMemcpyAsync(&total, rowptrC + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
            "merge: readback");
    SG_CUDA(cudaStreamSynchronize(s), "merge: sync");
    *nnz_c = total;
    return SPGEMM_OK;
}

spgemm_status spgemm_merge_numeric(int32_t c, const spgemm_csr* parts, const spgemm_opts* opts,
                                   void* stream, void* ws, size_t ws_bytes,
                                   const int64_t* rowptrC, void* colC, void* valC) {
    g_last_error.clear();
    int vt = 0;
    spgemm_status st = sg::check_merge_parts(c, parts, opts, &vt);
    if (st != SPGEMM_OK) return st;
    if (!rowptrC) return fail(SPGEMM_ERR_INVALID_ARG, "rowptrC is NULL");
    const long long m = parts[0].nrows, n = parts[0].ncols;
    const size_t need = spgemm_merge_workspace_size(c, m, n);
    if (!ws || ws_bytes < need)
        return fail(SPGEMM_ERR_OUT_OF_MEMORY, "merge workspace %zu bytes < %zu required", ws_bytes, need);
    if (((uintptr_t)ws) % kAlign) return fail(SPGEMM_ERR_INVALID_ARG, "workspace not aligned");
    if (!colC && m > 0) return fail(SPGEMM_ERR_INVALID_ARG, "colC is NULL");
    if (vt != SPGEMM_BOOL && !valC && m > 0) return fail(SPGEMM_ERR_INVALID_ARG, "valC is NULL");
    sg::DevCounters* cnt = (sg::DevCounters*)ws;
    int sms = device_sm_count(nullptr);
    SG_CUDA(cudaMemsetAsync(&cnt->work_counter[1], 0, sizeof(unsigned long long),
                            (cudaStream_t)stream), "merge: memset");
    const bool staged = opts && opts->merge_staged;
    cudaError_t e = sg::launch_merge(c, parts, vt, m, n, sms, (cudaStream_t)stream, true, nullptr,
                                     rowptrC, colC, valC, &cnt->err, &cnt->work_counter[1],
                                     staged);
    if (e != cudaSuccess) return cuda_fail(e, "merge numeric");
    return SPGEMM_OK;
}

spgemm_status spgemm_merge_check(void* stream, void* ws) {
    if (!ws) return fail(SPGEMM_ERR_INVALID_ARG, "workspace is NULL");
    int herr = 0;
    SG_CUDA(cudaMemcpyAsync(&herr, &((sg::DevCounters*)ws)->err, sizeof(int), cudaMemcpyDeviceToHost,
                            (cudaStream_t)stream), "merge check");
    SG_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "merge check");
    if (herr == sg::kDevWaitTimeout)
        return fail(SPGEMM_ERR_TIMEOUT, "a staged merge waited longer than its bound for a copy");
    if (herr) return fail(SPGEMM_ERR_INTERNAL, "device check failed in merge (code %d)", herr);
    return SPGEMM_OK;
}

}  // extern "C"
