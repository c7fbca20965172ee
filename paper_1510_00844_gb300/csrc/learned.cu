// Learned sizing of C (not in the paper): the row-size predictor, evaluated
// inside the row analysis, replaces the symbolic phase for hash-class rows.
//
//   1. plan with the predictor: every row gets a predicted capacity; rows of
//      at most dense_min products are binned by that capacity;
//   2. slots: the capacities are scanned into slot offsets (no symbolic pass
//      for any row);
//   3. numeric: every row is multiplied straight into its slot (same kernels,
//      same ascending-k order as the two-phase path); a dense row's segments
//      each take a share of the slot in proportion to their column chunks and
//      are packed together afterwards; a row that does not fit its slot, its
//      share or its hash table is listed instead of written;
//   4. listed rows are multiplied again by the exact two-phase path, and C is
//      assembled: with no listed row the slots already form C (row i spans
//      [slot_i, rowend_i)); listed rows whose exact output fits the spare
//      space kept after the slots are written there (their slot start moves,
//      C stays in slot form); otherwise rows are compacted into a plain CSR.
// Row contents are identical to the two-phase result in every case.
//
// Device memory comes from a caller callback (spgemm_alloc_fn), since sizes
// are only known step by step.
#include <cstdio>

#include "plan.h"

namespace sg {

// rowend of the rows with no products.
__global__ void fill_rowend_kernel(long long R, const unsigned char* __restrict__ cls,
                                   const int64_t* __restrict__ slots, int64_t* __restrict__ rowend) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < R;
         r += (long long)gridDim.x * blockDim.x) {
        if (cls[r] == kClassEmpty) rowend[r] = slots[r];
    }
}

// Row view of the listed rows of A (single product): rp/re of each listed row.
__global__ void gather_rows_kernel(long long cnt, const int32_t* __restrict__ list,
                                   const int64_t* __restrict__ rpA, const int64_t* __restrict__ reA,
                                   int64_t* __restrict__ rp_sub, int64_t* __restrict__ re_sub,
                                   int32_t* __restrict__ inv) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = list[t];
        rp_sub[t] = rpA[r];
        re_sub[t] = reA ? reA[r] : rpA[r + 1];
        inv[r] = (int32_t)t;
    }
}

// Listed rows re-run into the spare space at `base`: new slot start and end.
__global__ void relocate_rows_kernel(long long cnt, const int32_t* __restrict__ list,
                                     const int64_t* __restrict__ rp_x, long long base,
                                     int64_t* __restrict__ slots, int64_t* __restrict__ rowend) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = list[t];
        slots[r] = base + rp_x[t];
        rowend[r] = base + rp_x[t + 1];
    }
}

// Final row counts: slot rows from rowend, listed rows from the re-run.
__global__ void final_counts_kernel(long long R, const int64_t* __restrict__ slots,
                                    const int64_t* __restrict__ rowend,
                                    const int32_t* __restrict__ inv,
                                    const int64_t* __restrict__ rp_x, int64_t* __restrict__ cnt) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < R;
         r += (long long)gridDim.x * blockDim.x) {
        const int t = inv[r];
        cnt[r] = t >= 0 ? rp_x[t + 1] - rp_x[t] : rowend[r] - slots[r];
    }
}

// Compaction: one warp per row copies it from its slot or from the re-run.
template <class IT, class V>
__global__ void compact_kernel(long long R, const int64_t* __restrict__ slots,
                               const int32_t* __restrict__ inv, const int64_t* __restrict__ rp_x,
                               const IT* __restrict__ col_s, const V* __restrict__ val_s,
                               const IT* __restrict__ col_x, const V* __restrict__ val_x,
                               const int64_t* __restrict__ rp_f, IT* __restrict__ col_f,
                               V* __restrict__ val_f) {
    const int lane = lane_id();
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = warp; r < R; r += nwarps) {
        const int t = inv[r];
        const long long src = t >= 0 ? rp_x[t] : slots[r];
        const IT* cs = t >= 0 ? col_x : col_s;
        const V* vs = t >= 0 ? val_x : val_s;
        const long long dst = rp_f[r];
        const long long L = rp_f[r + 1] - dst;
        for (long long q = lane; q < L; q += 32) {
            col_f[dst + q] = cs[src + q];
            if constexpr (VOps<V>::has_val) val_f[dst + q] = vs[src + q];
        }
    }
}

template <class IT, class V>
cudaError_t launch_compact(long long R, int sms, cudaStream_t s, const int64_t* slots,
                           const int32_t* inv, const int64_t* rp_x, const void* col_s,
                           const void* val_s, const void* col_x, const void* val_x,
                           const int64_t* rp_f, void* col_f, void* val_f) {
    const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>((R + 7) / 8, (long long)sms * 8));
    count_launches(1);
    compact_kernel<IT, V><<<g, 256, 0, s>>>(R, slots, inv, rp_x, (const IT*)col_s, (const V*)val_s,
                                            (const IT*)col_x, (const V*)val_x, rp_f, (IT*)col_f,
                                            (V*)val_f);
    return cudaGetLastError();
}

}  // namespace sg

namespace {

size_t al(size_t x) { return (x + 255) / 256 * 256; }

spgemm_status lfail(spgemm_status st, const char* msg) {
    sg::set_last_error(msg);
    return st;
}

spgemm_status lcuda(cudaError_t e, const char* where) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: CUDA error %d (%s)", where, (int)e, cudaGetErrorString(e));
    sg::set_last_error(buf);
    return SPGEMM_ERR_CUDA;
}

}  // namespace

extern "C" {

spgemm_status spgemm_row_features(spgemm_plan_t P, float* X) {
    if (!P || (!X && P->R > 0)) return lfail(SPGEMM_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = P->it == SPGEMM_INDEX_I32 ? sg::launch_row_features<int32_t>(*P, X)
                                              : sg::launch_row_features<int64_t>(*P, X);
    if (e != cudaSuccess) return lcuda(e, "row features");
    return SPGEMM_OK;
}

spgemm_status spgemm_learned_multiply(const spgemm_csr* A, const spgemm_csr* B,
                                      const spgemm_opts* opts, const float* params, float margin,
                                      void* stream, spgemm_alloc_fn alloc, void* ctx,
                                      spgemm_learned_result* out) {
    if (!A || !B || !params || !alloc || !out) return lfail(SPGEMM_ERR_INVALID_ARG, "NULL argument");
    *out = spgemm_learned_result{};
    cudaStream_t s = (cudaStream_t)stream;
    const long long m = A->nrows;
    auto get = [&](size_t bytes) -> unsigned char* { return (unsigned char*)alloc(std::max<size_t>(bytes, 256), ctx); };
    // 1. plan with the predictor
    unsigned char* pws = get(sg::plan_workspace_bytes(1, m));
    if (!pws) return lfail(SPGEMM_ERR_OUT_OF_MEMORY, "allocation callback failed");
    spgemm_plan_t P = nullptr;
    spgemm_status st = sg::make_plan(1, A, B, opts, stream, pws, sg::plan_workspace_bytes(1, m),
                                     false, &P, params, margin);
    if (st != SPGEMM_OK) return st;
    struct Guard {
        spgemm_plan_t p;
        ~Guard() { spgemm_plan_destroy(p); }
    } guard{P};
    const size_t isz = P->it == SPGEMM_INDEX_I32 ? 4 : 8;
    const size_t vsz = sg::vt_bytes(P->vt);
    sg::WsLayout L = sg::workspace_layout(*P);
    unsigned char* ws = get(L.total + al(sizeof(unsigned)) + al((size_t)m * 4) + al((size_t)m * 4));
    if (!ws) return lfail(SPGEMM_ERR_OUT_OF_MEMORY, "allocation callback failed");
    unsigned* ocount = (unsigned*)(ws + L.total);
    int32_t* olist = (int32_t*)(ws + L.total + al(sizeof(unsigned)));
    int32_t* inv = (int32_t*)(ws + L.total + al(sizeof(unsigned)) + al((size_t)m * 4));
    // 2. slots: predicted capacities of all rows
    int64_t* slots = (int64_t*)get((size_t)(m + 1) * 8);
    const long long units = sg::dense_unit_count(*P);
    int64_t* unit_cnt = (int64_t*)get((size_t)std::max<long long>(units, 1) * 8);
    if (!slots || !unit_cnt) return lfail(SPGEMM_ERR_OUT_OF_MEMORY, "allocation callback failed");
    P->unit_cnt = unit_cnt;
    cudaError_t e = cudaSuccess;
    if (m > 0) e = cudaMemcpyAsync(slots, P->cap, (size_t)m * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(slots + m, 0, 8, s);
    if (e == cudaSuccess && units > 0) e = cudaMemsetAsync(unit_cnt, 0, (size_t)units * 8, s);
    if (e == cudaSuccess && P->ndense > 0)  // the tables the dense numeric kernel walks with
        e = P->it == SPGEMM_INDEX_I32 ? sg::launch_dense_tables<int32_t>(*P, ws)
                                      : sg::launch_dense_tables<int64_t>(*P, ws);
    if (e == cudaSuccess) e = sg::launch_exclusive_scan(slots, m + 1, (int64_t*)(ws + L.scan), s);
    long long total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, slots + m, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return lcuda(e, "learned: slots");
    // 3. numeric into the slots (with spare space after them for re-run rows)
    const long long spare = total / 32 + 65536;
    int64_t* rowend = (int64_t*)get((size_t)std::max<long long>(m, 1) * 8);
    unsigned char* col = get((size_t)(total + spare) * isz);
    unsigned char* val = vsz ? get((size_t)(total + spare) * vsz) : nullptr;
    if (!rowend || !col || (vsz && !val)) return lfail(SPGEMM_ERR_OUT_OF_MEMORY, "allocation callback failed");
    e = cudaMemsetAsync(ocount, 0, sizeof(unsigned), s);
    if (e == cudaSuccess && m > 0) e = cudaMemsetAsync(rowend, 0, (size_t)m * 8, s);
    if (e == cudaSuccess) {
        const bool i32 = P->it == SPGEMM_INDEX_I32;
        e = sg::with_value_type(P->vt, [&](auto tag) -> cudaError_t {
            using V = decltype(tag);
            void* vv = sg::VOps<V>::has_val ? (void*)val : nullptr;
            return i32 ? sg::launch_numeric<int32_t, V>(*P, ws, slots, total, col, vv, rowend, olist, ocount)
                       : sg::launch_numeric<int64_t, V>(*P, ws, slots, total, col, vv, rowend, olist, ocount);
        });
    }
    if (e == cudaSuccess && P->ndense > 0) {
        const bool i32 = P->it == SPGEMM_INDEX_I32;
        e = sg::with_value_type(P->vt, [&](auto tag) -> cudaError_t {
            using V = decltype(tag);
            void* vv = sg::VOps<V>::has_val ? (void*)val : nullptr;
            return i32 ? sg::launch_dense_slot_pack<int32_t, V>(*P, slots, col, vv, rowend)
                       : sg::launch_dense_slot_pack<int64_t, V>(*P, slots, col, vv, rowend);
        });
    }
    if (e == cudaSuccess && m > 0) {
        const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>((m + 255) / 256, (long long)P->sm_count * 8));
        sg::count_launches(1);
        sg::fill_rowend_kernel<<<g, 256, 0, s>>>(m, P->cls, slots, rowend);
        e = cudaGetLastError();
    }
    unsigned nover = 0;
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nover, ocount, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, &P->cnt->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return lcuda(e, "learned: numeric");
    if (herr) return lfail(SPGEMM_ERR_INTERNAL, "device check failed in the learned numeric phase");
    out->nrows = m;
    out->ncols = B->ncols;
    out->slot_total = total;
    out->overflow_rows = nover;
    out->total_flops = P->total_flops;
    if (nover == 0) {  // the slots are C
        out->rowptr = slots;
        out->rowend = rowend;
        out->col = col;
        out->val = val;
        out->nnz = total;  // entries of the col/val arrays (slots may have gaps)
        return SPGEMM_OK;
    }
    // 4. exact re-run of the listed rows, then compaction
    int64_t* rp_sub = (int64_t*)get((size_t)nover * 8);
    int64_t* re_sub = (int64_t*)get((size_t)nover * 8);
    if (!rp_sub || !re_sub) return lfail(SPGEMM_ERR_OUT_OF_MEMORY, "allocation callback failed");
    e = cudaMemsetAsync(inv, 0xff, (size_t)m * 4, s);
    if (e == cudaSuccess) {
        sg::count_launches(1);
        sg::gather_rows_kernel<<<(nover + 255) / 256, 256, 0, s>>>(nover, olist, A->rowptr, A->rowend,
                                                                    rp_sub, re_sub, inv);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return lcuda(e, "learned: gather");
    spgemm_csr Asub = *A;
    Asub.nrows = nover;
    Asub.rowptr = rp_sub;
    Asub.rowend = re_sub;
    spgemm_opts o{};
    if (opts) o = *opts;
    o.checked = 0;
    unsigned char* pws2 = get(sg::plan_workspace_bytes(1, nover));
    if (!pws2) return lfail(SPGEMM_ERR_OUT_OF_MEMORY, "allocation callback failed");
    spgemm_plan_t P2 = nullptr;
    st = spgemm_plan(&Asub, B, &o, stream, pws2, sg::plan_workspace_bytes(1, nover), &P2);
    if (st != SPGEMM_OK) return st;
    struct Guard2 {
        spgemm_plan_t p;
        ~Guard2() { spgemm_plan_destroy(p); }
    } guard2{P2};
    size_t ws2b = 0;
    spgemm_workspace_size(P2, &ws2b);
    unsigned char* ws2 = get(ws2b);
    int64_t* rp_x = (int64_t*)get((size_t)(nover + 1) * 8);
    if (!ws2 || !rp_x) return lfail(SPGEMM_ERR_OUT_OF_MEMORY, "allocation callback failed");
    int64_t nnz_x = 0;
    if ((st = spgemm_symbolic(P2, ws2, ws2b, rp_x, &nnz_x)) != SPGEMM_OK) return st;
    if (nnz_x <= spare) {  // re-run rows go to the spare space; C stays in slot form
        unsigned char* col_sp = col + (size_t)total * isz;
        unsigned char* val_sp = vsz ? val + (size_t)total * vsz : nullptr;
        if ((st = spgemm_numeric(P2, ws2, ws2b, rp_x, col_sp, val_sp)) != SPGEMM_OK) return st;
        sg::count_launches(1);
        sg::relocate_rows_kernel<<<(nover + 255) / 256, 256, 0, s>>>(nover, olist, rp_x, total,
                                                                      slots, rowend);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return lcuda(e, "learned: relocate");
        out->rowptr = slots;
        out->rowend = rowend;
        out->col = col;
        out->val = val;
        out->nnz = total + nnz_x;
        return SPGEMM_OK;
    }
    unsigned char* col_x = get((size_t)nnz_x * isz);
    unsigned char* val_x = vsz ? get((size_t)nnz_x * vsz) : nullptr;
    if (!col_x || (vsz && !val_x)) return lfail(SPGEMM_ERR_OUT_OF_MEMORY, "allocation callback failed");
    if ((st = spgemm_numeric(P2, ws2, ws2b, rp_x, col_x, val_x)) != SPGEMM_OK) return st;
    int64_t* rp_f = (int64_t*)get((size_t)(m + 1) * 8);
    if (!rp_f) return lfail(SPGEMM_ERR_OUT_OF_MEMORY, "allocation callback failed");
    const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>((m + 255) / 256, (long long)P->sm_count * 8));
    sg::count_launches(1);
    sg::final_counts_kernel<<<g, 256, 0, s>>>(m, slots, rowend, inv, rp_x, rp_f);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(rp_f + m, 0, 8, s);
    if (e == cudaSuccess) e = sg::launch_exclusive_scan(rp_f, m + 1, (int64_t*)(ws + L.scan), s);
    long long nnz = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nnz, rp_f + m, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return lcuda(e, "learned: final counts");
    unsigned char* col_f = get((size_t)nnz * isz);
    unsigned char* val_f = vsz ? get((size_t)nnz * vsz) : nullptr;
    if (!col_f || (vsz && !val_f)) return lfail(SPGEMM_ERR_OUT_OF_MEMORY, "allocation callback failed");
    const bool i32 = P->it == SPGEMM_INDEX_I32;
    e = sg::with_value_type(P->vt, [&](auto tag) -> cudaError_t {
        using V = decltype(tag);
        const bool hv = sg::VOps<V>::has_val;
        return i32 ? sg::launch_compact<int32_t, V>(m, P->sm_count, s, slots, inv, rp_x, col,
                                                    hv ? val : nullptr, col_x, hv ? val_x : nullptr,
                                                    rp_f, col_f, hv ? val_f : nullptr)
                   : sg::launch_compact<int64_t, V>(m, P->sm_count, s, slots, inv, rp_x, col,
                                                    hv ? val : nullptr, col_x, hv ? val_x : nullptr,
                                                    rp_f, col_f, hv ? val_f : nullptr);
    });
    if (e != cudaSuccess) return lcuda(e, "learned: compaction");
    out->rowptr = rp_f;
    out->rowend = nullptr;
    out->col = col_f;
    out->val = val_f;
    out->nnz = nnz;
    return SPGEMM_OK;
}

}  // extern "C"
