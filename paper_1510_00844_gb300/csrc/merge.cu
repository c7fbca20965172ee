// Sum of c partial products C = sum_s C_s, entries with equal (i, j) added in
// ascending s: the result of the paper's multiway merge with duplicate
// reduction (Sec. 4.3), used for the LocalMerge of the k-slice partials
// (Alg. 2).  The paper merges sorted triple lists with a heap of size c; here
// one warp owns a row and sweeps its column range in chunks of W columns: for
// each chunk it streams the chunk's part of every list in order s = 0..c-1
// (a list has distinct columns, so one round never repeats a slot) into a
// dense accumulator with a presence bitmap, then emits the chunk in column
// order.  Chunks no list touches are skipped by jumping to the smallest next
// column over the c cursors (lane s holds the cursor of list s).  Up to eight
// lists take merge_win_kernel, which keeps every list's next entries in
// flight; more lists take merge_kernel.
#include "plan.h"

namespace sg {

constexpr int kMaxMergeParts = 32;

template <class IT, class V>
struct MergeParts {
    const int64_t* rp[kMaxMergeParts];
    const int64_t* re[kMaxMergeParts];
    const IT* col[kMaxMergeParts];
    const V* val[kMaxMergeParts];
};

template <class IT, class V, int W, int WARPS, bool NUMERIC>
__global__ void __launch_bounds__(WARPS * 32)
    merge_kernel(int c, MergeParts<IT, V> parts, long long m, long long n,
                 int64_t* __restrict__ rowcnt, const int64_t* __restrict__ rpC,
                 IT* __restrict__ ciC, V* __restrict__ vC, int* err) {
    constexpr bool HV = NUMERIC && VOps<V>::has_val;
    constexpr int NWORDS = W / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const int w = threadIdx.x >> 5;
    constexpr size_t vbytes = HV ? sizeof(V) * W : 0;
    unsigned char* base = smem_raw + (size_t)w * (vbytes + W / 8);
    V* acc = reinterpret_cast<V*>(base);
    unsigned* bm = reinterpret_cast<unsigned*>(base + vbytes);
    for (int s = lane; s < W; s += 32)
        if constexpr (HV) acc[s] = VOps<V>::init();
    for (int t = lane; t < NWORDS; t += 32) bm[t] = 0u;
    __syncwarp();
    const long long gw = (long long)blockIdx.x * WARPS + w;
    const long long nw = (long long)gridDim.x * WARPS;
    for (long long i = gw; i < m; i += nw) {
        long long cur = 0, end = 0;
        if (lane < c) {
            cur = parts.rp[lane][i];
            end = parts.re[lane] ? parts.re[lane][i] : parts.rp[lane][i + 1];
        }
        long long out = NUMERIC ? rpC[i] : 0;
        const long long out_end = NUMERIC ? rpC[i + 1] : 0;
        long long count = 0;
        while (true) {
            long long nxt = (lane < c && cur < end) ? (long long)parts.col[lane][cur] : n;
            nxt = -warp_max(-nxt);  // warp min
            if (nxt >= n) break;
            const long long c0 = (nxt / W) * W;
            const long long c1 = min(c0 + (long long)W, n);
            for (int s = 0; s < c; ++s) {
                long long q0 = __shfl_sync(kFull, cur, s);
                const long long qe = __shfl_sync(kFull, end, s);
                const IT* col = parts.col[s];
                const V* val = parts.val[s];
                while (q0 < qe) {
                    long long q = q0 + lane;
                    bool valid = q < qe;
                    long long j = valid ? (long long)col[q] : c1;
                    valid = valid && j < c1;
                    int slot = (int)(j - c0);
                    if (valid) {
                        atomicOr(&bm[slot >> 5], 1u << (slot & 31));
                        if constexpr (HV) acc[slot] = VOps<V>::add(acc[slot], val[q]);
                    }
                    __syncwarp();
                    int got = __popc(__ballot_sync(kFull, valid));
                    q0 += got;
                    if (got < 32) break;
                }
                if (lane == s) cur = q0;
            }
            __syncwarp();
            // emit (numeric) or count (symbolic) the chunk, clearing it
            for (int t0 = 0; t0 < NWORDS; t0 += 32) {
                const int t = t0 + lane;
                unsigned word = t < NWORDS ? bm[t] : 0u;
                int pc = __popc(word);
                int incl = warp_incl_scan(pc);
                int tot = __shfl_sync(kFull, incl, 31);
                if constexpr (NUMERIC) {
                    long long pos = out + incl - pc;
                    while (word) {
                        int b = __ffs(word) - 1;
                        word &= word - 1;
                        int slot = t * 32 + b;
                        if (pos < out_end) {
                            ciC[pos] = (IT)(c0 + slot);
                            if constexpr (HV) vC[pos] = acc[slot];
                        }
                        if constexpr (HV) acc[slot] = VOps<V>::init();
                        ++pos;
                    }
                }
                if (t < NWORDS) bm[t] = 0u;
                out += tot;
                count += tot;
            }
            __syncwarp();
        }
        if constexpr (!NUMERIC) {
            if (lane == 0) rowcnt[i] = count;
        } else {
            if (lane == 0 && out != out_end) atomicExch(err, (int)kDevCountMismatch);
        }
    }
}

// The same sum for c <= CM lists with the loads of every list in flight
// together.  Each list keeps two windows of 32 consecutive entries in
// registers (lane x holds entry x of each): the window being consumed and
// the next one, whose loads are issued as soon as the previous window comes
// into use, so a list's next entries arrive while the current ones are
// accumulated.  Entries are consumed in column order chunk by chunk: the
// entries of list s inside the chunk are a prefix of what is left of its
// window (columns ascend), so one ballot per list and window step covers them.
template <class IT, class V, int W, int WARPS, bool NUMERIC, int CM>
__global__ void __launch_bounds__(WARPS * 32)
    merge_win_kernel(int c, MergeParts<IT, V> parts, long long m, long long n,
                     int64_t* __restrict__ rowcnt, const int64_t* __restrict__ rpC,
                     IT* __restrict__ ciC, V* __restrict__ vC, int* err,
                     unsigned long long* work) {
    constexpr bool HV = NUMERIC && VOps<V>::has_val;
    constexpr int NWORDS = W / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const int w = threadIdx.x >> 5;
    constexpr size_t vbytes = HV ? sizeof(V) * W : 0;
    unsigned char* base = smem_raw + (size_t)w * (vbytes + W / 8);
    V* acc = reinterpret_cast<V*>(base);
    unsigned* bm = reinterpret_cast<unsigned*>(base + vbytes);
    for (int s = lane; s < W; s += 32)
        if constexpr (HV) acc[s] = VOps<V>::init();
    for (int t = lane; t < NWORDS; t += 32) bm[t] = 0u;
    __syncwarp();
    // rows are taken one at a time from a counter: row sizes are heavy-tailed,
    // so a fixed stride would leave some warps with far more work
    while (true) {
        long long i = 0;
        if (lane == 0) i = (long long)atomicAdd(work, 1ull);
        i = __shfl_sync(kFull, i, 0);
        if (i >= m) break;
        long long b_own = 0, e_own = 0;
        if (lane < c) {
            b_own = parts.rp[lane][i];
            e_own = parts.re[lane] ? parts.re[lane][i] : parts.rp[lane][i + 1];
        }
        long long wb[CM];  // position of window A's first entry (warp-uniform)
        long long we[CM];  // end of list s in row i
        int off[CM];       // entries of window A already consumed
        long long ja[CM], jb[CM];
        V va[CM], vb[CM];
#pragma unroll
        for (int s = 0; s < CM; ++s) {
            wb[s] = __shfl_sync(kFull, b_own, s);
            we[s] = s < c ? __shfl_sync(kFull, e_own, s) : 0;
            off[s] = 0;
            const long long qa = wb[s] + lane, qb = qa + 32;
            ja[s] = qa < we[s] ? (long long)parts.col[s][qa] : n;
            jb[s] = qb < we[s] ? (long long)parts.col[s][qb] : n;
            va[s] = V{};
            vb[s] = V{};
            if constexpr (HV) {
                if (qa < we[s]) va[s] = parts.val[s][qa];
                if (qb < we[s]) vb[s] = parts.val[s][qb];
            }
        }
        long long out = NUMERIC ? rpC[i] : 0;
        const long long out_end = NUMERIC ? rpC[i + 1] : 0;
        long long count = 0;
        while (true) {
            long long nxt = n;
#pragma unroll
            for (int s = 0; s < CM; ++s) {
                const long long h = __shfl_sync(kFull, ja[s], off[s] & 31);
                if (wb[s] + off[s] < we[s]) nxt = min(nxt, h);
            }
            if (nxt >= n) break;
            const long long c0 = (nxt / W) * W;
            const long long c1 = min(c0 + (long long)W, n);
#pragma unroll
            for (int s = 0; s < CM; ++s) {
                while (true) {
                    const bool valid = lane >= off[s] && ja[s] < c1;
                    const int slot = (int)(ja[s] - c0);
                    if (valid) {
                        atomicOr(&bm[slot >> 5], 1u << (slot & 31));
                        if constexpr (HV) acc[slot] = VOps<V>::add(acc[slot], va[s]);
                    }
                    __syncwarp();
                    off[s] += __popc(__ballot_sync(kFull, valid));
                    if (off[s] < 32) break;
                    // window A used up: B moves in, the window after B is loaded
                    wb[s] += 32;
                    off[s] = 0;
                    ja[s] = jb[s];
                    va[s] = vb[s];
                    const long long qb = wb[s] + 32 + lane;
                    jb[s] = qb < we[s] ? (long long)parts.col[s][qb] : n;
                    if constexpr (HV)
                        if (qb < we[s]) vb[s] = parts.val[s][qb];
                    if (wb[s] >= we[s]) break;
                }
            }
            // emit (numeric) or count (symbolic) the chunk, clearing it
            for (int t0 = 0; t0 < NWORDS; t0 += 32) {
                const int t = t0 + lane;
                unsigned word = t < NWORDS ? bm[t] : 0u;
                const int pc = __popc(word);
                const int incl = warp_incl_scan(pc);
                const int tot = __shfl_sync(kFull, incl, 31);
                if constexpr (NUMERIC) {
                    long long pos = out + incl - pc;
                    while (word) {
                        const int b = __ffs(word) - 1;
                        word &= word - 1;
                        const int slot = t * 32 + b;
                        if (pos < out_end) {
                            ciC[pos] = (IT)(c0 + slot);
                            if constexpr (HV) vC[pos] = acc[slot];
                        }
                        if constexpr (HV) acc[slot] = VOps<V>::init();
                        ++pos;
                    }
                }
                if (t < NWORDS) bm[t] = 0u;
                out += tot;
                count += tot;
            }
            __syncwarp();
        }
        if constexpr (!NUMERIC) {
            if (lane == 0) rowcnt[i] = count;
        } else {
            if (lane == 0 && out != out_end) atomicExch(err, (int)kDevCountMismatch);
        }
    }
}

template <class IT, class V, bool NUMERIC>
cudaError_t launch_merge_t(int c, const spgemm_csr* parts, long long m, long long n,
                           int sm_count, cudaStream_t s, int64_t* rowcnt, const int64_t* rpC,
                           void* colC, void* valC, int* err, unsigned long long* work) {
    MergeParts<IT, V> mp{};
    for (int t = 0; t < c; ++t) {
        mp.rp[t] = parts[t].rowptr;
        mp.re[t] = parts[t].rowend;
        mp.col[t] = (const IT*)parts[t].col;
        mp.val[t] = (const V*)parts[t].val;
    }
    if (c <= 8) {
        // the count keeps only a bitmap, so its chunks can be wider
        constexpr int W = NUMERIC ? 1024 : 8192, WARPS = 8;
        auto k = c <= 2   ? merge_win_kernel<IT, V, W, WARPS, NUMERIC, 2>
                 : c <= 4 ? merge_win_kernel<IT, V, W, WARPS, NUMERIC, 4>
                          : merge_win_kernel<IT, V, W, WARPS, NUMERIC, 8>;
        constexpr size_t vb = (NUMERIC && VOps<V>::has_val) ? sizeof(V) : 0;
        const size_t smem = (size_t)WARPS * (W * vb + W / 8);
        if (smem > 48 * 1024) {
            cudaError_t e =
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        int occ = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, WARPS * 32, smem);
        if (occ < 1) occ = 1;
        const long long need = (m + WARPS - 1) / WARPS;
        const long long g = std::max<long long>(1, std::min(need, (long long)sm_count * occ));
        if (m > 0) {
            count_launches(1);
            k<<<(unsigned)g, WARPS * 32, smem, s>>>(c, mp, m, n, rowcnt, rpC, (IT*)colC,
                                                    (V*)valC, err, work);
        }
        return cudaGetLastError();
    }
    constexpr int W = 2048, WARPS = 4;
    auto k = merge_kernel<IT, V, W, WARPS, NUMERIC>;
    constexpr size_t vb = (NUMERIC && VOps<V>::has_val) ? sizeof(V) : 0;
    size_t smem = (size_t)WARPS * (W * vb + W / 8);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, WARPS * 32, smem);
    if (occ < 1) occ = 1;
    long long need = (m + WARPS - 1) / WARPS;
    long long g = std::max<long long>(1, std::min(need, (long long)sm_count * occ));
    if (m > 0) {
        count_launches(1);
        k<<<(unsigned)g, WARPS * 32, smem, s>>>(c, mp, m, n, rowcnt, rpC, (IT*)colC, (V*)valC, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_merge(int c, const spgemm_csr* parts, int vt, long long m, long long n,
                         int sm_count, cudaStream_t s, bool numeric, int64_t* rowcnt,
                         const int64_t* rpC, void* colC, void* valC, int* err,
                         unsigned long long* work) {
    const bool i32 = parts[0].index_type == SPGEMM_INDEX_I32;
#define SG_MERGE_CASE(V)                                                                         \
    return numeric ? (i32 ? launch_merge_t<int32_t, V, true>(c, parts, m, n, sm_count, s, rowcnt, \
                                                             rpC, colC, valC, err, work)                \
                          : launch_merge_t<int64_t, V, true>(c, parts, m, n, sm_count, s, rowcnt, \
                                                             rpC, colC, valC, err, work))               \
                   : (i32 ? launch_merge_t<int32_t, V, false>(c, parts, m, n, sm_count, s,       \
                                                              rowcnt, rpC, colC, valC, err, work)      \
                          : launch_merge_t<int64_t, V, false>(c, parts, m, n, sm_count, s,       \
                                                              rowcnt, rpC, colC, valC, err, work));
    return with_value_type(vt, [&](auto tag) -> cudaError_t {
        using V = decltype(tag);
        SG_MERGE_CASE(V)
    });
#undef SG_MERGE_CASE
}

}  // namespace sg
