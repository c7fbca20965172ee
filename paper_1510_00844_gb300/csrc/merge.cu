// Sum of c partial products C = sum_s C_s, entries with equal (i, j) added in
// ascending s: the result of the paper's multiway merge with duplicate
// reduction (Sec. 4.3), used for the LocalMerge of the k-slice partials
// (Alg. 2).  The paper merges sorted triple lists with a heap of size c; here
// one warp owns a row and sweeps its column range in chunks of W columns: for
// each chunk it streams the chunk's part of every list in order s = 0..c-1
// (a list has distinct columns, so one round never repeats a slot) into a
// dense accumulator with a presence bitmap, then emits the chunk in column
// order.  Chunks no list touches are skipped by jumping to the smallest next
// column over the c cursors (lane s holds the cursor of list s).
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

template <class IT, class V, bool NUMERIC>
cudaError_t launch_merge_t(int c, const spgemm_csr* parts, long long m, long long n,
                           int sm_count, cudaStream_t s, int64_t* rowcnt, const int64_t* rpC,
                           void* colC, void* valC, int* err) {
    constexpr int W = 2048, WARPS = 4;
    MergeParts<IT, V> mp{};
    for (int t = 0; t < c; ++t) {
        mp.rp[t] = parts[t].rowptr;
        mp.re[t] = parts[t].rowend;
        mp.col[t] = (const IT*)parts[t].col;
        mp.val[t] = (const V*)parts[t].val;
    }
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
                         const int64_t* rpC, void* colC, void* valC, int* err) {
    const bool i32 = parts[0].index_type == SPGEMM_INDEX_I32;
#define SG_MERGE_CASE(V)                                                                         \
    return numeric ? (i32 ? launch_merge_t<int32_t, V, true>(c, parts, m, n, sm_count, s, rowcnt, \
                                                             rpC, colC, valC, err)                \
                          : launch_merge_t<int64_t, V, true>(c, parts, m, n, sm_count, s, rowcnt, \
                                                             rpC, colC, valC, err))               \
                   : (i32 ? launch_merge_t<int32_t, V, false>(c, parts, m, n, sm_count, s,       \
                                                              rowcnt, rpC, colC, valC, err)      \
                          : launch_merge_t<int64_t, V, false>(c, parts, m, n, sm_count, s,       \
                                                              rowcnt, rpC, colC, valC, err));
    return with_value_type(vt, [&](auto tag) -> cudaError_t {
        using V = decltype(tag);
        SG_MERGE_CASE(V)
    });
#undef SG_MERGE_CASE
}

}  // namespace sg
