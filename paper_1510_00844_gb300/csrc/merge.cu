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
// flight; more lists take merge_kernel.  The count pass of up to four int32
// lists in 16-byte aligned arrays takes merge_count4_kernel (four columns
// per lane per load).
#include <type_traits>

#include "plan.h"

namespace sg {

constexpr int kMaxMergeParts = 32;

template <class IT, class V>
struct MergeParts {
    const int64_t* rp[kMaxMergeParts];
    const int64_t* re[kMaxMergeParts];
    const IT* col[kMaxMergeParts];
    const V* val[kMaxMergeParts];
    long long len[kMaxMergeParts];  // length of col/val of part s
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
// together.  Each list keeps three windows of 32 consecutive entries in
// registers (lane x holds entry x of each): the window being consumed and
// the next two; when a window is used up the one after the last is loaded,
// so a list's next entries arrive while the current ones are accumulated.
// Entries are consumed in column order chunk by chunk: the entries of list s
// inside the chunk are a prefix of what is left of its window (columns
// ascend), so one ballot per list and window step covers them.  Rows are
// taken from a counter; the count pass only adds up the row's columns.
template <class V>
constexpr bool kStoreFirst = std::is_same<V, double>::value || std::is_same<V, float>::value ||
                             std::is_same<V, int64_t>::value;

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
        IT ja[CM], jb[CM], jc[CM];
        V va[CM], vb[CM], vc[CM];
#pragma unroll
        for (int s = 0; s < CM; ++s) {
            wb[s] = __shfl_sync(kFull, b_own, s);
            we[s] = s < c ? __shfl_sync(kFull, e_own, s) : 0;
            off[s] = 0;
            const long long qa = wb[s] + lane, qb = qa + 32, qc = qa + 64;
            ja[s] = qa < we[s] ? parts.col[s][qa] : IT(0);
            jb[s] = qb < we[s] ? parts.col[s][qb] : IT(0);
            jc[s] = qc < we[s] ? parts.col[s][qc] : IT(0);
            va[s] = V{};
            vb[s] = V{};
            vc[s] = V{};
            if constexpr (HV) {
                if (qa < we[s]) va[s] = parts.val[s][qa];
                if (qb < we[s]) vb[s] = parts.val[s][qb];
                if (qc < we[s]) vc[s] = parts.val[s][qc];
            }
        }
        long long out = NUMERIC ? rpC[i] : 0;
        const long long out_end = NUMERIC ? rpC[i + 1] : 0;
        long long count = 0;
        while (true) {
            long long nxt = n;
#pragma unroll
            for (int s = 0; s < CM; ++s) {
                const long long h = (long long)__shfl_sync(kFull, ja[s], off[s] & 31);
                if (wb[s] + off[s] < we[s]) nxt = min(nxt, h);
            }
            if (nxt >= n) break;
            const long long c0 = (nxt / W) * W;
            const long long c1 = min(c0 + (long long)W, n);
#pragma unroll
            for (int s = 0; s < CM; ++s) {
                while (true) {
                    const bool valid =
                        lane >= off[s] && wb[s] + lane < we[s] && (long long)ja[s] < c1;
                    const int slot = (int)((long long)ja[s] - c0);
                    if (valid) {
                        atomicOr(&bm[slot >> 5], 1u << (slot & 31));
                        if constexpr (HV) {
                            if (kStoreFirst<V> && s == 0) acc[slot] = va[s];
                            else acc[slot] = VOps<V>::add(acc[slot], va[s]);
                        }
                    }
                    __syncwarp();
                    off[s] += __popc(__ballot_sync(kFull, valid));
                    if (off[s] < 32) break;
                    // window A used up: B and C move up, the window after C is loaded
                    wb[s] += 32;
                    off[s] = 0;
                    ja[s] = jb[s];
                    va[s] = vb[s];
                    jb[s] = jc[s];
                    vb[s] = vc[s];
                    const long long qc = wb[s] + 64 + lane;
                    if (qc < we[s]) {
                        jc[s] = parts.col[s][qc];
                        if constexpr (HV) vc[s] = parts.val[s][qc];
                    }
                    if (wb[s] >= we[s]) break;
                }
            }
            // emit the chunk (numeric) or add up its columns (count), clearing it
            if constexpr (NUMERIC) {
                for (int t0 = 0; t0 < NWORDS; t0 += 32) {
                    const int t = t0 + lane;
                    unsigned word = t < NWORDS ? bm[t] : 0u;
                    const int pc = __popc(word);
                    const int incl = warp_incl_scan(pc);
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
                    if (t < NWORDS) bm[t] = 0u;
                    out += __shfl_sync(kFull, incl, 31);
                }
            } else {
                // only the row total is needed: per-lane counts, summed once
                for (int t = lane; t < NWORDS; t += 32) {
                    count += __popc(bm[t]);
                    bm[t] = 0u;
                }
            }
            __syncwarp();
        }
        if constexpr (!NUMERIC) {
            count = warp_sum(count);
            if (lane == 0) rowcnt[i] = count;
        } else {
            if (lane == 0 && out != out_end) atomicExch(err, (int)kDevCountMismatch);
        }
    }
}

// ------------------------------------------------ staged numeric merge
// The numeric sum for c <= CM lists whose column and value arrays start on
// 16-byte boundaries, with every list's entries staged in shared memory by
// bulk asynchronous copies (cp.async.bulk, the TMA's one-dimensional form):
// each warp keeps two buffers of WIN entries per list; while the warp
// accumulates from one, the next window of that list is in flight into the
// other, so each list has up to 2 x WIN entries in flight with no registers
// held.  A buffer's copy signals an mbarrier (transaction count = its
// bytes); the warp waits on it with a bound (a wait that exceeds the bound
// records kDevWaitTimeout, lets the copies it issued land, and ends the
// warp's work).  Windows start at multiples of four entries (16 bytes of
// int32 columns, 32 of float64 values); the last entries of an array that a
// 16-byte copy cannot reach are loaded by the lanes.  Entries are then
// consumed in column order chunk by chunk exactly as in merge_win_kernel.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// One arrival that also expects `bytes` of asynchronous copies.
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_to_shared(void* dst, const void* src, unsigned bytes,
                                               unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

constexpr unsigned long long kMergeWaitNs = 2000000000ull;   // 2 s

// Bounded wait for the phase of `bar` with the given parity.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    if (mbar_test(bar, parity)) return true;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (true) {
        if (mbar_test(bar, parity)) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > kMergeWaitNs) return false;
    }
}

template <class IT, class V, int W, int WARPS, int CM, int WIN>
struct MergeStage {
    static constexpr bool HV = VOps<V>::has_val;
    static constexpr size_t vbytes = HV ? sizeof(V) * W : 0;
    static constexpr size_t bufbytes = (size_t)WIN * (sizeof(IT) + (HV ? sizeof(V) : 0));
    // per warp: accumulator, bitmap, barriers, then 2 buffers per list (16-byte aligned)
    static constexpr size_t head = (vbytes + W / 8 + 16 * CM + 15) / 16 * 16;
    static constexpr size_t warp_bytes = head + 2 * CM * bufbytes;
};

template <class IT, class V, int W, int WARPS, int CM, int WIN>
__global__ void __launch_bounds__(WARPS * 32)
    merge_stage_kernel(int c, MergeParts<IT, V> parts, long long m, long long n,
                       const int64_t* __restrict__ rpC, IT* __restrict__ ciC, V* __restrict__ vC,
                       int* err, unsigned long long* work) {
    using L = MergeStage<IT, V, W, WARPS, CM, WIN>;
    constexpr bool HV = L::HV;
    constexpr int NWORDS = W / 32;
    static_assert(WIN % 32 == 0, "windows hold whole rounds of 32 entries");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const int w = threadIdx.x >> 5;
    unsigned char* base = smem_raw + (size_t)w * L::warp_bytes;
    V* acc = reinterpret_cast<V*>(base);
    unsigned* bm = reinterpret_cast<unsigned*>(base + L::vbytes);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(base + L::vbytes + W / 8);
    unsigned char* bufs = base + L::head;
    auto bcol = [&](int s, int b) {
        return reinterpret_cast<IT*>(bufs + (size_t)(2 * s + b) * L::bufbytes);
    };
    auto bval = [&](int s, int b) {
        return reinterpret_cast<V*>(bufs + (size_t)(2 * s + b) * L::bufbytes + WIN * sizeof(IT));
    };
    for (int t = lane; t < W; t += 32)
        if constexpr (HV) acc[t] = VOps<V>::init();
    for (int t = lane; t < NWORDS; t += 32) bm[t] = 0u;
    if (lane < 2 * CM) mbar_init(&bar[lane]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    unsigned parity = 0u;   // bit 2s+b: parity of buffer b of list s's next phase
    unsigned pending = 0u;  // bit 2s+b: buffer b of list s has a copy in flight
    // lane 0 stages window [ws, ws + WIN) of list s (clipped to the row end
    // rounded up to four entries) into buffer b
    auto issue = [&](int s, int b, long long ws, long long e) {
        pending |= 1u << (2 * s + b);
        const long long len = parts.len[s];
        const long long we = min(ws + WIN, (e + 3) & ~3LL);
        const long long wc = max(ws, min(we, len & ~3LL));   // end of the 16-byte copies
        if (lane == 0) {
            const unsigned nb = (unsigned)(wc - ws);
            unsigned bytes = nb * (unsigned)sizeof(IT);
            if constexpr (HV) bytes += nb * (unsigned)sizeof(V);
            mbar_arrive_tx(&bar[2 * s + b], bytes);
            if (nb > 0) {
                bulk_to_shared(bcol(s, b), parts.col[s] + ws, nb * (unsigned)sizeof(IT),
                               &bar[2 * s + b]);
                if constexpr (HV)
                    bulk_to_shared(bval(s, b), parts.val[s] + ws, nb * (unsigned)sizeof(V),
                                   &bar[2 * s + b]);
            }
        }
        // the array's last entries past the copies, if the window reaches them
        const long long q = wc + lane;
        if (q < min(we, e) && q < len) {
            bcol(s, b)[q - ws] = parts.col[s][q];
            if constexpr (HV) bval(s, b)[q - ws] = parts.val[s][q];
        }
    };
    bool ok = true;
    while (ok) {
        long long i = 0;
        if (lane == 0) i = (long long)atomicAdd(work, 1ull);
        i = __shfl_sync(kFull, i, 0);
        if (i >= m) break;
        long long b_own = 0, e_own = 0;
        if (lane < c) {
            b_own = parts.rp[lane][i];
            e_own = parts.re[lane] ? parts.re[lane][i] : parts.rp[lane][i + 1];
        }
        long long pos[CM], end[CM], bst[CM];
        int cur[CM];
        // the previous row's reads of the buffers come before the new copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
#pragma unroll
        for (int s = 0; s < CM; ++s) {
            pos[s] = s < c ? __shfl_sync(kFull, b_own, s) : 0;
            end[s] = s < c ? __shfl_sync(kFull, e_own, s) : 0;
            bst[s] = pos[s] & ~3LL;
            cur[s] = 0;
            if (pos[s] < end[s]) {
                issue(s, 0, bst[s], end[s]);
                if (bst[s] + WIN < end[s]) issue(s, 1, bst[s] + WIN, end[s]);
            }
        }
        __syncwarp();
        // wait for a buffer's copy and take its phase
        auto take = [&](int s, int b) {
            const int t = 2 * s + b;
            if (!mbar_wait(&bar[t], (parity >> t) & 1u)) return false;
            parity ^= 1u << t;
            pending &= ~(1u << t);
            return true;
        };
#pragma unroll
        for (int s = 0; s < CM; ++s)
            if (ok && pos[s] < end[s]) ok = take(s, 0);
        if (!ok) break;
        long long out = rpC[i];
        const long long out_end = rpC[i + 1];
        while (ok) {
            long long nxt = n;
#pragma unroll
            for (int s = 0; s < CM; ++s)
                if (pos[s] < end[s]) nxt = min(nxt, (long long)bcol(s, cur[s])[pos[s] - bst[s]]);
            if (nxt >= n) break;
            const long long c0 = (nxt / W) * W;
            const long long c1 = min(c0 + (long long)W, n);
#pragma unroll
            for (int s = 0; s < CM; ++s) {
                while (ok && pos[s] < end[s]) {
                    const long long lim = min(bst[s] + WIN, end[s]);
                    const long long q = pos[s] + lane;
                    const IT* cb = bcol(s, cur[s]);
                    bool valid = q < lim;
                    long long col = 0;
                    if (valid) {
                        col = (long long)cb[q - bst[s]];
                        valid = col < c1;
                    }
                    if (valid) {
                        const int slot = (int)(col - c0);
                        atomicOr(&bm[slot >> 5], 1u << (slot & 31));
                        if constexpr (HV) {
                            const V v = bval(s, cur[s])[q - bst[s]];
                            if (kStoreFirst<V> && s == 0) acc[slot] = v;
                            else acc[slot] = VOps<V>::add(acc[slot], v);
                        }
                    }
                    __syncwarp();
                    const int got = __popc(__ballot_sync(kFull, valid));
                    pos[s] += got;
                    if (pos[s] >= end[s]) break;          // the row's entries of list s are done
                    if (pos[s] < lim) {
                        if (got < 32) break;              // the chunk ends inside the buffer
                        continue;                         // a full round: the chunk may go on
                    }
                    // buffer used up (pos == bst + WIN < end): the other buffer holds
                    // the next window; this one is refilled with the window after it
                    const long long nw = bst[s] + 2 * WIN;
                    if (nw < end[s]) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue(s, cur[s], nw, end[s]);
                        __syncwarp();
                    }
                    cur[s] ^= 1;
                    bst[s] += WIN;
                    ok = take(s, cur[s]);
                }
            }
            if (!ok) break;
            // emit the chunk in column order, clearing it
            for (int t0 = 0; t0 < NWORDS; t0 += 32) {
                const int t = t0 + lane;
                unsigned word = t < NWORDS ? bm[t] : 0u;
                const int pc = __popc(word);
                const int incl = warp_incl_scan(pc);
                long long p = out + incl - pc;
                while (word) {
                    const int bit = __ffs(word) - 1;
                    word &= word - 1;
                    const int slot = t * 32 + bit;
                    if (p < out_end) {
                        ciC[p] = (IT)(c0 + slot);
                        if constexpr (HV) vC[p] = acc[slot];
                    }
                    if constexpr (HV) acc[slot] = VOps<V>::init();
                    ++p;
                }
                if (t < NWORDS) bm[t] = 0u;
                out += __shfl_sync(kFull, incl, 31);
            }
            __syncwarp();
        }
        if (ok && lane == 0 && out != out_end) atomicExch(err, (int)kDevCountMismatch);
    }
    if (!ok) {
        if (lane == 0) atomicExch(err, (int)kDevWaitTimeout);
        // let the copies this warp still has in flight land before it ends
        // (each wait bounded again)
        for (int t = 0; t < 2 * CM; ++t)
            if ((pending >> t) & 1u) mbar_wait(&bar[t], (parity >> t) & 1u);
    }
}

// The count of the merge for int32 columns in 16-byte aligned arrays: the
// same sweep with four columns per lane per load (128 entries per window),
// so four times the bytes of every list are in flight.  Entry x of a window
// is component x % 4 of lane x / 4; windows start at multiples of four
// entries, and entries outside [row begin, row end) are masked by position.
__device__ __forceinline__ int4 merge_load4(const int32_t* __restrict__ col, long long q,
                                            long long len) {
    if (q + 4 <= len) return *reinterpret_cast<const int4*>(col + q);
    int4 r = make_int4(0, 0, 0, 0);
    if (q < len) r.x = col[q];
    if (q + 1 < len) r.y = col[q + 1];
    if (q + 2 < len) r.z = col[q + 2];
    if (q + 3 < len) r.w = col[q + 3];
    return r;
}

__device__ __forceinline__ int comp4(const int4& v, int j) {
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

template <class V, int W, int WARPS, int CM>
__global__ void __launch_bounds__(WARPS * 32)
    merge_count4_kernel(int c, MergeParts<int32_t, V> parts, long long m, long long n,
                        int64_t* __restrict__ rowcnt, unsigned long long* work) {
    constexpr int NWORDS = W / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const int w = threadIdx.x >> 5;
    unsigned* bm = reinterpret_cast<unsigned*>(smem_raw + (size_t)w * (W / 8));
    for (int t = lane; t < NWORDS; t += 32) bm[t] = 0u;
    __syncwarp();
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
        long long wb[CM], we[CM];
        int off[CM];
        int4 xa[CM], xb[CM], xc[CM];
#pragma unroll
        for (int s = 0; s < CM; ++s) {
            const long long b = __shfl_sync(kFull, b_own, s);
            we[s] = s < c ? __shfl_sync(kFull, e_own, s) : 0;
            wb[s] = b & ~3LL;
            off[s] = (int)(b - wb[s]);
            xa[s] = xb[s] = xc[s] = make_int4(0, 0, 0, 0);
            if (b < we[s]) {
                const long long q = wb[s] + 4 * lane;
                xa[s] = merge_load4(parts.col[s], q, parts.len[s]);
                if (wb[s] + 128 < we[s]) xb[s] = merge_load4(parts.col[s], q + 128, parts.len[s]);
                if (wb[s] + 256 < we[s]) xc[s] = merge_load4(parts.col[s], q + 256, parts.len[s]);
            }
        }
        long long count = 0;
        while (true) {
            long long nxt = n;
#pragma unroll
            for (int s = 0; s < CM; ++s) {
                const int h = __shfl_sync(kFull, comp4(xa[s], off[s] & 3), (off[s] >> 2) & 31);
                if (wb[s] + off[s] < we[s]) nxt = min(nxt, (long long)h);
            }
            if (nxt >= n) break;
            const long long c0 = (nxt / W) * W;
            const long long c1 = min(c0 + (long long)W, n);
#pragma unroll
            for (int s = 0; s < CM; ++s) {
                while (true) {
                    int got = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int e = 4 * lane + j;
                        const long long col = comp4(xa[s], j);
                        const bool valid = e >= off[s] && wb[s] + e < we[s] && col < c1;
                        if (valid) {
                            const int slot = (int)(col - c0);
                            atomicOr(&bm[slot >> 5], 1u << (slot & 31));
                        }
                        got += __popc(__ballot_sync(kFull, valid));
                    }
                    off[s] += got;
                    if (off[s] < 128) break;
                    // window A used up: B and C move up, the window after C is loaded
                    wb[s] += 128;
                    off[s] = 0;
                    xa[s] = xb[s];
                    xb[s] = xc[s];
                    if (wb[s] + 256 < we[s])
                        xc[s] = merge_load4(parts.col[s], wb[s] + 256 + 4 * lane, parts.len[s]);
                    if (wb[s] >= we[s]) break;
                }
            }
            __syncwarp();
            for (int t = lane; t < NWORDS; t += 32) {
                count += __popc(bm[t]);
                bm[t] = 0u;
            }
            __syncwarp();
        }
        count = warp_sum(count);
        if (lane == 0) rowcnt[i] = count;
    }
}

template <class IT, class V, bool NUMERIC>
cudaError_t launch_merge_t(int c, const spgemm_csr* parts, long long m, long long n,
                           int sm_count, cudaStream_t s, int64_t* rowcnt, const int64_t* rpC,
                           void* colC, void* valC, int* err, unsigned long long* work,
                           bool staged_opt) {
    MergeParts<IT, V> mp{};
    bool aligned16 = true;
    for (int t = 0; t < c; ++t) {
        mp.rp[t] = parts[t].rowptr;
        mp.re[t] = parts[t].rowend;
        mp.col[t] = (const IT*)parts[t].col;
        mp.val[t] = (const V*)parts[t].val;
        mp.len[t] = parts[t].nnz;
        aligned16 = aligned16 && ((uintptr_t)parts[t].col % 16) == 0;
    }
    if constexpr (!NUMERIC && std::is_same<IT, int32_t>::value) {
        if (c <= 4 && aligned16) {
            constexpr int W = 8192, WARPS = 4;
            auto k = c <= 2 ? merge_count4_kernel<V, W, WARPS, 2> : merge_count4_kernel<V, W, WARPS, 4>;
            const size_t smem = (size_t)WARPS * (W / 8);
            int occ = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, WARPS * 32, smem);
            if (occ < 1) occ = 1;
            const long long need = (m + WARPS - 1) / WARPS;
            const long long g = std::max<long long>(1, std::min(need, (long long)sm_count * occ));
            if (m > 0) {
                count_launches(1);
                k<<<(unsigned)g, WARPS * 32, smem, s>>>(c, mp, m, n, rowcnt, work);
            }
            return cudaGetLastError();
        }
    }
    if constexpr (NUMERIC) {
        bool staged = staged_opt && c <= 4;
        for (int t = 0; t < c; ++t)
            staged = staged && ((uintptr_t)parts[t].col % 16) == 0 &&
                     (!VOps<V>::has_val || ((uintptr_t)parts[t].val % 16) == 0);
        if (staged) {
            constexpr int W = 1024, WARPS = 4, WIN = 64;
            auto k = c <= 2 ? merge_stage_kernel<IT, V, W, WARPS, 2, WIN>
                            : merge_stage_kernel<IT, V, W, WARPS, 4, WIN>;
            const size_t smem = (size_t)WARPS * (c <= 2 ? MergeStage<IT, V, W, WARPS, 2, WIN>::warp_bytes
                                                          : MergeStage<IT, V, W, WARPS, 4, WIN>::warp_bytes);
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
                k<<<(unsigned)g, WARPS * 32, smem, s>>>(c, mp, m, n, rpC, (IT*)colC, (V*)valC,
                                                        err, work);
            }
            return cudaGetLastError();
        }
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
                         unsigned long long* work, bool staged) {
    const bool i32 = parts[0].index_type == SPGEMM_INDEX_I32;
    return with_value_type(vt, [&](auto tag) -> cudaError_t {
        using V = decltype(tag);
        if (numeric)
            return i32 ? launch_merge_t<int32_t, V, true>(c, parts, m, n, sm_count, s, rowcnt, rpC,
                                                          colC, valC, err, work, staged)
                       : launch_merge_t<int64_t, V, true>(c, parts, m, n, sm_count, s, rowcnt, rpC,
                                                          colC, valC, err, work, staged);
        return i32 ? launch_merge_t<int32_t, V, false>(c, parts, m, n, sm_count, s, rowcnt, rpC,
                                                       colC, valC, err, work, staged)
                   : launch_merge_t<int64_t, V, false>(c, parts, m, n, sm_count, s, rowcnt, rpC,
                                                       colC, valC, err, work, staged);
    });
}

}  // namespace sg
