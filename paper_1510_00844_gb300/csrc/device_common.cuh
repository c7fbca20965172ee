// Device-side building blocks shared by the sparse-product kernels:
// value semirings, warp scans, the per-warp hash table, and the batch walker
// that turns a run of A(i,:) entries into lanes of B(k,:) entries in
// ascending k.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

namespace sg {

constexpr unsigned kFull = 0xffffffffu;

// Error codes written to the plan's device error word.
enum DevErr : int {
    kDevOk = 0,
    kDevTableFull = 1,   // a hash probe ran over the whole table
    kDevCountMismatch = 2,
    kDevBadIndex = 3,    // checked mode: column out of range / unsorted
    kDevBadRowptr = 4,
    kDevCapacity = 5,    // C did not fit the output capacity
    kDevArena = 6,       // a dense row is longer than the cursor arena slot
    kDevTooWide = 7,     // a dense row in a product wider than the shared-memory bitmap
    kDevWaitTimeout = 9, // a bounded wait for asynchronous copies gave up
};

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned lanemask_le() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <class T>
__device__ __forceinline__ T warp_incl_scan(T x) {
    const int lane = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

template <class T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
    return x;
}

template <class T>
__device__ __forceinline__ T warp_min(T x) {
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        T y = __shfl_xor_sync(kFull, x, d);
        x = x < y ? x : y;
    }
    return x;
}

template <class T>
__device__ __forceinline__ T warp_max(T x) {
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        T y = __shfl_xor_sync(kFull, x, d);
        x = x > y ? x : y;
    }
    return x;
}

// ---------------------------------------------------------------- values
// Values are multiplied then added with explicit round-to-nearest
// intrinsics, so no multiply-add is ever fused: every product is rounded
// before it joins the running sum, as in the plain definition.  Sums start
// from -0.0, the identity of IEEE addition (-0 + x == x for every x,
// including +0 and -0), so the first product enters the sum unchanged.  (On
// this GPU a fused multiply-add is also slower here than the two separate
// operations, whose multiply leaves the accumulator's dependency chain.)
struct NoVal {};

template <class V>
struct VOps;

template <>
struct VOps<double> {
    static constexpr bool has_val = true;
    __device__ static __forceinline__ double init() { return -0.0; }
    __device__ static __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ static __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
};

template <>
struct VOps<float> {
    static constexpr bool has_val = true;
    __device__ static __forceinline__ float init() { return -0.0f; }
    __device__ static __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ static __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
};

template <>
struct VOps<int64_t> {  // two's-complement wraparound
    static constexpr bool has_val = true;
    __device__ static __forceinline__ int64_t init() { return 0; }
    __device__ static __forceinline__ int64_t mul(int64_t a, int64_t b) {
        return (int64_t)((unsigned long long)a * (unsigned long long)b);
    }
    __device__ static __forceinline__ int64_t add(int64_t a, int64_t b) {
        return (int64_t)((unsigned long long)a + (unsigned long long)b);
    }
};

template <>
struct VOps<NoVal> {  // (or, and): pattern only
    static constexpr bool has_val = false;
    __device__ static __forceinline__ NoVal init() { return {}; }
    __device__ static __forceinline__ NoVal mul(NoVal, NoVal) { return {}; }
    __device__ static __forceinline__ NoVal add(NoVal, NoVal) { return {}; }
};

// The (min, +) and (min, select2nd) semirings (the operations MIS-2
// aggregation is built from, Alg. 3), stored as plain double / int64 values.
// A min reduction starts at its identity (+infinity, INT64_MAX) and keeps the
// running value x unless the next term y satisfies y < x, so a NaN term is
// never the minimum and the first of equal terms is kept; the result does not
// depend on the order of the terms except through that first-kept rule, and
// every path adds terms in ascending k (ascending slice for the merge).
template <class T>
struct MinPlus {
    T x;
};
template <class T>
struct MinSel {
    T x;
};

template <>
struct VOps<MinPlus<double>> {
    static constexpr bool has_val = true;
    __device__ static __forceinline__ MinPlus<double> init() {
        return {__longlong_as_double(0x7ff0000000000000LL)};
    }
    __device__ static __forceinline__ MinPlus<double> mul(MinPlus<double> a, MinPlus<double> b) {
        return {__dadd_rn(a.x, b.x)};
    }
    __device__ static __forceinline__ MinPlus<double> add(MinPlus<double> s, MinPlus<double> t) {
        return {t.x < s.x ? t.x : s.x};
    }
};

template <>
struct VOps<MinPlus<int64_t>> {  // sums wrap around (two's complement)
    static constexpr bool has_val = true;
    __device__ static __forceinline__ MinPlus<int64_t> init() { return {INT64_MAX}; }
    __device__ static __forceinline__ MinPlus<int64_t> mul(MinPlus<int64_t> a, MinPlus<int64_t> b) {
        return {(int64_t)((unsigned long long)a.x + (unsigned long long)b.x)};
    }
    __device__ static __forceinline__ MinPlus<int64_t> add(MinPlus<int64_t> s, MinPlus<int64_t> t) {
        return {t.x < s.x ? t.x : s.x};
    }
};

template <class T>
struct VOps<MinSel<T>> {
    static constexpr bool has_val = true;
    __device__ static __forceinline__ MinSel<T> init() {
        if constexpr (std::is_floating_point<T>::value)
            return {__longlong_as_double(0x7ff0000000000000LL)};
        else
            return {INT64_MAX};
    }
    __device__ static __forceinline__ MinSel<T> mul(MinSel<T>, MinSel<T> b) { return b; }
    __device__ static __forceinline__ MinSel<T> add(MinSel<T> s, MinSel<T> t) {
        return {t.x < s.x ? t.x : s.x};
    }
};

template <class V>
__device__ __forceinline__ V shfl_val(V v, int src) {
    if constexpr (VOps<V>::has_val) return __shfl_sync(kFull, v, src);
    else return v;
}

template <class T>
__device__ __forceinline__ MinPlus<T> shfl_val(MinPlus<T> v, int src) {
    return {__shfl_sync(kFull, v.x, src)};
}

template <class T>
__device__ __forceinline__ MinSel<T> shfl_val(MinSel<T> v, int src) {
    return {__shfl_sync(kFull, v.x, src)};
}

template <class V>
__device__ __forceinline__ V load_val(const V* p, int64_t q) {
    if constexpr (VOps<V>::has_val) return p[q];
    else return V{};
}

// ---------------------------------------------------------------- keys
// Hash-table keys hold column indices; -1 marks an empty slot.
template <class IT>
struct KeyT;
template <>
struct KeyT<int32_t> { using type = int; };
template <>
struct KeyT<int64_t> { using type = long long; };

__device__ __forceinline__ int key_cas(int* a, int cmp, int v) { return atomicCAS(a, cmp, v); }
__device__ __forceinline__ long long key_cas(long long* a, long long cmp, long long v) {
    return (long long)atomicCAS((unsigned long long*)a, (unsigned long long)cmp,
                                (unsigned long long)v);
}

template <int LOG2T, class K>
__device__ __forceinline__ unsigned hash_slot(K key) {
    unsigned long long x = (unsigned long long)key * 0x9E3779B97F4A7C15ull;
    return (unsigned)(x >> (64 - LOG2T));
}

// Insert `key` into a warp-private open-addressing table of 2^LOG2T slots
// (linear probing).  Returns the slot; is_new is true for the one lane whose
// CAS claimed an empty slot.  The probe stops after 2^LOG2T slots (a full
// table), records kDevTableFull and returns -1.
template <int LOG2T, class K>
__device__ __forceinline__ int hash_insert(K* keys, K key, bool& is_new, int* err) {
    constexpr unsigned T = 1u << LOG2T;
    unsigned h = hash_slot<LOG2T>(key);
    volatile K* vk = keys;
    for (unsigned it = 0; it < T; ++it) {
        K cur = vk[h];
        if (cur == key) {
            is_new = false;
            return (int)h;
        }
        if (cur == K(-1)) {
            K old = key_cas(&keys[h], K(-1), key);
            if (old == K(-1)) {
                is_new = true;
                return (int)h;
            }
            if (old == key) {
                is_new = false;
                return (int)h;
            }
        }
        h = (h + 1) & (T - 1);
    }
    atomicExch(err, (int)kDevTableFull);
    is_new = false;
    return -1;
}

// Ordered accumulation of one warp round into a warp-private array.
// Lanes hold (slot, v) for consecutive products in ascending k (lane order =
// product order).  Lanes that hit the same slot are grouped; the r-th lane of
// a group adds in step r, so each slot receives its products in lane order,
// i.e. in ascending k, exactly like a sequential loop.
template <class V>
__device__ __forceinline__ void ordered_add(V* acc, int slot, bool valid, V v) {
    if constexpr (VOps<V>::has_val) {
        const int lane = lane_id();
        unsigned grp = __match_any_sync(kFull, valid ? slot : -1 - lane);
        int rank = __popc(grp & lanemask_lt());
        int maxr = (int)__reduce_max_sync(kFull, valid ? (unsigned)rank : 0u);
        for (int r = 0; r <= maxr; ++r) {
            if (valid && rank == r) acc[slot] = VOps<V>::add(acc[slot], v);
            __syncwarp();
        }
    }
}

// Rounds in which every lane holds a distinct slot (one k at a time).
template <class V>
__device__ __forceinline__ void plain_add(V* acc, int slot, bool valid, V v) {
    if constexpr (VOps<V>::has_val) {
        if (valid) acc[slot] = VOps<V>::add(acc[slot], v);
        __syncwarp();
    }
}

// ---------------------------------------------------------------- walker
// Walk a batch of nb (<= 32) A entries held one per lane: lane e owns the B
// range [lo_e, lo_e + len_e).  Entries are visited in lane order.  An entry
// with len >= 32 is processed alone, 32 B entries per round (its columns are
// distinct, so a round has no repeated slot: `ordered` = false).  A maximal
// run of consecutive shorter entries is flattened: round t gives lane x the
// (32t + x)-th product of the run, found by a binary search over the run's
// exclusive prefix; such rounds can repeat a slot (`ordered` = true).
// f(q, e, valid, ordered) is called by all 32 lanes together; q is the B
// position, e the owning entry (lane) index.
template <class F>
__device__ __forceinline__ void walk_batch(int nb, long long lo, int len, F&& f) {
    const int lane = lane_id();
    unsigned long_mask = __ballot_sync(kFull, lane < nb && len >= 32);
    int cur = 0;
    while (cur < nb) {
        if ((long_mask >> cur) & 1u) {
            long long l0 = __shfl_sync(kFull, lo, cur);
            int L = __shfl_sync(kFull, len, cur);
            for (int t = 0; t < L; t += 32) {
                int x = t + lane;
                f(l0 + x, cur, x < L, false);
            }
            ++cur;
        } else {
            unsigned after = long_mask & (cur == 31 ? 0u : (~0u << (cur + 1)));
            int end = after ? (__ffs(after) - 1) : nb;
            int mylen = (lane >= cur && lane < end) ? len : 0;
            int incl = warp_incl_scan(mylen);
            int excl = incl - mylen;
            int total = __shfl_sync(kFull, incl, 31);
            int key = lane < cur ? -1 : (lane >= end ? 0x7fffffff : excl);
            for (int f0 = 0; f0 < total; f0 += 32) {
                int fi = f0 + lane;
                int e = 0;
#pragma unroll
                for (int b = 16; b; b >>= 1) {
                    int kc = __shfl_sync(kFull, key, e + b);
                    if (kc <= fi) e += b;
                }
                long long l0 = __shfl_sync(kFull, lo, e);
                int ex = __shfl_sync(kFull, excl, e);
                f(l0 + (fi - ex), e, fi < total, true);
            }
            cur = end;
        }
    }
}

// Same walk as walk_batch, four rounds at a time: f4(q[4], e[4], valid[4],
// ordered) receives the B positions of rounds t = 0..3 (round t precedes
// round t+1), so the callee can issue all their loads before using them.
template <class F4>
__device__ __forceinline__ void walk_batch4(int nb, long long lo, int len, F4&& f4) {
    const int lane = lane_id();
    unsigned long_mask = __ballot_sync(kFull, lane < nb && len >= 32);
    int cur = 0;
    while (cur < nb) {
        long long q[4];
        int ev[4];
        bool vl[4];
        if ((long_mask >> cur) & 1u) {
            const long long l0 = __shfl_sync(kFull, lo, cur);
            const int L = __shfl_sync(kFull, len, cur);
            for (int t0 = 0; t0 < L; t0 += 128) {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int x = t0 + 32 * t + lane;
                    q[t] = l0 + x;
                    ev[t] = cur;
                    vl[t] = x < L;
                }
                f4(q, ev, vl, false);
            }
            ++cur;
        } else {
            unsigned after = long_mask & (cur == 31 ? 0u : (~0u << (cur + 1)));
            int end = after ? (__ffs(after) - 1) : nb;
            int mylen = (lane >= cur && lane < end) ? len : 0;
            int incl = warp_incl_scan(mylen);
            int excl = incl - mylen;
            int total = __shfl_sync(kFull, incl, 31);
            int key = lane < cur ? -1 : (lane >= end ? 0x7fffffff : excl);
            for (int f0 = 0; f0 < total; f0 += 128) {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int fi = f0 + 32 * t + lane;
                    int e = 0;
#pragma unroll
                    for (int b = 16; b; b >>= 1) {
                        int kc = __shfl_sync(kFull, key, e + b);
                        if (kc <= fi) e += b;
                    }
                    const long long l0 = __shfl_sync(kFull, lo, e);
                    const int ex = __shfl_sync(kFull, excl, e);
                    q[t] = l0 + (fi - ex);
                    ev[t] = e;
                    vl[t] = fi < total;
                }
                f4(q, ev, vl, true);
            }
            cur = end;
        }
    }
}

// All products of a batch flattened in entry order, four rounds per call of
// f4(q[4], e[4], valid[4]); used where the order of products does not matter
// (symbolic phase) or is restored by the callee.
template <class F4>
__device__ __forceinline__ void walk_flat4(int nb, long long lo, int len, F4&& f4) {
    const int lane = lane_id();
    const int incl = warp_incl_scan(lane < nb ? len : 0);
    const int excl = incl - (lane < nb ? len : 0);
    const int total = __shfl_sync(kFull, incl, 31);
    const int key = lane < nb ? excl : 0x7fffffff;
    for (int f0 = 0; f0 < total; f0 += 128) {
        long long q[4];
        int ev[4];
        bool vl[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int fi = f0 + 32 * t + lane;
            int e = 0;
#pragma unroll
            for (int b = 16; b; b >>= 1) {
                int kc = __shfl_sync(kFull, key, e + b);
                if (kc <= fi) e += b;
            }
            const long long l0 = __shfl_sync(kFull, lo, e);
            const int ex = __shfl_sync(kFull, excl, e);
            q[t] = l0 + (fi - ex);
            ev[t] = e;
            vl[t] = fi < total;
        }
        f4(q, ev, vl);
    }
}

}  // namespace sg
