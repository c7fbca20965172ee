// Kernels of the two-phase sparse product C = A.B (Gustavson, Alg. 1, on
// CSR rows) and the k-slice bounds (Sec. 4.1).  Templates over the column
// index type IT (int32_t / int64_t) and the value type V (double, float,
// int64_t, the min-semiring wrappers, NoVal for the Boolean semiring).
//
// Row classes (decided from flops_i = sum_{k in A(i,:)} nnz(B(k,:)), Sec. 2):
//   EMPTY       flops_i == 0
//   HASH(b)     flops_i <= dense_min (<= 1024): one warp per row, warp-private
//               hash table in shared memory (keys for the symbolic phase, keys
//               + values for the numeric phase), output sorted in the warp
//               (bitonic sort up to 64 entries, stable radix sort above).
//   DENSE(b)    flops_i > dense_min: symbolic = one block per row with a
//               bitmap of all n columns in shared memory (also yields
//               per-chunk counts); numeric = one warp per (row, column
//               segment) sweeping column chunks of width W with a dense
//               accumulator, so the output comes out sorted.  DENSE rows are
//               bucketed by floor(log2 flops_i), largest first.
#pragma once

#include "device_common.cuh"

namespace sg {

constexpr int kNumHashBins = 4;
__host__ __device__ constexpr int hash_bin_flops(int b) {
    return b == 0 ? 32 : b == 1 ? 128 : b == 2 ? 512 : 1024;
}
constexpr int kDenseMinLog2 = 10;  // flops > 1024 -> dense
constexpr int kDenseMaxLog2 = 40;
constexpr int kClassEmpty = 0;
constexpr int kClassHash0 = 1;
constexpr int kClassDense0 = kClassHash0 + kNumHashBins;          // largest-flops bucket
constexpr int kNumClasses = kClassDense0 + (kDenseMaxLog2 - kDenseMinLog2 + 1);
constexpr int kSegGrid = 16;
// Table size (log2 slots) of hash bin 0, whose rows (at most 32 products)
// take the table-free short-row path instead.
constexpr int kShortLog2T = 6;
// Dense chunk configurations (columns per chunk, warps per block): one is
// chosen per plan (spgemm_opts.dense_chunk forces one).
constexpr int kDenseW0 = 1024, kDenseWarps0 = 8;
constexpr int kDenseW1 = 2048, kDenseWarps1 = 4;

// One product of a batch (C_p = A_p . B_p).  Rows of all products are
// numbered globally: product p owns global rows [row_base, row_base + m) and
// global B rows [brow_base, brow_base + l).  The workspace offsets give each
// product its slice of the shared tables.
struct ProdDesc {
    long long m, l, n;
    long long row_base, brow_base;
    const int64_t* rpA;
    const int64_t* reA;
    const void* ciA;
    const void* vA;
    const int64_t* rpB;
    const void* ciB;
    const void* vB;
    long long nnzB;
    long long chunk_base;  // dense chunk counts: chunk_base + i * P + c
    long long seg_base;    // segment table: seg_base + k * (kSegGrid + 1) + g
    long long run_base;    // run lengths: run_base + q (q a position in B's arrays)
    int P;                 // column chunks per row
    int pad;
};

constexpr int kMaxDenseClasses = kDenseMaxLog2 - kDenseMinLog2 + 1;

struct DevCounters {
    unsigned long long class_count[kNumClasses];
    unsigned long long class_cursor[kNumClasses];
    unsigned long long class_off[kNumClasses + 1];
    unsigned long long unit_begin[kMaxDenseClasses + 1];  // dense work units per class
    unsigned long long total_flops;
    unsigned long long max_flops;
    unsigned long long work_counter[4];  // dynamic row grabbing
    unsigned long long max_dense_len;    // longest A row among dense rows
    int err;
    int unsupported;
    int seg_log2;                        // dense work-unit size of the plan
    int pad[29];
};

// Product owning global row r: the largest p with rb[p] <= r.
__device__ __forceinline__ int find_prod(const long long* __restrict__ rb, int nprod, long long r) {
    int lo = 0, hi = nprod - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (rb[mid] <= r) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Everything a kernel needs about global row r.
template <class IT, class V>
struct RowCtx {
    long long i, a0, a1, n;
    const IT* ciA;
    const V* vA;
    const int64_t* rpB;
    const IT* ciB;
    const V* vB;
    long long chunk_base, seg_base, run_base;
    int P;
};

template <class IT, class V>
__device__ __forceinline__ RowCtx<IT, V> row_ctx(const ProdDesc* __restrict__ D,
                                                 const long long* __restrict__ rb, int nprod,
                                                 long long r) {
    const int p = nprod > 1 ? find_prod(rb, nprod, r) : 0;
    const ProdDesc& d = D[p];
    RowCtx<IT, V> c;
    c.i = r - d.row_base;
    c.a0 = d.rpA[c.i];
    c.a1 = d.reA ? d.reA[c.i] : d.rpA[c.i + 1];
    c.n = d.n;
    c.ciA = (const IT*)d.ciA;
    c.vA = (const V*)d.vA;
    c.rpB = d.rpB;
    c.ciB = (const IT*)d.ciB;
    c.vB = (const V*)d.vB;
    c.chunk_base = d.chunk_base;
    c.seg_base = d.seg_base;
    c.run_base = d.run_base;
    c.P = d.P;
    return c;
}

// The rows rows[first], rows[first + stride], ... (< nrows) of a class,
// walked by one warp.  (Loading the next rows' ids and bounds while a row is
// processed was measured on the short rows of the AMG hierarchy and gained
// nothing.)
template <class IT, class V, class F>
__device__ __forceinline__ void for_class_rows(const ProdDesc* __restrict__ D,
                                               const long long* __restrict__ rb, int nprod,
                                               const int32_t* __restrict__ crow, long long first,
                                               long long nrows, long long stride, F&& f) {
    for (long long rr = first; rr < nrows; rr += stride) {
        const long long r = crow[rr];
        f(row_ctx<IT, V>(D, rb, nprod, r), r);
    }
}

// Rows [r0, r1) of a block by class: with base == nullptr, count them per
// class into loc; else place row r at base[c] + a slot taken from loc[c].
// Lanes of a warp with the same class take one atomic together.
__device__ __forceinline__ void bin_block_rows(const unsigned char* __restrict__ cls,
                                               int32_t* __restrict__ rows, long long r0,
                                               long long r1, unsigned long long* loc,
                                               const unsigned long long* base) {
    const int lane = threadIdx.x & 31;
    for (long long b = r0 + (threadIdx.x & ~31); b < r1; b += blockDim.x) {
        const long long r = b + lane;
        const bool valid = r < r1;
        const int c = valid ? (int)cls[r] : -1 - lane;
        const unsigned grp = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(grp) - 1;
        const int rank = __popc(grp & ((1u << lane) - 1u));
        unsigned long long first = 0;
        if (valid && lane == leader) first = atomicAdd(&loc[c], (unsigned long long)__popc(grp));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (valid && base) rows[base[c] + first + rank] = (int32_t)r;
    }
}

// Tile of the int64 exclusive scan: 256 threads x 16 items.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

// Class of a row with `flops` products: EMPTY, the smallest hash bin that
// holds flops << hash_shift while flops <= dense_min (<= 1024; the largest
// bin takes the rest), else the dense bucket of floor(log2 flops), largest
// first.
__host__ __device__ __forceinline__ int row_class(long long flops, int dense_min,
                                                  int hash_shift = 0) {
    if (flops == 0) return kClassEmpty;
    if (flops <= dense_min) {
#pragma unroll
        for (int b = 0; b < kNumHashBins - 1; ++b)
            if ((flops << hash_shift) <= hash_bin_flops(b)) return kClassHash0 + b;
        return kClassHash0 + kNumHashBins - 1;
    }
#ifdef __CUDA_ARCH__
    int lg = 63 - __clzll(flops);
#else
    int lg = 63 - __builtin_clzll((unsigned long long)flops);
#endif
    if (lg > kDenseMaxLog2) lg = kDenseMaxLog2;
    if (lg < kDenseMinLog2) lg = kDenseMinLog2;
    return kClassDense0 + (kDenseMaxLog2 - lg);
}

// Segments per row of dense class t (floor(log2 flops) = kDenseMaxLog2 - t):
// about 2^seg_log2 products per segment (a plan knob; by default chosen from
// the plan's flops so that big products get fewer, longer units), at most
// kSegGrid.
__host__ __device__ __forceinline__ int dense_class_segments(int t, int seg_log2) {
    const int lg = kDenseMaxLog2 - t;
    int sh = lg + 1 - seg_log2;
    if (sh < 0) sh = 0;
    if (sh > 4) sh = 4;  // kSegGrid = 16
    return 1 << sh;
}

__device__ __forceinline__ long long row_end(const int64_t* rp, const int64_t* re, long long i) {
    return re ? re[i] : rp[i + 1];
}

// ----------------------------------------------------------------- K1: flops
// Per global row (a warp per tile of 32 rows): flops_i, its class, per-class
// counts, total and max flops, longest dense row; a product whose dense rows
// need more columns than the shared-memory bitmap holds is flagged.
// Learned sizing (not in the paper): when `prm` is given, the warp also
// evaluates the row-size predictor on each row's features (one lane per
// hidden unit), writes the predicted capacity cap_out[r] = clamp(2^(y +
// margin) - 1, max_k |B(k,:)|, min(flops, n)), and bins rows of at most
// dense_min products by that capacity instead of by their flops.
constexpr int kSizerF = 6;

template <class IT>
__device__ __forceinline__ void analyze_kernel_body(long long R, const ProdDesc* __restrict__ D,
                               const long long* __restrict__ rb, int nprod, long long max_dense_n,
                               int dense_min, int64_t* __restrict__ flops_out,
                               unsigned char* __restrict__ cls_out, DevCounters* cnt,
                               const float* __restrict__ prm, float margin,
                               int64_t* __restrict__ cap_out, int hash_shift,
        const long long vbid, const long long vnb) {
    __shared__ unsigned long long hist[kNumClasses];
    __shared__ unsigned long long blk_total, blk_max, blk_dlen;
    __shared__ int blk_unsup;
    __shared__ float sp[32 * kSizerF + 32 + 32 * 32 + 32 + 32 + 1];
    if (prm)
        for (int q = threadIdx.x; q < 32 * kSizerF + 32 + 32 * 32 + 32 + 32 + 1; q += blockDim.x)
            sp[q] = prm[q];
    for (int t = threadIdx.x; t < kNumClasses; t += blockDim.x) hist[t] = 0;
    if (threadIdx.x == 0) {
        blk_total = 0;
        blk_max = 0;
        blk_dlen = 0;
        blk_unsup = 0;
    }
    __syncthreads();
    const int lane = lane_id();
    const long long warp = ((long long)vbid * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)vnb * blockDim.x) >> 5;
    unsigned long long my_total = 0, my_max = 0;
    // Tiles of 32 rows: a row of at most 32 A entries is summed by its own
    // lane (eight entries' loads in flight at a time); longer rows by the
    // whole warp, one after another.  The predictor then runs row by row with
    // a lane per hidden unit.
    for (long long tile = warp; tile * 32 < R; tile += nwarps) {
        const long long r = tile * 32 + lane;
        const bool in = r < R;
        RowCtx<IT, NoVal> c{};
        if (in) c = row_ctx<IT, NoVal>(D, rb, nprod, r);
        const long long d = in ? c.a1 - c.a0 : 0;
        long long f = 0, mx = 0;
        if (in && d <= 32) {
            for (long long p0 = c.a0; p0 < c.a1; p0 += 8) {
                long long k[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) k[u] = p0 + u < c.a1 ? (long long)c.ciA[p0 + u] : -1;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (k[u] >= 0) {
                        const long long len = c.rpB[k[u] + 1] - c.rpB[k[u]];
                        f += len;
                        mx = len > mx ? len : mx;
                    }
                }
            }
        }
        for (unsigned lm = __ballot_sync(kFull, in && d > 32); lm; lm &= lm - 1u) {
            const int src = __ffs(lm) - 1;
            const RowCtx<IT, NoVal> cs = row_ctx<IT, NoVal>(D, rb, nprod, tile * 32 + src);
            long long fs = 0, ms = 0;
            for (long long p = cs.a0 + lane; p < cs.a1; p += 32) {
                const long long k = (long long)cs.ciA[p];
                const long long len = cs.rpB[k + 1] - cs.rpB[k];
                fs += len;
                ms = len > ms ? len : ms;
            }
            fs = warp_sum(fs);
            ms = warp_max(ms);
            if (lane == src) {
                f = fs;
                mx = ms;
            }
        }
        long long cap = 0;
        if (prm) {
            const float* W1 = sp;
            const float* b1 = W1 + 32 * kSizerF;
            const float* W2 = b1 + 32;
            const float* b2 = W2 + 32 * 32;
            const float* w3 = b2 + 32;
            for (unsigned pm = __ballot_sync(kFull, in && f > 0); pm; pm &= pm - 1u) {
                const int j = __ffs(pm) - 1;
                const long long fj = __shfl_sync(kFull, f, j);
                const long long dj = __shfl_sync(kFull, d, j);
                const long long mj = __shfl_sync(kFull, mx, j);
                const long long nj = __shfl_sync(kFull, c.n, j);
                const long long ub = fj < nj ? fj : nj;
                float x[kSizerF];
                x[0] = log2f(1.f + (float)fj);
                x[1] = log2f(1.f + (float)dj);
                x[2] = log2f(1.f + (float)mj);
                x[3] = log2f(1.f + (float)nj);
                x[4] = log2f(1.f + (float)fj / (float)dj);
                x[5] = log2f(1.f + (float)ub);
                float z = b1[lane];
                for (int q = 0; q < kSizerF; ++q) z = __fadd_rn(z, __fmul_rn(W1[lane * kSizerF + q], x[q]));
                const float h1 = z > 0.f ? z : 0.f;
                float z2 = b2[lane];
                for (int k = 0; k < 32; ++k)
                    z2 = __fadd_rn(z2, __fmul_rn(W2[lane * 32 + k], __shfl_sync(kFull, h1, k)));
                const float h2 = z2 > 0.f ? z2 : 0.f;
                const float y = warp_sum(__fmul_rn(w3[lane], h2)) + w3[32];
                const float est = exp2f(y + margin) - 1.f;
                long long cj = est >= (float)ub ? ub : (long long)ceilf(est > 0.f ? est : 0.f);
                if (cj < mj) cj = mj;
                if (cj > ub) cj = ub;
                if (lane == j) cap = cj;
            }
        }
        int cl = -1 - lane;
        if (in) {
            flops_out[r] = f;
            if (cap_out) cap_out[r] = prm ? cap : f;
            cl = row_class(f, dense_min, hash_shift);
            if (prm && cl > kClassEmpty && cl < kClassDense0) {
                cl = row_class(cap > 0 ? cap : 1, dense_min, hash_shift);
                // bin 0 is the short-row path (one product per lane): a row
                // with more products takes bin 1's table whatever its size
                if (cl == kClassHash0 && f > 32) cl = kClassHash0 + 1;
            }
            cls_out[r] = (unsigned char)cl;
            if (cl >= kClassDense0) {
                if (c.n > max_dense_n) blk_unsup = 1;
                atomicMax(&blk_dlen, (unsigned long long)d);
            }
            my_total += (unsigned long long)f;
            if ((unsigned long long)f > my_max) my_max = (unsigned long long)f;
        }
        // one shared atomic per class present in the tile
        const unsigned grp = __match_any_sync(kFull, cl);
        if (in && (grp & lanemask_lt()) == 0u) atomicAdd(&hist[cl], (unsigned long long)__popc(grp));
    }
    my_total = warp_sum(my_total);
    my_max = warp_max(my_max);
    if (lane == 0) {
        atomicAdd(&blk_total, my_total);
        atomicMax(&blk_max, my_max);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kNumClasses; t += blockDim.x)
        if (hist[t]) atomicAdd(&cnt->class_count[t], hist[t]);
    if (threadIdx.x == 0) {
        atomicAdd(&cnt->total_flops, blk_total);
        atomicMax(&cnt->max_flops, blk_max);
        atomicMax(&cnt->max_dense_len, blk_dlen);
        if (blk_unsup) atomicExch(&cnt->unsupported, 1);
    }
}

template <class IT>
__global__ void analyze_kernel(long long R, const ProdDesc* __restrict__ D,
                               const long long* __restrict__ rb, int nprod, long long max_dense_n,
                               int dense_min, int64_t* __restrict__ flops_out,
                               unsigned char* __restrict__ cls_out, DevCounters* cnt,
                               const float* __restrict__ prm, float margin,
                               int64_t* __restrict__ cap_out, int hash_shift) {
    analyze_kernel_body<IT>(R, D, rb, nprod, max_dense_n, dense_min, flops_out, cls_out, cnt,
        prm, margin, cap_out, hash_shift, (long long)blockIdx.x, (long long)gridDim.x);
}

// Features of every global row for the row-size predictor (log2(1 + .) of
// flops, |A(i,:)|, max_k |B(k,:)|, n, flops/|A(i,:)|, min(flops, n)).
template <class IT>
__global__ void row_features_kernel(long long R, const ProdDesc* __restrict__ D,
                                    const long long* __restrict__ rb, int nprod,
                                    float* __restrict__ X) {
    const int lane = lane_id();
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = warp; r < R; r += nwarps) {
        const RowCtx<IT, NoVal> c = row_ctx<IT, NoVal>(D, rb, nprod, r);
        long long f = 0, mx = 0;
        for (long long p = c.a0 + lane; p < c.a1; p += 32) {
            long long k = (long long)c.ciA[p];
            const long long len = c.rpB[k + 1] - c.rpB[k];
            f += len;
            mx = len > mx ? len : mx;
        }
        f = warp_sum(f);
        mx = warp_max(mx);
        if (lane == 0) {
            const long long d = c.a1 - c.a0;
            const long long ub = f < c.n ? f : c.n;
            float* x = X + r * kSizerF;
            x[0] = log2f(1.f + (float)f);
            x[1] = log2f(1.f + (float)d);
            x[2] = log2f(1.f + (float)mx);
            x[3] = log2f(1.f + (float)c.n);
            x[4] = log2f(1.f + (d > 0 ? (float)f / (float)d : 0.f));
            x[5] = log2f(1.f + (float)ub);
        }
    }
}

// ----------------------------------------------------------- checked mode
// One warp per row: rowptr monotone, columns in [0, ncols), strictly ascending.
template <class IT>
__global__ void validate_kernel(long long m, long long ncols, long long nnz, const int64_t* rp,
                                const int64_t* re, const IT* ci, int* err) {
    const int lane = lane_id();
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < m; i += nwarps) {
        long long a0 = rp[i], a1 = row_end(rp, re, i);
        if (a0 < 0 || a1 < a0 || a1 > nnz || (!re && i == 0 && a0 != 0)) {
            if (lane == 0) atomicExch(err, (int)kDevBadRowptr);
            continue;
        }
        for (long long p = a0 + lane; p < a1; p += 32) {
            long long c = (long long)ci[p];
            bool bad = c < 0 || c >= ncols || (p + 1 < a1 && (long long)ci[p + 1] <= c);
            if (bad) atomicExch(err, (int)kDevBadIndex);
        }
    }
}

// ------------------------------------------ short rows (hash bin 0)
// A row of at most 32 products needs no table.  Lane x takes the row's x-th
// product in ascending k (then in B(k,:)'s order): the A entries are read in
// batches of 32 and each batch's products are flattened onto the lanes after
// those of earlier batches; the owner of product f is the last entry whose
// exclusive prefix of run lengths is <= f (a five-step search over the
// lanes, always a lane of the batch).  Equal columns are then grouped with
// __match_any_sync.  Returns the number of products, or -1 if the row has
// more than 32 (a row of hash bin 0 never does).
template <class IT, class V, bool VALS>
__device__ __forceinline__ int short_row_gather(const RowCtx<IT, V>& c,
                                                typename KeyT<IT>::type& key, V& v) {
    using K = typename KeyT<IT>::type;
    const int lane = lane_id();
    int have = 0;
    key = K(-1);
    v = VOps<V>::init();
    for (long long b = c.a0; b < c.a1; b += 32) {
        const int nb = (int)min(32LL, c.a1 - b);
        long long lo = 0;
        int len = 0;
        V a = VOps<V>::init();
        if (lane < nb) {
            const long long k = (long long)c.ciA[b + lane];
            lo = c.rpB[k];
            // capped: more than 32 products in one B row already makes the
            // row too long for this path, and keeps the scan in int range
            len = (int)min(c.rpB[k + 1] - lo, 33LL);
            if constexpr (VALS) a = load_val(c.vA, b + lane);
        }
        const int incl = warp_incl_scan(len);
        const int tot = __shfl_sync(kFull, incl, 31);
        if (tot == 0) continue;
        if (have + tot > 32) return -1;
        const int excl = incl - len;
        const int f = lane - have;
        int e = 0;
#pragma unroll
        for (int w = 16; w; w >>= 1) {
            const int cand = e + w;
            const int ex = __shfl_sync(kFull, excl, cand & 31);
            if (cand < nb && ex <= f) e = cand;
        }
        const long long lo_e = __shfl_sync(kFull, lo, e);
        const int ex_e = __shfl_sync(kFull, excl, e);
        const V a_e = shfl_val(a, e);
        if (f >= 0 && f < tot) {
            const long long q = lo_e + (f - ex_e);
            key = (K)c.ciB[q];
            if constexpr (VALS) v = VOps<V>::mul(a_e, load_val(c.vB, q));
        }
        have += tot;
    }
    return have;
}

// Symbolic count of a short row: the number of distinct columns.
template <class IT>
__device__ __forceinline__ void short_row_symbolic(const RowCtx<IT, NoVal>& c, long long r,
                                                   int64_t* __restrict__ rowcnt, int* err) {
    using K = typename KeyT<IT>::type;
    const int lane = lane_id();
    K key;
    NoVal v;
    const int np = short_row_gather<IT, NoVal, false>(c, key, v);
    if (np < 0) {
        if (lane == 0) atomicExch(err, (int)kDevTableFull);
        return;
    }
    const bool valid = lane < np;
    const K kk = valid ? key : (K)(-1 - lane);
    const unsigned grp = __match_any_sync(kFull, kk);
    const bool leader = valid && (grp & lanemask_lt()) == 0u;
    const int cnt = __popc(__ballot_sync(kFull, leader));
    if (lane == 0) rowcnt[r] = cnt;
}

// Numeric pass of a short row: the lowest lane of each group of equal
// columns adds the group's products in lane order from the identity (the
// order in which the hash path adds them), and writes its column at the
// number of groups with a smaller column.  Slot mode as in the hash path.
template <class IT, class V>
__device__ __forceinline__ void short_row_numeric(const RowCtx<IT, V>& c, long long r,
                                                  const int64_t* __restrict__ rpC, long long cap,
                                                  IT* __restrict__ ciC, V* __restrict__ vC,
                                                  int* err, int64_t* __restrict__ rowend,
                                                  int32_t* __restrict__ overflow,
                                                  unsigned* overflow_count) {
    using K = typename KeyT<IT>::type;
    constexpr bool HV = VOps<V>::has_val;
    const int lane = lane_id();
    // the output range does not depend on the products: loaded first
    const long long out = rpC[r];
    long long rcnt = rpC[r + 1] - out;
    K key;
    V v;
    const int np = short_row_gather<IT, V, HV>(c, key, v);
    if (np < 0) {
        if (lane == 0) atomicExch(err, (int)kDevTableFull);
        return;
    }
    const bool valid = lane < np;
    const K kk = valid ? key : (K)(-1 - lane);
    const unsigned grp = __match_any_sync(kFull, kk);
    const bool leader = valid && (grp & lanemask_lt()) == 0u;
    const unsigned L = __ballot_sync(kFull, leader);
    const int cnt = __popc(L);
    V sum = VOps<V>::init();
    if constexpr (HV) {
        unsigned rem = leader ? grp : 0u;
        const int maxc = (int)__reduce_max_sync(kFull, (unsigned)__popc(rem));
        for (int t = 0; t < maxc; ++t) {
            const int src = rem ? __ffs(rem) - 1 : lane;
            const V x = shfl_val(v, src);
            if (rem) {
                sum = VOps<V>::add(sum, x);
                rem &= rem - 1u;
            }
        }
    }
    int pos = 0;
    for (unsigned Lr = L; Lr; Lr &= Lr - 1u) {
        const K kj = __shfl_sync(kFull, kk, __ffs(Lr) - 1);
        pos += kj < kk ? 1 : 0;
    }
    if (rowend != nullptr) {
        if (cnt > rcnt) {
            if (lane == 0) {
                overflow[atomicAdd(overflow_count, 1u)] = (int32_t)r;
                rowend[r] = -1;
            }
            return;
        }
        rcnt = cnt;
        if (lane == 0) rowend[r] = out + cnt;
    } else if (cnt != rcnt && lane == 0) {
        atomicExch(err, (int)kDevCountMismatch);
    }
    if (out + rcnt > cap && lane == 0) atomicExch(err, (int)kDevCapacity);
    if (leader && pos < rcnt && out + pos < cap) {
        ciC[out + pos] = (IT)kk;
        if constexpr (HV) vC[out + pos] = sum;
    }
}

// --------------------------------------------------- symbolic: hash rows
// One warp per row; table of 2^LOG2T keys per warp.  Row count -> rowcnt[i].
template <class IT, int LOG2T, int WARPS>
__device__ __forceinline__ void symbolic_hash_kernel_body(
    const ProdDesc* __restrict__ D, const long long* __restrict__ rb,
                         int nprod, const int32_t* __restrict__ rows, const DevCounters* cnt,
                         int cls, int64_t* __restrict__ rowcnt, int* err,
        const long long vbid, const long long vnb) {
    using K = typename KeyT<IT>::type;
    constexpr int T = 1 << LOG2T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const int w = threadIdx.x >> 5;
    const long long nrows = (long long)cnt->class_count[cls];
    const int32_t* crow = rows + cnt->class_off[cls];
    const long long gw = (long long)vbid * WARPS + w;
    const long long nw = (long long)vnb * WARPS;
    if constexpr (LOG2T == kShortLog2T) {
        // rows of at most 32 products: no table
        for_class_rows<IT, NoVal>(D, rb, nprod, crow, gw, nrows, nw,
                                  [&](const RowCtx<IT, NoVal>& c, long long r) {
                                      short_row_symbolic<IT>(c, r, rowcnt, err);
                                  });
        return;
    }
    K* keys = reinterpret_cast<K*>(smem_raw) + (size_t)w * T;
    for (int s = lane; s < T; s += 32) keys[s] = K(-1);
    __syncwarp();
    for (long long rr = gw; rr < nrows; rr += nw) {
        const long long r = crow[rr];
        const RowCtx<IT, NoVal> c = row_ctx<IT, NoVal>(D, rb, nprod, r);
        const long long a0 = c.a0, a1 = c.a1;
        const IT* ciA = c.ciA;
        const int64_t* rpB = c.rpB;
        const IT* ciB = c.ciB;
        int count = 0;
        for (long long b = a0; b < a1; b += 32) {
            const int nb = (int)min(32LL, a1 - b);
            long long lo = 0;
            int len = 0;
            if (lane < nb) {
                long long k = (long long)ciA[b + lane];
                lo = rpB[k];
                len = (int)(rpB[k + 1] - lo);
            }
            walk_flat4(nb, lo, len, [&](const long long (&q)[4], const int (&)[4],
                                        const bool (&valid)[4]) {
                K kk[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) kk[t] = valid[t] ? (K)ciB[q[t]] : K(-1);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    bool is_new = false;
                    if (valid[t]) hash_insert<LOG2T>(keys, kk[t], is_new, err);
                    count += __popc(__ballot_sync(kFull, is_new));
                }
            });
        }
        if (lane == 0) rowcnt[r] = count;
        for (int s = lane; s < T; s += 32) keys[s] = K(-1);
        __syncwarp();
    }
}

template <class IT, int LOG2T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    symbolic_hash_kernel(const ProdDesc* __restrict__ D, const long long* __restrict__ rb,
                         int nprod, const int32_t* __restrict__ rows, const DevCounters* cnt,
                         int cls, int64_t* __restrict__ rowcnt, int* err) {
    symbolic_hash_kernel_body<IT, LOG2T, WARPS>(D, rb, nprod, rows, cnt, cls, rowcnt, err,
        (long long)blockIdx.x, (long long)gridDim.x);
}

// -------------------------------------------------- symbolic: dense rows
// One block per row (dynamic row grabbing), bitmap of the product's n columns
// in shared memory (sized for the largest n of the batch).  Also writes the
// per-chunk counts chunkcnt[chunk_base + i*P + c] (chunk c covers columns
// [c*W, (c+1)*W)), which the numeric phase uses to skip empty chunks.
// MAXT / MINB: launch bounds of the instantiation (a register cap that lets
// six 256-thread or three 512-thread blocks share an SM, or one 1024-thread
// block for a bitmap that leaves room for only one block).
// Groups: the block may be split into `groups` equal groups of whole warps
// (named barriers 1..groups), each with its own bitmap of max_words words,
// so that several rows are in flight in one block; groups == 1 is the
// whole block.
constexpr int kMaxSymGroups = 8;

__device__ __forceinline__ void group_sync(int g, int gthreads, int groups) {
    if (groups == 1) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(gthreads) : "memory");
}

template <class IT, int MAXT, int MINB>
__device__ __forceinline__ void symbolic_dense_kernel_body(const ProdDesc* __restrict__ D,
                                      const long long* __restrict__ rb, int nprod,
                                      const int32_t* __restrict__ rows, const DevCounters* cnt,
                                      int max_words, int chunk_words,
                                      int32_t* __restrict__ chunkcnt, int64_t* __restrict__ rowcnt,
                                      unsigned long long* work, int* err,
        const long long vbid, const long long vnb, const int groups = 1) {
    extern __shared__ unsigned bm_all[];
    __shared__ long long row_total_g[kMaxSymGroups];
    __shared__ long long cur_row_g[kMaxSymGroups];
    const int gthreads = blockDim.x / groups;
    const int g = threadIdx.x / gthreads;
    const int gt = threadIdx.x - g * gthreads;
    unsigned* bm = bm_all + (size_t)g * max_words;
    long long& row_total = row_total_g[g];
    long long& cur_row = cur_row_g[g];
    const int lane = lane_id();
    const int w = gt >> 5;
    const int nwarps = gthreads >> 5;
    unsigned long long nd = 0;
    for (int t = kClassDense0; t < kNumClasses; ++t) nd += cnt->class_count[t];
    const long long nrows = (long long)nd;
    const int32_t* drow = rows + cnt->class_off[kClassDense0];
    for (int t = gt; t < max_words; t += gthreads) bm[t] = 0u;
    if (gt == 0) row_total = 0;
    group_sync(g, gthreads, groups);
    while (true) {
        if (gt == 0) cur_row = (long long)atomicAdd(work, 1ull);
        group_sync(g, gthreads, groups);
        const long long rr = cur_row;
        if (rr >= nrows) break;
        const long long r = drow[rr];
        const RowCtx<IT, NoVal> cx = row_ctx<IT, NoVal>(D, rb, nprod, r);
        const long long a0 = cx.a0, a1 = cx.a1;
        const IT* ciA = cx.ciA;
        const int64_t* rpB = cx.rpB;
        const IT* ciB = cx.ciB;
        const int NW = (int)((cx.n + 31) >> 5);
        const int P = cx.P;
        if (NW > max_words) {  // n beyond the shared-memory bitmap: reported, row skipped
            if (gt == 0) atomicExch(err, (int)kDevTooWide);
            group_sync(g, gthreads, groups);
            continue;
        }
        for (long long b = a0 + (long long)w * 32; b < a1; b += (long long)nwarps * 32) {
            const int nb = (int)min(32LL, a1 - b);
            long long lo = 0;
            int len = 0;
            if (lane < nb) {
                long long k = (long long)ciA[b + lane];
                lo = rpB[k];
                len = (int)(rpB[k + 1] - lo);
            }
            walk_batch4(nb, lo, len, [&](const long long (&q)[4], const int (&)[4],
                                         const bool (&valid)[4], bool) {
                long long j[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) j[t] = valid[t] ? (long long)ciB[q[t]] : -1;
                // one shared atomic per product: OR-ing the lanes' bits of a
                // common word first (a segmented scan, or __match_any_sync with
                // __reduce_or_sync) was measured 3x and 5x slower
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (j[t] >= 0) atomicOr(&bm[j[t] >> 5], 1u << (j[t] & 31));
            });
        }
        group_sync(g, gthreads, groups);
        long long part = 0;
        for (int c = w; c < P; c += nwarps) {
            const int w0 = c * chunk_words;
            const int w1 = min(NW, w0 + chunk_words);
            int s = 0;
            for (int t = w0 + lane; t < w1; t += 32) {
                s += __popc(bm[t]);
                bm[t] = 0u;
            }
            s = warp_sum(s);
            if (lane == 0) chunkcnt[cx.chunk_base + cx.i * P + c] = s;
            part += s;
        }
        if (lane == 0 && part) atomicAdd((unsigned long long*)&row_total, (unsigned long long)part);
        group_sync(g, gthreads, groups);
        if (gt == 0) {
            rowcnt[r] = row_total;
            row_total = 0;
        }
        group_sync(g, gthreads, groups);
    }
}

template <class IT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) symbolic_dense_kernel(const ProdDesc* __restrict__ D,
                                      const long long* __restrict__ rb, int nprod,
                                      const int32_t* __restrict__ rows, const DevCounters* cnt,
                                      int max_words, int chunk_words,
                                      int32_t* __restrict__ chunkcnt, int64_t* __restrict__ rowcnt,
                                      unsigned long long* work, int* err) {
    symbolic_dense_kernel_body<IT, MAXT, MINB>(D, rb, nprod, rows, cnt, max_words, chunk_words,
        chunkcnt, rowcnt, work, err, (long long)blockIdx.x, (long long)gridDim.x);
}

// ---------------------------------------------------- numeric: hash rows
template <class K, class V>
__device__ __forceinline__ void warp_bitonic_sort(K* keys, V* vals, int N) {
    const int lane = lane_id();
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < N; i += 32) {
                int ixj = i ^ j;
                if (ixj > i) {
                    K ki = keys[i], kj = keys[ixj];
                    bool up = (i & k) == 0;
                    if ((ki > kj) == up) {
                        keys[i] = kj;
                        keys[ixj] = ki;
                        if constexpr (VOps<V>::has_val) {
                            V t = vals[i];
                            vals[i] = vals[ixj];
                            vals[ixj] = t;
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Stable LSD radix sort of N (key, value) pairs by one warp, 8-bit digits
// over the low `bits` bits of the keys (keys are >= 0).  Ping-pongs between
// (k0, v0) and (k1, v1); returns true if the sorted pairs end in (k1, v1).
// Each pass: digit histogram, exclusive scan, then a scatter in rounds of 32
// keys in input order where lanes with equal digits take consecutive slots
// in lane order, so equal digits keep their input order.
template <class K, class V>
__device__ __forceinline__ bool warp_radix_sort(K* k0, V* v0, K* k1, V* v1, int N, int bits,
                                                int* cnt) {
    constexpr bool HV = VOps<V>::has_val;
    const int lane = lane_id();
    bool flip = false;
    for (int shift = 0; shift < bits; shift += 8) {
        K* kin = flip ? k1 : k0;
        V* vin = flip ? v1 : v0;
        K* kout = flip ? k0 : k1;
        V* vout = flip ? v0 : v1;
        for (int t = lane; t < 256; t += 32) cnt[t] = 0;
        __syncwarp();
        for (int i = lane; i < N; i += 32) atomicAdd(&cnt[(int)((kin[i] >> shift) & 255)], 1);
        __syncwarp();
        int loc[8];
        int sum = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            loc[t] = cnt[lane * 8 + t];
            sum += loc[t];
        }
        int run = warp_incl_scan(sum) - sum;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            cnt[lane * 8 + t] = run;
            run += loc[t];
        }
        __syncwarp();
        for (int i0 = 0; i0 < N; i0 += 32) {
            const int i = i0 + lane;
            const bool valid = i < N;
            K kk = valid ? kin[i] : K(0);
            V vv{};
            if constexpr (HV)
                if (valid) vv = vin[i];
            const int d = valid ? (int)((kk >> shift) & 255) : 256 + lane;
            const unsigned grp = __match_any_sync(kFull, d);
            const int rank = __popc(grp & lanemask_lt());
            const int base = valid ? cnt[d] : 0;
            __syncwarp();
            if (valid) {
                kout[base + rank] = kk;
                if constexpr (HV) vout[base + rank] = vv;
                if ((grp >> lane) == 1u) cnt[d] = base + __popc(grp);  // highest lane of the group
            }
            __syncwarp();
        }
        flip = !flip;
    }
    return flip;
}

// One warp per row; table of 2^LOG2T (key, value) slots; products added in
// ascending k (ordered rounds); table compacted, sorted, written.
template <class IT, class V, int LOG2T, int WARPS>
__device__ __forceinline__ void numeric_hash_kernel_body(
    const ProdDesc* __restrict__ D, const long long* __restrict__ rb,
                        int nprod, const int32_t* __restrict__ rows, const DevCounters* cnt,
                        int cls, const int64_t* __restrict__ rpC, long long cap,
                        IT* __restrict__ ciC, V* __restrict__ vC, int* err,
                        int64_t* __restrict__ rowend, int32_t* __restrict__ overflow,
                        unsigned* overflow_count,
        const long long vbid, const long long vnb) {
    using K = typename KeyT<IT>::type;
    constexpr int T = 1 << LOG2T;
    constexpr bool HV = VOps<V>::has_val;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const int w = threadIdx.x >> 5;
    if constexpr (LOG2T == kShortLog2T) {
        // rows of at most 32 products: no table
        const long long nrows = (long long)cnt->class_count[cls];
        const int32_t* crow = rows + cnt->class_off[cls];
        const long long gw = (long long)vbid * WARPS + w;
        const long long nw = (long long)vnb * WARPS;
        for_class_rows<IT, V>(D, rb, nprod, crow, gw, nrows, nw,
                              [&](const RowCtx<IT, V>& c, long long r) {
                                  short_row_numeric<IT, V>(c, r, rpC, cap, ciC, vC, err, rowend,
                                                           overflow, overflow_count);
                              });
        return;
    }
    // layout per warp: T values (if any), T keys, 256 radix counters
    constexpr size_t vbytes = HV ? sizeof(V) * T : 0;
    unsigned char* base = smem_raw + (size_t)w * (vbytes + sizeof(K) * T + 256 * sizeof(int));
    V* acc = reinterpret_cast<V*>(base);
    K* keys = reinterpret_cast<K*>(base + vbytes);
    int* rcnt_smem = reinterpret_cast<int*>(base + vbytes + sizeof(K) * T);
    // slot mode (learned sizing): rows go to predicted slots [rpC[r], rpC[r+1]);
    // a row that does not fit its slot or its table is listed for an exact re-run
    const bool slot_mode = rowend != nullptr;
    __shared__ int warp_fail[WARPS];
    int* fail = slot_mode ? &warp_fail[w] : err;
    if (lane == 0) warp_fail[w] = 0;
    __syncwarp();
    for (int s = lane; s < T; s += 32) {
        keys[s] = K(-1);
        if constexpr (HV) acc[s] = VOps<V>::init();
    }
    __syncwarp();
    const long long nrows = (long long)cnt->class_count[cls];
    const int32_t* crow = rows + cnt->class_off[cls];
    const long long gw = (long long)vbid * WARPS + w;
    const long long nw = (long long)vnb * WARPS;
    for (long long rr = gw; rr < nrows; rr += nw) {
        const long long r = crow[rr];
        const RowCtx<IT, V> c = row_ctx<IT, V>(D, rb, nprod, r);
        const long long a0 = c.a0, a1 = c.a1;
        const IT* ciA = c.ciA;
        const V* vA = c.vA;
        const int64_t* rpB = c.rpB;
        const IT* ciB = c.ciB;
        const V* vB = c.vB;
        // A row of at most 32 A entries has its one batch loaded here, once.
        // If its products hardly repeat a column (nnz(C(i,:)) >= 3/4 of its
        // flops, known exactly outside slot mode) and fit half the table, it
        // is expanded, sorted and compressed instead of hashed: products go
        // to the table's lower half in ascending k, a stable radix sort by
        // column keeps that order among equal columns, and each run of equal
        // columns is reduced from the identity in that order, as the hash
        // path would.
        bool pre = false;
        long long lo_p = 0;
        int len_p = 0;
        V a_p = VOps<V>::init();
        if constexpr (LOG2T >= 10) {
            if (!slot_mode && a1 > a0 && a1 - a0 <= 32) {
                const int nb = (int)(a1 - a0);
                if (lane < nb) {
                    const long long k = (long long)ciA[a0 + lane];
                    lo_p = rpB[k];
                    len_p = (int)(rpB[k + 1] - lo_p);
                    a_p = load_val(vA, a0 + lane);
                }
                pre = true;
                const long long fl = warp_sum((long long)len_p);
                const long long nz = rpC[r + 1] - rpC[r];
                if (fl <= T / 2 && 4 * nz >= 3 * fl) {
                    int nf = 0;
                    walk_batch4(nb, lo_p, len_p, [&](const long long (&q)[4], const int (&e)[4],
                                                     const bool (&vl)[4], bool) {
                        K key[4];
                        V bq[4];
                        V ae[4];
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            ae[t] = shfl_val(a_p, e[t]);
                            key[t] = K(0);
                            bq[t] = V{};
                            if (vl[t]) {
                                key[t] = (K)ciB[q[t]];
                                bq[t] = load_val(vB, q[t]);
                            }
                        }
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            // the valid lanes of a round are a prefix of the warp
                            if (vl[t]) {
                                keys[nf + lane] = key[t];
                                if constexpr (HV) acc[nf + lane] = VOps<V>::mul(ae[t], bq[t]);
                            }
                            nf += __popc(__ballot_sync(kFull, vl[t]));
                        }
                    });
                    __syncwarp();
                    const int bits = c.n > 1 ? 64 - __clzll((unsigned long long)(c.n - 1)) : 1;
                    const bool up = warp_radix_sort<K, V>(keys, acc, keys + T / 2, acc + T / 2, nf,
                                                          bits, rcnt_smem);
                    const K* sk = up ? keys + T / 2 : keys;
                    const V* sv = up ? acc + T / 2 : acc;
                    const long long out = rpC[r];
                    int outp = 0;
                    for (int i0 = 0; i0 < nf; i0 += 32) {
                        const int i = i0 + lane;
                        const bool in = i < nf;
                        const K kk = in ? sk[i] : K(0);
                        const bool start = in && (i == 0 || sk[i - 1] != kk);
                        const unsigned sm = __ballot_sync(kFull, start);
                        if (start) {
                            V sum = VOps<V>::init();
                            if constexpr (HV) {
                                sum = VOps<V>::add(sum, sv[i]);
                                for (int j = i + 1; j < nf && sk[j] == kk; ++j)
                                    sum = VOps<V>::add(sum, sv[j]);
                            }
                            const long long pq = out + outp + __popc(sm & lanemask_lt());
                            if (pq < cap) {
                                ciC[pq] = (IT)kk;
                                if constexpr (HV) vC[pq] = sum;
                            }
                        }
                        outp += __popc(sm);
                    }
                    if (lane == 0 && (long long)outp != nz) atomicExch(err, (int)kDevCountMismatch);
                    if (lane == 0 && out + outp > cap) atomicExch(err, (int)kDevCapacity);
                    __syncwarp();
                    // both halves back to the empty table
                    for (int t = lane; t < nf; t += 32) {
                        keys[t] = K(-1);
                        keys[T / 2 + t] = K(-1);
                        if constexpr (HV) {
                            acc[t] = VOps<V>::init();
                            acc[T / 2 + t] = VOps<V>::init();
                        }
                    }
                    __syncwarp();
                    continue;
                }
            }
        }
        for (long long b = a0; b < a1; b += 32) {
            const int nb = (int)min(32LL, a1 - b);
            long long lo = 0;
            int len = 0;
            V a = VOps<V>::init();
            if (pre) {  // the row's single batch, loaded above
                lo = lo_p;
                len = len_p;
                a = a_p;
            } else if (lane < nb) {
                long long k = (long long)ciA[b + lane];
                lo = rpB[k];
                len = (int)(rpB[k + 1] - lo);
                a = load_val(vA, b + lane);
            }
            // four rounds per step: their loads are issued together, then
            // the rounds are inserted and accumulated in order
            walk_batch4(nb, lo, len, [&](const long long (&q)[4], const int (&e)[4],
                                         const bool (&vl)[4], bool ordered) {
                K key[4];
                V bq[4];
                V ae[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    ae[t] = shfl_val(a, e[t]);
                    key[t] = K(-1);
                    bq[t] = V{};
                    if (vl[t]) {
                        key[t] = (K)ciB[q[t]];
                        bq[t] = load_val(vB, q[t]);
                    }
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    int slot = -1;
                    V v{};
                    if (vl[t]) {
                        bool is_new;
                        slot = hash_insert<LOG2T>(keys, key[t], is_new, fail);
                        v = VOps<V>::mul(ae[t], bq[t]);
                    }
                    const bool valid = vl[t] && slot >= 0;
                    if (ordered) ordered_add(acc, slot, valid, v);
                    else plain_add(acc, slot, valid, v);
                }
            });
        }
        // compact occupied slots to the front (ascending slot order)
        const long long out = rpC[r];
        int rcnt = (int)(rpC[r + 1] - out);
        int pos = 0;
        for (int s0 = 0; s0 < T; s0 += 32) {
            K kk = keys[s0 + lane];
            V vv{};
            if constexpr (HV) vv = acc[s0 + lane];
            bool occ = kk != K(-1);
            unsigned msk = __ballot_sync(kFull, occ);
            __syncwarp();
            int p = pos + __popc(msk & lanemask_lt());
            if (occ) {
                keys[p] = kk;
                if constexpr (HV) acc[p] = vv;
            }
            pos += __popc(msk);
            __syncwarp();
        }
        if (slot_mode) {
            __syncwarp();
            const bool bad = warp_fail[w] != 0 || pos > rcnt;
            if (bad) {
                if (lane == 0) {
                    overflow[atomicAdd(overflow_count, 1u)] = (int32_t)r;
                    rowend[r] = -1;
                    warp_fail[w] = 0;
                }
                for (int sl = lane; sl < T; sl += 32) {
                    keys[sl] = K(-1);
                    if constexpr (HV) acc[sl] = VOps<V>::init();
                }
                __syncwarp();
                continue;
            }
            rcnt = pos;
            if (lane == 0) rowend[r] = out + pos;
        } else if (pos != rcnt && lane == 0) {
            atomicExch(err, (int)kDevCountMismatch);
        }
        if (out + rcnt > cap && lane == 0) atomicExch(err, (int)kDevCapacity);
        const K* sk = keys;
        const V* sv = acc;
        if (pos <= 64) {
            int N = 1;
            while (N < pos) N <<= 1;
            const K kmax = sizeof(K) == 4 ? (K)0x7fffffff : (K)0x7fffffffffffffffLL;
            for (int s = pos + lane; s < N; s += 32) keys[s] = kmax;
            __syncwarp();
            warp_bitonic_sort<K, V>(keys, acc, N);
        } else {
            // pos <= T/2: the upper half of the table is the second buffer
            const int bits = c.n > 1 ? 64 - __clzll((unsigned long long)(c.n - 1)) : 1;
            const bool in_upper = warp_radix_sort<K, V>(keys, acc, keys + T / 2, acc + T / 2, pos,
                                                        bits, rcnt_smem);
            if (in_upper) {
                sk = keys + T / 2;
                sv = acc + T / 2;
            }
        }
        const int lim = (int)max(0LL, min((long long)min(pos, rcnt), cap - out));
        for (int t = lane; t < lim; t += 32) {
            ciC[out + t] = (IT)sk[t];
            if constexpr (HV) vC[out + t] = sv[t];
        }
        __syncwarp();
        for (int s = lane; s < T; s += 32) {
            keys[s] = K(-1);
            if constexpr (HV) acc[s] = VOps<V>::init();
        }
        __syncwarp();
    }
}

template <class IT, class V, int LOG2T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    numeric_hash_kernel(const ProdDesc* __restrict__ D, const long long* __restrict__ rb,
                        int nprod, const int32_t* __restrict__ rows, const DevCounters* cnt,
                        int cls, const int64_t* __restrict__ rpC, long long cap,
                        IT* __restrict__ ciC, V* __restrict__ vC, int* err,
                        int64_t* __restrict__ rowend, int32_t* __restrict__ overflow,
                        unsigned* overflow_count) {
    numeric_hash_kernel_body<IT, V, LOG2T, WARPS>(D, rb, nprod, rows, cnt, cls, rpC, cap, ciC,
        vC, err, rowend, overflow, overflow_count, (long long)blockIdx.x, (long long)gridDim.x);
}

// --------------------------------------------------- numeric: dense rows
// Work units: a dense row's P column chunks (width W) are cut into G equal
// segments (G in {1, 2, 4, ..., kSegGrid}, chosen per flops class so that a
// unit carries a bounded share of flops); one warp owns a unit.  For each
// chunk of its segment the warp walks A(i,:) in order and, per entry, the part
// of B(k,:) inside the chunk, found from a cursor that the previous chunk left
// (the first cursor of a segment comes from segtab, the position of the first
// column >= the segment start in every B row).  Products go into a dense
// accumulator acc[W] with presence flags, in ascending k; the chunk is then
// emitted in column order.  Cursors live in a per-warp arena slot.


__host__ __device__ __forceinline__ long long seg_chunk(int g, int P) {
    return ((long long)g * P) / kSegGrid;
}

// Where a warp stands in B(k,:) while it sweeps the chunks of a row: the
// first unconsumed position, its column (INT_MAX once B(k,:) is used up) and
// its run length (entries from pos to the end of that column's chunk).
struct __align__(16) DenseCursor {
    long long pos;
    int col;
    int rl;
};

// One run of a batch in the dense numeric kernel: the flattened product f
// of the run sits at B position off + f, and is scaled by a = A(i,k).
template <class V>
struct __align__(16) DenseRun {
    long long off;
    V a;
};

// runlen[run_base + q] = number of entries from q to the end of q's column
// chunk (col / W) inside its row of B: the length of the part of B(k,:) that
// a chunk sweep consumes in one step.  nextrun[run_base + q] = {length, first
// column} of the run that follows the one starting at q ({0, INT_MAX} at the
// row's end), so a cursor advances with one load whose address it knows
// before the chunk's products are accumulated.  One warp per B row of every
// product: run lengths in windows of 32 from the row end backwards, then the
// successor table in a forward pass over what the warp wrote.
template <class IT>
__device__ __forceinline__ void runlen_kernel_body(long long LB, const ProdDesc* __restrict__ D,
                              const long long* __restrict__ bb, int nprod, int W,
                              int32_t* __restrict__ runlen, int2* __restrict__ nextrun,
                              const DevCounters* cnt,
        const long long vbid, const long long vnb) {
    if (cnt->class_off[kNumClasses] == cnt->class_off[kClassDense0]) return;  // no dense rows
    const int lane = lane_id();
    const long long warp = ((long long)vbid * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)vnb * blockDim.x) >> 5;
    for (long long kb = warp; kb < LB; kb += nwarps) {
        const int pr = nprod > 1 ? find_prod(bb, nprod, kb) : 0;
        const ProdDesc& d = D[pr];
        const long long k = kb - d.brow_base;
        const IT* ciB = (const IT*)d.ciB;
        int32_t* rl = runlen + d.run_base;
        int2* nr = nextrun + d.run_base;
        const long long s0 = d.rpB[k], s1 = d.rpB[k + 1];
        long long carry_end = s1;          // run end of the window after this one
        long long carry_chunk = -1;        // chunk of the first entry of that window
        for (long long hi = s1; hi > s0; hi -= 32) {
            const long long lo = max(s0, hi - 32);
            const long long q = lo + lane;
            const bool in = q < hi;
            const long long ch = in ? (long long)ciB[q] / W : -2;
            long long nxt = __shfl_down_sync(kFull, ch, 1);
            if (lane == 31 || q + 1 >= hi) nxt = carry_chunk;
            const bool last = in && nxt != ch;   // q ends its run inside this window
            const unsigned lm = __ballot_sync(kFull, last);
            const unsigned ge = lm & (0xffffffffu << lane);
            long long end;
            if (ge) end = lo + (__ffs(ge) - 1) + 1;
            else end = carry_end;
            if (in) rl[q] = (int32_t)(end - q);
            // first entry of this window seeds the carry for the window before it
            carry_end = __shfl_sync(kFull, end, 0);
            carry_chunk = __shfl_sync(kFull, ch, 0);
        }
        __syncwarp();   // the run lengths of the whole row are visible to the warp
        for (long long q = s0 + lane; q < s1; q += 32) {
            const long long q2 = q + rl[q];
            int2 x = make_int2(0, 0x7fffffff);
            if (q2 < s1) x = make_int2(rl[q2], (int)ciB[q2]);
            nr[q] = x;
        }
        __syncwarp();
    }
}

template <class IT>
__global__ void runlen_kernel(long long LB, const ProdDesc* __restrict__ D,
                              const long long* __restrict__ bb, int nprod, int W,
                              int32_t* __restrict__ runlen, int2* __restrict__ nextrun,
                              const DevCounters* cnt) {
    runlen_kernel_body<IT>(LB, D, bb, nprod, W, runlen, nextrun, cnt, (long long)blockIdx.x,
        (long long)gridDim.x);
}

// segtab[seg_base + k * (kSegGrid+1) + g] = first position p in B(k,:) with
// col >= seg_chunk(g, P) * W, relative to rowptr[k].
template <class IT>
__device__ __forceinline__ void segtab_kernel_body(long long LB, const ProdDesc* __restrict__ D,
                              const long long* __restrict__ bb, int nprod, int W,
                              int32_t* __restrict__ segtab, const DevCounters* cnt,
        const long long vbid, const long long vnb) {
    if (cnt->class_off[kNumClasses] == cnt->class_off[kClassDense0]) return;  // no dense rows
    const long long total = LB * (kSegGrid + 1);
    for (long long t = (long long)vbid * blockDim.x + threadIdx.x; t < total;
         t += (long long)vnb * blockDim.x) {
        const long long kb = t / (kSegGrid + 1);
        const int g = (int)(t - kb * (kSegGrid + 1));
        const int pr = nprod > 1 ? find_prod(bb, nprod, kb) : 0;
        const ProdDesc& d = D[pr];
        const long long k = kb - d.brow_base;
        const IT* ciB = (const IT*)d.ciB;
        const long long key = seg_chunk(g, d.P) * W;
        long long lo = d.rpB[k], hi = d.rpB[k + 1];
        const long long base = lo;
        while (lo < hi) {
            long long mid = (lo + hi) >> 1;
            if ((long long)ciB[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        segtab[d.seg_base + k * (kSegGrid + 1) + g] = (int32_t)(lo - base);
    }
}

template <class IT>
__global__ void segtab_kernel(long long LB, const ProdDesc* __restrict__ D,
                              const long long* __restrict__ bb, int nprod, int W,
                              int32_t* __restrict__ segtab, const DevCounters* cnt) {
    segtab_kernel_body<IT>(LB, D, bb, nprod, W, segtab, cnt, (long long)blockIdx.x,
        (long long)gridDim.x);
}

// Products of one batch of (up to 32) A entries inside the chunk starting at
// column c0: lane e holds entry e's run (here, its B position pos, length len
// and a = A(i,k)).  The runs are flattened into rounds of 32 products in
// ascending k, four rounds per step so that their loads overlap; a round's
// products are multiplied and added in k order (lanes of one round that hit
// the same slot add in lane order, i.e. in ascending k).
template <class IT, class V>
__device__ __forceinline__ void dense_batch(bool here, long long pos, int len, V a, long long c0,
                                            const IT* __restrict__ ciB, const V* __restrict__ vB,
                                            V* acc, unsigned* bm, DenseRun<V>* runs) {
    const unsigned hmask = __ballot_sync(kFull, here);
    const int mylen = here ? len : 0;
    const int incl = warp_incl_scan(mylen);
    const int excl = incl - mylen;
    const int total = __shfl_sync(kFull, incl, 31);
    // nonempty runs in k order: run e starts at flattened position excl_e, its
    // products are B[off_e + f] for f in the run
    if (here) {
        DenseRun<V> re;
        re.off = pos - excl;
        re.a = a;
        runs[__popc(hmask & lanemask_lt())] = re;
    }
    __syncwarp();
    // The run of lane x in the round starting at w0 is (runs started before
    // w0) + (runs starting in [w0, w0 + x]) - 1, from an OR of start bits.
    int started = 0;
    for (int f0 = 0; f0 < total; f0 += 128) {
        const int nsub = min(4, (total - f0 + 31) >> 5);
        long long jj[4];
        V bv[4];
        V av[4];
        bool vl[4];
        bool multi[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            vl[t] = false;
            multi[t] = false;
            jj[t] = c0;
            bv[t] = V{};
            av[t] = V{};
            if (t < nsub) {
                const int w0 = f0 + 32 * t;
                const unsigned sbit =
                    (here && excl >= w0 && excl < w0 + 32) ? (1u << (excl - w0)) : 0u;
                const unsigned M = __reduce_or_sync(kFull, sbit);
                const int e = started + __popc(M & lanemask_le()) - 1;
                started += __popc(M);
                multi[t] = (M & ~1u) != 0u;
                const int fi = w0 + lane_id();
                vl[t] = fi < total;
                if (vl[t]) {
                    const DenseRun<V> re = runs[e];
                    const long long q = re.off + fi;
                    jj[t] = (long long)ciB[q];
                    bv[t] = load_val(vB, q);
                    av[t] = re.a;
                }
            }
        }
        V v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            v[t] = V{};
            if (t < nsub && vl[t]) v[t] = VOps<V>::mul(av[t], bv[t]);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (t < nsub) {
                const int slot = (int)(jj[t] - c0);
                if (vl[t]) atomicOr(&bm[slot >> 5], 1u << (slot & 31));
                if (multi[t]) ordered_add(acc, slot, vl[t], v[t]);
                else plain_add(acc, slot, vl[t], v[t]);
            }
        }
    }
    __syncwarp();
}

// The register cap (three 8-warp or six 4-warp blocks per SM) keeps 24
// warps resident, which the shared-memory accumulators allow.
template <class IT, class V, int W, int WARPS>
__device__ __forceinline__ void numeric_dense_kernel_body(
    const ProdDesc* __restrict__ D, const long long* __restrict__ rb,
                         int nprod, const int32_t* __restrict__ rows, const DevCounters* cnt,
                         const int32_t* __restrict__ chunkcnt, const int32_t* __restrict__ segtab,
                         const int32_t* __restrict__ runlen, const int2* __restrict__ nextrun,
                         DenseCursor* __restrict__ arena, long long arena_stride,
                         const int64_t* __restrict__ rpC, long long cap, IT* __restrict__ ciC,
                         V* __restrict__ vC, long long max_dense_n, unsigned long long* work,
                         int* err, int64_t* __restrict__ rowend, int32_t* __restrict__ overflow,
                         unsigned* overflow_count, int64_t* __restrict__ unit_cnt,
        const long long vbid, const long long vnb) {
    constexpr bool HV = VOps<V>::has_val;
    constexpr int kNone = 0x7fffffff;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const int w = threadIdx.x >> 5;
    constexpr size_t vbytes = HV ? sizeof(V) * W : 0;
    unsigned char* base = smem_raw + (size_t)w * (vbytes + W / 8 + 32 * sizeof(DenseRun<V>));
    V* acc = reinterpret_cast<V*>(base);
    unsigned* bm = reinterpret_cast<unsigned*>(base + vbytes);
    DenseRun<V>* runs = reinterpret_cast<DenseRun<V>*>(base + vbytes + W / 8);
    DenseCursor* cursor = arena + ((long long)vbid * WARPS + w) * arena_stride;
    for (int s = lane; s < W; s += 32)
        if constexpr (HV) acc[s] = VOps<V>::init();
    for (int s = lane; s < W / 32; s += 32) bm[s] = 0u;
    __syncwarp();
    const unsigned long long* ub = cnt->unit_begin;
    const long long total_units = (long long)ub[kMaxDenseClasses];
    const int32_t* drow = rows + cnt->class_off[kClassDense0];
    while (true) {
        long long u = 0;
        if (lane == 0) u = (long long)atomicAdd(work, 1ull);
        u = __shfl_sync(kFull, u, 0);
        if (u >= total_units) break;
        int b = 0;
        while (b + 1 < kMaxDenseClasses && (long long)ub[b + 1] <= u) ++b;
        const int G = dense_class_segments(b, cnt->seg_log2);
        const long long local = u - (long long)ub[b];
        const long long rr = (long long)(cnt->class_off[kClassDense0 + b] -
                                         cnt->class_off[kClassDense0]) + local / G;
        const int seg = (int)(local % G);
        const long long r = drow[rr];
        const RowCtx<IT, V> cx = row_ctx<IT, V>(D, rb, nprod, r);
        const int P = cx.P;
        const long long n = cx.n;
        if (n > max_dense_n) continue;
        const int g0 = seg * (kSegGrid / G);
        const int cs = (int)seg_chunk(g0, P);
        const int ce = (int)seg_chunk(g0 + kSegGrid / G, P);
        if (cs >= ce) continue;
        const long long a0 = cx.a0, a1 = cx.a1;
        if (a1 - a0 > arena_stride) {
            if (lane == 0) atomicExch(err, (int)kDevArena);
            continue;
        }
        const IT* ciA = cx.ciA;
        const V* vA = cx.vA;
        const int64_t* rpB = cx.rpB;
        const IT* ciB = cx.ciB;
        const V* vB = cx.vB;
        const int32_t* ccnt = chunkcnt + cx.chunk_base + cx.i * P;
        const int32_t* stab = segtab + cx.seg_base;
        const int32_t* rlen = runlen + cx.run_base;
        const int2* nrun = nextrun + cx.run_base;
        // Slot mode (learned sizing, no symbolic pass): the row's predicted
        // slot [rpC[r], rpC[r+1]) is split over its segments in proportion
        // to their chunks; a segment that outgrows its share lists the row
        // for an exact re-run.  Otherwise the chunk counts of the symbolic
        // pass give the segment's exact place in C.
        const bool slot_mode = rowend != nullptr;
        long long out, out_end;
        if (slot_mode) {
            const long long span = rpC[r + 1] - rpC[r];
            out = rpC[r] + span * cs / P;
            out_end = rpC[r] + span * ce / P;
        } else {
            long long before = 0;
            for (int c = lane; c < cs; c += 32) before += ccnt[c];
            before = warp_sum(before);
            out = rpC[r] + before;
            long long seg_total = 0;
            for (int c = cs + lane; c < ce; c += 32) seg_total += ccnt[c];
            seg_total = warp_sum(seg_total);
            if (seg_total == 0) continue;
            out_end = out + seg_total;
            if (out_end > cap) {
                if (lane == 0) atomicExch(err, (int)kDevCapacity);
                continue;
            }
        }
        const long long out_begin = out;
        // cursors at the segment start; the smallest column over all cursors
        // names the next chunk with any product, so chunks without products
        // are jumped over
        int min_next = kNone;
        for (long long p = a0 + lane; p < a1; p += 32) {
            const long long k = (long long)ciA[p];
            const long long s1 = rpB[k + 1];
            const long long c0p = g0 == 0 ? rpB[k] : rpB[k] + stab[k * (kSegGrid + 1) + g0];
            DenseCursor nc;
            nc.pos = c0p;
            nc.col = c0p < s1 ? (int)ciB[c0p] : kNone;
            nc.rl = c0p < s1 ? rlen[c0p] : 0;
            cursor[p - a0] = nc;
            min_next = min(min_next, nc.col);
        }
        min_next = warp_min(min_next);
        __syncwarp();
        for (int c = max(cs, min_next / W); c < ce;) {
            const long long c0 = (long long)c * W;
            const long long c1 = min(c0 + (long long)W, n);
            int cnext = kNone;  // smallest column after this chunk
            // batches of 32 entries: cursors and A values are loaded together
            // (neither address depends on the other); a cursor's next run is
            // loaded before the batch is accumulated and used after it
            for (long long bb = a0; bb < a1; bb += 32) {
                const long long p = bb + lane;
                DenseCursor cur{0, kNone, 0};
                V a = VOps<V>::init();
                if (p < a1) {
                    cur = cursor[p - a0];
                    a = load_val(vA, p);
                }
                const bool here = p < a1 && (long long)cur.col < c1;
                int2 nx = make_int2(0, kNone);
                if (here) nx = nrun[cur.pos];
                if (__any_sync(kFull, here))
                    dense_batch<IT, V>(here, cur.pos, cur.rl, a, c0, ciB, vB, acc, bm, runs);
                if (here) {
                    DenseCursor nc;
                    nc.pos = cur.pos + cur.rl;
                    nc.col = nx.y;
                    nc.rl = nx.x;
                    cursor[p - a0] = nc;
                    cnext = min(cnext, nc.col);
                } else {
                    cnext = min(cnext, cur.col);
                }
            }
            // emit the chunk in column order: lane t owns bitmap word t (32
            // columns), a warp scan of the popcounts gives each lane its output
            // run; words and values are reset on the way
            constexpr int NWORDS = W / 32;
            for (int t0 = 0; t0 < NWORDS; t0 += 32) {
                const int wi0 = t0 + lane;
                unsigned word = wi0 < NWORDS ? bm[wi0] : 0u;
                const int pc = __popc(word);
                const int pincl = warp_incl_scan(pc);
                long long pos = out + (pincl - pc);
                while (word) {
                    const int bit = __ffs(word) - 1;
                    word &= word - 1;
                    const int s = wi0 * 32 + bit;
                    if (pos < out_end) {
                        ciC[pos] = (IT)(c0 + s);
                        if constexpr (HV) vC[pos] = acc[s];
                    }
                    if constexpr (HV) acc[s] = VOps<V>::init();
                    ++pos;
                }
                if (wi0 < NWORDS) bm[wi0] = 0u;
                out += __shfl_sync(kFull, pincl, 31);
            }
            __syncwarp();
            const int jump = warp_min(cnext) / W;
            c = max(c + 1, jump);
        }
        if (lane == 0) {
            if (!slot_mode) {
                if (out != out_end) atomicExch(err, (int)kDevCountMismatch);
            } else if (out > out_end) {
                if (atomicCAS((unsigned long long*)&rowend[r], 0ull, ~0ull) == 0ull)
                    overflow[atomicAdd(overflow_count, 1u)] = (int32_t)r;
            } else {
                unit_cnt[u] = out - out_begin;
            }
        }
    }
}

template <class IT, class V, int W, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 24 / WARPS)
    numeric_dense_kernel(const ProdDesc* __restrict__ D, const long long* __restrict__ rb,
                         int nprod, const int32_t* __restrict__ rows, const DevCounters* cnt,
                         const int32_t* __restrict__ chunkcnt, const int32_t* __restrict__ segtab,
                         const int32_t* __restrict__ runlen, const int2* __restrict__ nextrun,
                         DenseCursor* __restrict__ arena, long long arena_stride,
                         const int64_t* __restrict__ rpC, long long cap, IT* __restrict__ ciC,
                         V* __restrict__ vC, long long max_dense_n, unsigned long long* work,
                         int* err, int64_t* __restrict__ rowend, int32_t* __restrict__ overflow,
                         unsigned* overflow_count, int64_t* __restrict__ unit_cnt) {
    numeric_dense_kernel_body<IT, V, W, WARPS>(D, rb, nprod, rows, cnt, chunkcnt, segtab, runlen,
        nextrun, arena, arena_stride, rpC, cap, ciC, vC, max_dense_n, work, err, rowend,
        overflow, overflow_count, unit_cnt, (long long)blockIdx.x, (long long)gridDim.x);
}

// Learned sizing: close the gaps a slot-mode dense row leaves between its
// segments (each segment moves left to follow the previous one) and set
// rowend.  One warp per dense row; rows listed for a re-run are skipped.
template <class IT, class V>
__global__ void dense_slot_pack_kernel(const ProdDesc* __restrict__ D,
                                       const long long* __restrict__ rb, int nprod,
                                       const int32_t* __restrict__ rows,
                                       const DevCounters* __restrict__ cnt,
                                       const int64_t* __restrict__ rpC,
                                       const int64_t* __restrict__ unit_cnt,
                                       int64_t* __restrict__ rowend, IT* __restrict__ ciC,
                                       V* __restrict__ vC) {
    constexpr bool HV = VOps<V>::has_val;
    const int lane = lane_id();
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long d0 = (long long)cnt->class_off[kClassDense0];
    const long long nd = (long long)cnt->class_off[kNumClasses] - d0;
    const unsigned long long* ub = cnt->unit_begin;
    for (long long rr = warp; rr < nd; rr += nwarps) {
        int b = 0;
        while (b + 1 < kMaxDenseClasses &&
               (long long)cnt->class_off[kClassDense0 + b + 1] - d0 <= rr)
            ++b;
        const int G = dense_class_segments(b, cnt->seg_log2);
        const long long local = rr - ((long long)cnt->class_off[kClassDense0 + b] - d0);
        const long long u0 = (long long)ub[b] + local * G;
        const long long r = rows[d0 + rr];
        if (rowend[r] != 0) continue;  // listed for a re-run
        const int P = D[nprod > 1 ? find_prod(rb, nprod, r) : 0].P;
        const long long start = rpC[r];
        const long long span = rpC[r + 1] - start;
        long long dst = start;
        for (int g = 0; g < G; ++g) {
            const int g0 = g * (kSegGrid / G);
            const long long src = start + span * seg_chunk(g0, P) / P;
            const long long len = unit_cnt[u0 + g];
            if (src != dst) {
                // dst < src: a forward copy in steps of 128 entries (all of a
                // step read before any is written) never overwrites an entry
                // before it is read; four loads per lane are in flight
                for (long long q = 0; q < len; q += 128) {
                    IT cv[4];
                    V vv[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const long long x = q + 32 * t + lane;
                        cv[t] = IT{};
                        vv[t] = V{};
                        if (x < len) {
                            cv[t] = ciC[src + x];
                            if constexpr (HV) vv[t] = vC[src + x];
                        }
                    }
                    __syncwarp();
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const long long x = q + 32 * t + lane;
                        if (x < len) {
                            ciC[dst + x] = cv[t];
                            if constexpr (HV) vC[dst + x] = vv[t];
                        }
                    }
                    __syncwarp();
                }
            }
            dst += len;
        }
        if (lane == 0) rowend[r] = dst;
    }
}

// ------------------------------------------------------------ k-slices
// bounds[s*m + i] = first position in A(i,:) with column >= floor(s*l/c).
template <class IT>
__global__ void kslice_bounds_kernel(long long m, long long l, int c,
                                     const int64_t* __restrict__ rp, const IT* __restrict__ ci,
                                     int64_t* __restrict__ bounds) {
    const long long total = m * (long long)(c + 1);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long s = t / m, i = t - s * m;
        const long long key = (s * l) / c;
        long long lo = rp[i], hi = rp[i + 1];
        while (lo < hi) {
            long long mid = (lo + hi) >> 1;
            if ((long long)ci[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        bounds[t] = lo;
    }
}

}  // namespace sg
