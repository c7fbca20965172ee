// Non-template kernels: row binning, int64 exclusive scan, empty rows; and
// their host launchers.
#include "plan.h"

namespace sg {

// Class offsets (exclusive scan of the counts) and the dense work-unit
// prefix, one thread.
__global__ void class_offsets_kernel(DevCounters* cnt, int seg_log2) {
    cnt->seg_log2 = seg_log2;
    unsigned long long s = 0;
    for (int c = 0; c < kNumClasses; ++c) {
        cnt->class_cursor[c] = s;
        cnt->class_off[c] = s;
        s += cnt->class_count[c];
    }
    cnt->class_off[kNumClasses] = s;
    unsigned long long u = 0;
    for (int t = 0; t < kMaxDenseClasses; ++t) {
        cnt->unit_begin[t] = u;
        u += cnt->class_count[kClassDense0 + t] *
             (unsigned long long)dense_class_segments(t, seg_log2);
    }
    cnt->unit_begin[kMaxDenseClasses] = u;
}

// Scatter global row ids into their class segment (order inside a class is
// free; rows are independent).  Each block counts its rows per class in
// shared memory, reserves one range per class with a single global atomic,
// then places its rows.  Lanes of a warp with the same class are grouped, so
// one atomic per class and warp does the counting (rows of one product often
// share a class).
__global__ void bin_rows_kernel(long long R, const unsigned char* __restrict__ cls,
                                int32_t* __restrict__ rows, DevCounters* cnt) {
    __shared__ unsigned long long loc[kNumClasses];
    __shared__ unsigned long long base[kNumClasses];
    const long long per_block = (R + gridDim.x - 1) / gridDim.x;
    const long long r0 = (long long)blockIdx.x * per_block;
    const long long r1 = min(R, r0 + per_block);
    for (int t = threadIdx.x; t < kNumClasses; t += blockDim.x) loc[t] = 0;
    __syncthreads();
    bin_block_rows(cls, rows, r0, r1, loc, nullptr);
    __syncthreads();
    for (int t = threadIdx.x; t < kNumClasses; t += blockDim.x) {
        base[t] = loc[t] ? atomicAdd(&cnt->class_cursor[t], loc[t]) : 0;
        loc[t] = 0;
    }
    __syncthreads();
    bin_block_rows(cls, rows, r0, r1, loc, base);
}

// ------------------------------------------------------------------ scan
// In-place exclusive scan of int64 x[0..N).  Tiles of 4096 (256 x 16).

__global__ void scan_reduce_kernel(const int64_t* __restrict__ x, long long N,
                                   int64_t* __restrict__ part) {
    __shared__ long long ws[kScanThreads / 32];
    long long base = (long long)blockIdx.x * kScanTile;
    long long s = 0;
    for (int t = 0; t < kScanItems; ++t) {
        long long idx = base + (long long)t * kScanThreads + threadIdx.x;
        if (idx < N) s += x[idx];
    }
    s = warp_sum(s);
    if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long v = threadIdx.x < kScanThreads / 32 ? ws[threadIdx.x] : 0;
        v = warp_sum(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

// Exclusive scan of the tile sums with one block of 1024 threads (carry loop).
__global__ void scan_partials_kernel(int64_t* part, long long nparts) {
    __shared__ long long ws[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b = 0; b < nparts; b += blockDim.x) {
        long long idx = b + threadIdx.x;
        long long v = idx < nparts ? part[idx] : 0;
        long long inc = warp_incl_scan(v);
        if (lane_id() == 31) ws[threadIdx.x >> 5] = inc;
        __syncthreads();
        if (threadIdx.x < 32) {
            long long w = ws[threadIdx.x];
            long long wi = warp_incl_scan(w);
            ws[threadIdx.x] = wi - w;
        }
        __syncthreads();
        long long excl = carry + ws[threadIdx.x >> 5] + inc - v;
        if (idx < nparts) part[idx] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
}

__global__ void scan_apply_kernel(int64_t* __restrict__ x, long long N,
                                  const int64_t* __restrict__ part) {
    __shared__ long long ws[kScanThreads / 32];
    __shared__ long long carry;
    long long base = (long long)blockIdx.x * kScanTile;
    if (threadIdx.x == 0) carry = part[blockIdx.x];
    __syncthreads();
    for (int t = 0; t < kScanItems; ++t) {
        long long idx = base + (long long)t * kScanThreads + threadIdx.x;
        long long v = idx < N ? x[idx] : 0;
        long long inc = warp_incl_scan(v);
        if (lane_id() == 31) ws[threadIdx.x >> 5] = inc;
        __syncthreads();
        if (threadIdx.x < 32) {
            long long w = threadIdx.x < kScanThreads / 32 ? ws[threadIdx.x] : 0;
            long long wi = warp_incl_scan(w);
            if (threadIdx.x < kScanThreads / 32) ws[threadIdx.x] = wi - w;
        }
        __syncthreads();
        long long excl = carry + ws[threadIdx.x >> 5] + inc - v;
        if (idx < N) x[idx] = excl;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = excl + v;
        __syncthreads();
    }
}

// Empty rows: count 0.
__global__ void zero_rows_kernel(const int32_t* __restrict__ rows, const DevCounters* cnt,
                                 int64_t* __restrict__ rowcnt) {
    const long long nrows = (long long)cnt->class_count[kClassEmpty];
    const int32_t* erow = rows + cnt->class_off[kClassEmpty];
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
         r += (long long)gridDim.x * blockDim.x)
        rowcnt[erow[r]] = 0;
}

// Relative row pointers of every product: out[out_base_p + i] = g[rb_p + i] - g[rb_p].
__global__ void product_rowptr_kernel(long long R, const long long* __restrict__ rb, int nprod,
                                      const int64_t* __restrict__ g, int64_t* __restrict__ out) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < R + nprod;
         t += (long long)gridDim.x * blockDim.x) {
        // entry t belongs to product p with rb[p] + p <= t < rb[p+1] + p + 1
        int lo = 0, hi = nprod - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (rb[mid] + mid <= t) lo = mid;
            else hi = mid - 1;
        }
        const long long i = t - rb[lo] - lo;
        out[t] = g[rb[lo] + i] - g[rb[lo]];
    }
}

cudaError_t launch_class_offsets(Plan& P) {
    count_launches(1);
    class_offsets_kernel<<<1, 1, 0, P.stream>>>(P.cnt, P.seg_log2);
    return cudaGetLastError();
}

cudaError_t launch_binning(Plan& P) {
    const long long R = P.R;
    count_launches(1);
    class_offsets_kernel<<<1, 1, 0, P.stream>>>(P.cnt, P.seg_log2);
    if (R > 0) {
        int blocks = (int)std::max<long long>(1, std::min<long long>((R + 1023) / 1024, (long long)P.sm_count * 4));
        count_launches(1);
        bin_rows_kernel<<<blocks, 256, 0, P.stream>>>(R, P.cls, P.rows, P.cnt);
    }
    return cudaGetLastError();
}

size_t scan_temp_bytes(long long N) {
    long long parts = (N + kScanTile - 1) / kScanTile;
    return (size_t)std::max<long long>(parts, 1) * sizeof(int64_t);
}

cudaError_t launch_exclusive_scan(int64_t* x, long long N, int64_t* temp, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    long long parts = (N + kScanTile - 1) / kScanTile;
    count_launches(1);
    scan_reduce_kernel<<<(unsigned)parts, kScanThreads, 0, s>>>(x, N, temp);
    count_launches(1);
    scan_partials_kernel<<<1, 1024, 0, s>>>(temp, parts);
    count_launches(1);
    scan_apply_kernel<<<(unsigned)parts, kScanThreads, 0, s>>>(x, N, temp);
    return cudaGetLastError();
}

cudaError_t launch_zero_rows(const Plan& P, int64_t* rowcnt) {
    int blocks = P.sm_count * 4;
    count_launches(1);
    zero_rows_kernel<<<blocks, 256, 0, P.stream>>>(P.rows, P.cnt, rowcnt);
    return cudaGetLastError();
}

cudaError_t launch_product_rowptr(const Plan& P, const int64_t* g, int64_t* out) {
    const long long total = P.R + P.nprod;
    int blocks = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, (long long)P.sm_count * 8));
    count_launches(1);
    product_rowptr_kernel<<<blocks, 256, 0, P.stream>>>(P.R, P.rb, P.nprod, g, out);
    return cudaGetLastError();
}

}  // namespace sg
