// Distance-2 maximal independent set and the aggregation built on it: the
// restriction operator R of the paper's AMG experiments (Sec. 5.4, Alg. 3).
//
// Every round (the loop of Alg. 3):
//   x      = key(seed, t, v) for candidates, +inf (INT64_MAX) otherwise;
//   m1, m2 = (min, select2nd) products A.x and A.m1 (the smallest candidate
//            key within distance 1 and 2);
//   new    = candidates whose key is <= min(m1, m2) (the smallest within
//            distance 2; keys are unique, so no two new members are close);
//   a1, a2 = (min, select2nd) products of the new members' indicator, which
//            reach every vertex within distance 2 of a new member;
//   candidates lose the new members and every vertex a1 or a2 reaches.
// key(seed, t, v) = ((splitmix64(seed ^ (t * 0xD1B54A32D192ED03) + v) >> 33)
// << 31) | v, SplitMix64 as published by Steele, Lea and Flood (the vertex id
// in the low 31 bits makes keys unique).
// Aggregates: members numbered in increasing vertex order own themselves and
// their neighbours; every other vertex joins the smallest-numbered aggregate
// among its neighbours.  R(v, agg(v)) = 1.
//
// The (min, select2nd) product with a dense vector uses a group of 8 lanes per
// row of A (rows of a mesh matrix are short).
#include <cstdio>

#include "plan.h"

namespace sg {

constexpr long long kInf64 = 0x7fffffffffffffffLL;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void mis2_keys_kernel(long long n, const unsigned char* __restrict__ cand,
                                 unsigned long long seed, unsigned long long t,
                                 long long* __restrict__ x) {
    const unsigned long long base = seed ^ (t * 0xD1B54A32D192ED03ull);
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const unsigned long long h = splitmix64(base + (unsigned long long)v);
        x[v] = cand[v] ? (long long)(((h >> 33) << 31) | (unsigned long long)v) : kInf64;
    }
}

// y(i) = min over k in A(i,:) of x(k); 8 lanes per row.
template <class IT>
__global__ void min_adjacent_kernel(long long n, const int64_t* __restrict__ rp,
                                    const int64_t* __restrict__ re, const IT* __restrict__ col,
                                    const long long* __restrict__ x, long long* __restrict__ y) {
    const int sub = threadIdx.x & 7;
    const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const long long ng = ((long long)gridDim.x * blockDim.x) >> 3;
    const long long rounds = (n + ng - 1) / ng;
    for (long long it = 0; it < rounds; ++it) {     // uniform trip count for the shuffles
        const long long i = g + it * ng;
        long long mn = kInf64;
        if (i < n) {
            const long long a = rp[i], b = re ? re[i] : rp[i + 1];
            for (long long q = a + sub; q < b; q += 8) {
                const long long v = x[(long long)col[q]];
                mn = v < mn ? v : mn;
            }
        }
#pragma unroll
        for (int d = 4; d; d >>= 1) {
            const long long o = __shfl_xor_sync(kFull, mn, d);
            mn = o < mn ? o : mn;
        }
        if (i < n && sub == 0) y[i] = mn;
    }
}

__global__ void mis2_select_kernel(long long n, const long long* __restrict__ x,
                                   const long long* __restrict__ m1, const long long* __restrict__ m2,
                                   unsigned char* __restrict__ cand, unsigned char* __restrict__ member,
                                   long long* __restrict__ ind) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long mm = m1[v] < m2[v] ? m1[v] : m2[v];
        const bool add = cand[v] && x[v] <= mm;
        if (add) {
            member[v] = 1;
            cand[v] = 0;
        }
        ind[v] = add ? 0 : kInf64;
    }
}

__global__ void mis2_prune_kernel(long long n, const long long* __restrict__ a1,
                                  const long long* __restrict__ a2, unsigned char* __restrict__ cand,
                                  unsigned long long* __restrict__ left) {
    unsigned long long mine = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        if (cand[v] && (a1[v] < kInf64 || a2[v] < kInf64)) cand[v] = 0;
        mine += cand[v];
    }
    mine = warp_sum(mine);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(left, mine);
}

__global__ void flags_to_i64_kernel(long long n, const unsigned char* __restrict__ f,
                                    int64_t* __restrict__ out) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        out[v] = f[v];
}

// agg = member id (exclusive scan of the flags) for members, +inf otherwise
__global__ void member_ids_kernel(long long n, const unsigned char* __restrict__ member,
                                  const int64_t* __restrict__ scan, long long* __restrict__ agg) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        agg[v] = member[v] ? (long long)scan[v] : kInf64;
}

// keep assigned ids; take the neighbours' minimum elsewhere
__global__ void fill_from_kernel(long long n, long long* __restrict__ agg,
                                 const long long* __restrict__ near) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        if (agg[v] == kInf64) agg[v] = near[v];
}

template <class IT>
__global__ void restriction_kernel(long long n, const long long* __restrict__ agg,
                                   int64_t* __restrict__ rowptr, IT* __restrict__ col,
                                   double* __restrict__ val, int* __restrict__ bad) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v <= n;
         v += (long long)gridDim.x * blockDim.x) {
        rowptr[v] = v;
        if (v < n) {
            if (agg[v] == kInf64) atomicExch(bad, 1);
            col[v] = (IT)agg[v];
            val[v] = 1.0;
        }
    }
}

}  // namespace sg

namespace {

spgemm_status mfail2(spgemm_status st, const char* msg) {
    sg::set_last_error(msg);
    return st;
}

size_t al(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" {

size_t spgemm_mis2_workspace_size(int64_t n) {
    if (n < 0) n = 0;
    const size_t v8 = al((size_t)std::max<int64_t>(n, 1) * 8);
    return 2 * al((size_t)std::max<int64_t>(n, 1)) + 5 * v8 + al(8) + al(sizeof(int)) +
           al(sg::scan_temp_bytes(n + 1)) + al((size_t)(n + 1) * 8);
}

spgemm_status spgemm_mis2_restriction(const spgemm_csr* A, uint64_t seed, void* stream, void* ws,
                                      size_t ws_bytes, int64_t* rowptrR, void* colR,
                                      double* valR, int64_t* naggs_host, int32_t* rounds_host) {
    sg::set_last_error("");
    if (!A || !A->rowptr || A->nrows < 0 || A->nrows != A->ncols || (A->nnz > 0 && !A->col))
        return mfail2(SPGEMM_ERR_INVALID_ARG, "mis2: A must be a square CSR");
    if (A->nrows > 0x7fffffffLL)
        return mfail2(SPGEMM_ERR_NOT_SUPPORTED, "mis2: at most 2^31-1 vertices");
    if (!rowptrR || !colR || !valR || !naggs_host || !rounds_host)
        return mfail2(SPGEMM_ERR_INVALID_ARG, "mis2: NULL output");
    const long long n = A->nrows;
    if (!ws || ws_bytes < spgemm_mis2_workspace_size(n))
        return mfail2(SPGEMM_ERR_INVALID_ARG, "mis2: workspace missing or too small");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* w = (unsigned char*)ws;
    const size_t f1 = al((size_t)std::max<long long>(n, 1));
    const size_t v8 = al((size_t)std::max<long long>(n, 1) * 8);
    unsigned char* cand = w;
    unsigned char* member = w + f1;
    long long* x = (long long*)(w + 2 * f1);
    long long* m1 = (long long*)(w + 2 * f1 + v8);
    long long* m2 = (long long*)(w + 2 * f1 + 2 * v8);
    long long* a1 = (long long*)(w + 2 * f1 + 3 * v8);
    long long* a2 = (long long*)(w + 2 * f1 + 4 * v8);
    unsigned long long* left = (unsigned long long*)(w + 2 * f1 + 5 * v8);
    int* bad = (int*)(w + 2 * f1 + 5 * v8 + al(8));
    int64_t* temp = (int64_t*)(w + 2 * f1 + 5 * v8 + al(8) + al(sizeof(int)));
    int64_t* scan = (int64_t*)((unsigned char*)temp + al(sg::scan_temp_bytes(n + 1)));
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)sms * 8));
    const unsigned gr = (unsigned)std::max<long long>(1, std::min<long long>((n * 8 + 255) / 256, (long long)sms * 16));
    const bool i32 = A->index_type == SPGEMM_INDEX_I32;
    auto minadj = [&](const long long* xin, long long* yout) {
        sg::count_launches(1);
        if (i32)
            sg::min_adjacent_kernel<int32_t><<<gr, 256, 0, s>>>(n, A->rowptr, A->rowend,
                                                                (const int32_t*)A->col, xin, yout);
        else
            sg::min_adjacent_kernel<int64_t><<<gr, 256, 0, s>>>(n, A->rowptr, A->rowend,
                                                                (const int64_t*)A->col, xin, yout);
    };
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = cudaMemsetAsync(cand, 1, (size_t)n, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(member, 0, (size_t)n, s);
    }
    int rounds = 0;
    unsigned long long remaining = (unsigned long long)n;
    while (e == cudaSuccess && remaining > 0) {
        if (rounds >= 1 << 20) return mfail2(SPGEMM_ERR_INTERNAL, "mis2: no progress");
        e = cudaMemsetAsync(left, 0, 8, s);
        if (e != cudaSuccess) break;
        sg::count_launches(1);
        sg::mis2_keys_kernel<<<g, 256, 0, s>>>(n, cand, seed, (unsigned long long)rounds, x);
        minadj(x, m1);
        minadj(m1, m2);
        sg::count_launches(1);
        sg::mis2_select_kernel<<<g, 256, 0, s>>>(n, x, m1, m2, cand, member, x);
        minadj(x, a1);
        minadj(a1, a2);
        sg::count_launches(1);
        sg::mis2_prune_kernel<<<g, 256, 0, s>>>(n, a1, a2, cand, left);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&remaining, left, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        ++rounds;
    }
    // aggregates
    long long naggs = 0;
    if (e == cudaSuccess && n > 0) {
        sg::count_launches(1);
        sg::flags_to_i64_kernel<<<g, 256, 0, s>>>(n, member, scan);
        e = cudaMemsetAsync(scan + n, 0, 8, s);
        if (e == cudaSuccess) e = sg::launch_exclusive_scan(scan, n + 1, temp, s);
        if (e == cudaSuccess) {
            sg::count_launches(1);
            sg::member_ids_kernel<<<g, 256, 0, s>>>(n, member, scan, x);
            minadj(x, m1);
            sg::count_launches(1);
            sg::fill_from_kernel<<<g, 256, 0, s>>>(n, x, m1);
            minadj(x, m1);
            sg::count_launches(1);
            sg::fill_from_kernel<<<g, 256, 0, s>>>(n, x, m1);
            e = cudaMemsetAsync(bad, 0, sizeof(int), s);
        }
        if (e == cudaSuccess) {
            sg::count_launches(1);
            if (i32)
                sg::restriction_kernel<int32_t><<<g, 256, 0, s>>>(n, x, rowptrR, (int32_t*)colR, valR, bad);
            else
                sg::restriction_kernel<int64_t><<<g, 256, 0, s>>>(n, x, rowptrR, (int64_t*)colR, valR, bad);
            e = cudaGetLastError();
        }
        int hbad = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&naggs, scan + n, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && hbad)
            return mfail2(SPGEMM_ERR_INTERNAL, "mis2: a vertex was left without an aggregate");
    } else if (e == cudaSuccess) {
        e = cudaMemsetAsync(rowptrR, 0, 8, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return mfail2(SPGEMM_ERR_CUDA, cudaGetErrorString(e));
    *naggs_host = naggs;
    *rounds_host = rounds;
    return SPGEMM_OK;
}

}  // extern "C"
