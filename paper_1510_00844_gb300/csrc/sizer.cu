// Row-size predictor for learned sizing of C (not in the paper).
//
// A 3-layer MLP, x (kSizerF features) -> relu(W1 x + b1) (32) ->
// relu(W2 h1 + b2) (32) -> y = w3 . h2 + b3, float32, trained with
// mean-squared error by hand-written kernels: a block takes 128 samples, one
// thread per sample runs forward and backward and stages its activations and
// deltas in shared memory; the block then forms the parameter gradients as
// sums over its samples (one thread per parameter) and adds them to the
// global gradient.  Adam updates the parameters.  Parameter layout: W1
// (32 x F, row-major), b1, W2 (32 x 32, row-major), b2, w3, b3.
#include <cstdio>
#include <cstring>

#include "plan.h"

namespace sg {

constexpr int kSizerH = 32;
constexpr int kSizerTile = 128;

__host__ __device__ constexpr int sizer_params(int F) {
    return kSizerH * F + kSizerH + kSizerH * kSizerH + kSizerH + kSizerH + 1;
}

// y = MLP(x) for N samples (one thread per sample).
__global__ void sizer_forward_kernel(const float* __restrict__ X, long long N, int F,
                                     const float* __restrict__ prm, float* __restrict__ y) {
    extern __shared__ float sp[];
    const int P = sizer_params(F);
    for (int q = threadIdx.x; q < P; q += blockDim.x) sp[q] = prm[q];
    __syncthreads();
    const float* W1 = sp;
    const float* b1 = W1 + kSizerH * F;
    const float* W2 = b1 + kSizerH;
    const float* b2 = W2 + kSizerH * kSizerH;
    const float* w3 = b2 + kSizerH;
    const float b3 = w3[kSizerH];
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        float h1[kSizerH];
        for (int j = 0; j < kSizerH; ++j) {
            float z = b1[j];
            for (int f = 0; f < F; ++f) z = __fadd_rn(z, __fmul_rn(W1[j * F + f], X[s * F + f]));
            h1[j] = z > 0.f ? z : 0.f;
        }
        float out = b3;
        for (int j = 0; j < kSizerH; ++j) {
            float z = b2[j];
            for (int k = 0; k < kSizerH; ++k) z = __fadd_rn(z, __fmul_rn(W2[j * kSizerH + k], h1[k]));
            const float h2 = z > 0.f ? z : 0.f;
            out = __fadd_rn(out, __fmul_rn(w3[j], h2));
        }
        y[s] = out;
    }
}

// Gradient of 0.5 * sum_s (y_s - t_s)^2 / norm over samples [s0, s0 + count)
// (rows taken through `order` when given), added to grad; the summed
// squared error / (2 norm) is added to *loss.
__global__ void sizer_grad_kernel(const float* __restrict__ X, const float* __restrict__ T,
                                  const long long* __restrict__ order, long long s0,
                                  long long count, int F, float norm,
                                  const float* __restrict__ prm, float* __restrict__ grad,
                                  float* __restrict__ loss) {
    extern __shared__ float sm[];
    const int P = sizer_params(F);
    float* sp = sm;                                  // parameters
    float* sx = sp + P;                              // x      [tile][F]
    float* sh1 = sx + kSizerTile * F;                // h1     [tile][32]
    float* sh2 = sh1 + kSizerTile * kSizerH;         // h2     [tile][32]
    float* sd1 = sh2 + kSizerTile * kSizerH;         // dz1    [tile][32]
    float* sd2 = sd1 + kSizerTile * kSizerH;         // dz2    [tile][32]
    float* sdy = sd2 + kSizerTile * kSizerH;         // dy     [tile]
    __shared__ float bl;
    for (int q = threadIdx.x; q < P; q += blockDim.x) sp[q] = prm[q];
    if (threadIdx.x == 0) bl = 0.f;
    __syncthreads();
    const float* W1 = sp;
    const float* b1 = W1 + kSizerH * F;
    const float* W2 = b1 + kSizerH;
    const float* b2 = W2 + kSizerH * kSizerH;
    const float* w3 = b2 + kSizerH;
    const float b3 = w3[kSizerH];
    for (long long t0 = (long long)blockIdx.x * kSizerTile; t0 < count;
         t0 += (long long)gridDim.x * kSizerTile) {
        const int i = threadIdx.x;
        const long long t = t0 + i;
        const bool valid = i < kSizerTile && t < count;
        if (i < kSizerTile) {
            float z1[kSizerH], z2[kSizerH];
            const long long s = valid ? (order ? order[s0 + t] : s0 + t) : 0;
            for (int f = 0; f < F; ++f) sx[i * F + f] = valid ? X[s * F + f] : 0.f;
            for (int j = 0; j < kSizerH; ++j) {
                float z = b1[j];
                for (int f = 0; f < F; ++f) z = __fadd_rn(z, __fmul_rn(W1[j * F + f], sx[i * F + f]));
                z1[j] = z;
                sh1[i * kSizerH + j] = z > 0.f ? z : 0.f;
            }
            float y = b3;
            for (int j = 0; j < kSizerH; ++j) {
                float z = b2[j];
                for (int k = 0; k < kSizerH; ++k)
                    z = __fadd_rn(z, __fmul_rn(W2[j * kSizerH + k], sh1[i * kSizerH + k]));
                z2[j] = z;
                const float h2 = z > 0.f ? z : 0.f;
                sh2[i * kSizerH + j] = h2;
                y = __fadd_rn(y, __fmul_rn(w3[j], h2));
            }
            const float r = valid ? y - T[s] : 0.f;
            const float dy = r / norm;
            sdy[i] = dy;
            if (valid) atomicAdd(&bl, 0.5f * r * r / norm);
            for (int j = 0; j < kSizerH; ++j) sd2[i * kSizerH + j] = z2[j] > 0.f ? dy * w3[j] : 0.f;
            for (int k = 0; k < kSizerH; ++k) {
                float a = 0.f;
                for (int j = 0; j < kSizerH; ++j) a += sd2[i * kSizerH + j] * W2[j * kSizerH + k];
                sd1[i * kSizerH + k] = z1[k] > 0.f ? a : 0.f;
            }
        }
        __syncthreads();
        // parameter gradients: sums over the tile's samples
        for (int q = threadIdx.x; q < P; q += blockDim.x) {
            float g = 0.f;
            if (q < kSizerH * F) {
                const int j = q / F, f = q % F;
                for (int s = 0; s < kSizerTile; ++s) g += sd1[s * kSizerH + j] * sx[s * F + f];
            } else if (q < kSizerH * F + kSizerH) {
                const int j = q - kSizerH * F;
                for (int s = 0; s < kSizerTile; ++s) g += sd1[s * kSizerH + j];
            } else if (q < kSizerH * F + kSizerH + kSizerH * kSizerH) {
                const int r2 = q - kSizerH * F - kSizerH;
                const int j = r2 / kSizerH, k = r2 % kSizerH;
                for (int s = 0; s < kSizerTile; ++s) g += sd2[s * kSizerH + j] * sh1[s * kSizerH + k];
            } else if (q < kSizerH * F + 2 * kSizerH + kSizerH * kSizerH) {
                const int j = q - (kSizerH * F + kSizerH + kSizerH * kSizerH);
                for (int s = 0; s < kSizerTile; ++s) g += sd2[s * kSizerH + j];
            } else if (q < P - 1) {
                const int j = q - (kSizerH * F + 2 * kSizerH + kSizerH * kSizerH);
                for (int s = 0; s < kSizerTile; ++s) g += sdy[s] * sh2[s * kSizerH + j];
            } else {
                for (int s = 0; s < kSizerTile; ++s) g += sdy[s];
            }
            atomicAdd(&grad[q], g);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, bl);
}

// Adam step t (1-based) with bias correction.
__global__ void sizer_adam_kernel(int P, float* __restrict__ prm, const float* __restrict__ g,
                                  float* __restrict__ m, float* __restrict__ v, float lr,
                                  float b1, float b2, float eps, int t) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    const float gq = g[q];
    m[q] = b1 * m[q] + (1.f - b1) * gq;
    v[q] = b2 * v[q] + (1.f - b2) * gq * gq;
    const float mh = m[q] / (1.f - powf(b1, (float)t));
    const float vh = v[q] / (1.f - powf(b2, (float)t));
    prm[q] -= lr * mh / (sqrtf(vh) + eps);
}

size_t grad_smem(int F) {
    return sizeof(float) * ((size_t)sizer_params(F) + (size_t)kSizerTile * F +
                            4 * (size_t)kSizerTile * kSizerH + kSizerTile);
}

cudaError_t launch_sizer_grad(const float* X, const float* T, const long long* order,
                              long long s0, long long count, int F, float norm, const float* prm,
                              float* grad, float* loss, cudaStream_t s, int sms) {
    const size_t smem = grad_smem(F);
    cudaError_t e = cudaFuncSetAttribute(sizer_grad_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (count + kSizerTile - 1) / kSizerTile;
    const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>(tiles, (long long)sms * 2));
    count_launches(1);
    sizer_grad_kernel<<<g, 256, smem, s>>>(X, T, order, s0, count, F, norm, prm, grad, loss);
    return cudaGetLastError();
}

// Training target of row i: log2(1 + nnz(C(i,:))) from the row pointers of
// the exact symbolic phase.
__global__ void sizer_targets_kernel(const int64_t* __restrict__ rp, long long m,
                                     float* __restrict__ T) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x)
        T[i] = log2f(1.f + (float)(rp[i + 1] - rp[i]));
}

// Byte record of a trained predictor (little-endian): magic, format version,
// F, hidden width, feature-set id, target id, parameter count, the float32
// parameters, then a 64-bit FNV-1a hash of everything before it.
constexpr char kSizerMagic[8] = {'S', 'G', 'S', 'I', 'Z', 'E', 'R', 0};
constexpr uint32_t kSizerVersion = 1;
constexpr uint32_t kSizerFeatureSet = 1;  // the six log2(1 + .) row features
constexpr uint32_t kSizerTarget = 1;      // log2(1 + nnz(C(i,:)))
constexpr size_t kSizerHeader = 8 + 6 * sizeof(uint32_t);

inline size_t sizer_record_bytes(int F) {
    return kSizerHeader + sizeof(float) * (size_t)sizer_params(F) + sizeof(uint64_t);
}

inline uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 14695981039346656037ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace sg

extern "C" {

int32_t spgemm_sizer_param_count(int32_t features) { return sg::sizer_params(features); }

spgemm_status spgemm_sizer_forward(const float* X, int64_t N, int32_t F, const float* params,
                                   float* y, void* stream) {
    if (N < 0 || F < 1 || F > 64 || (N > 0 && (!X || !params || !y))) {
        sg::set_last_error("sizer_forward: bad arguments");
        return SPGEMM_ERR_INVALID_ARG;
    }
    if (N == 0) return SPGEMM_OK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>((N + 127) / 128, (long long)sms * 8));
    sg::count_launches(1);
    sg::sizer_forward_kernel<<<g, 128, sizeof(float) * sg::sizer_params(F), (cudaStream_t)stream>>>(
        X, N, F, params, y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        sg::set_last_error(cudaGetErrorString(e));
        return SPGEMM_ERR_CUDA;
    }
    return SPGEMM_OK;
}

spgemm_status spgemm_sizer_grad(const float* X, const float* T, int64_t N, int32_t F,
                                const float* params, float* grad, float* loss, void* stream) {
    if (N <= 0 || F < 1 || F > 64 || !X || !T || !params || !grad || !loss) {
        sg::set_last_error("sizer_grad: bad arguments");
        return SPGEMM_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * sg::sizer_params(F), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e == cudaSuccess)
        e = sg::launch_sizer_grad(X, T, nullptr, 0, N, F, (float)N, params, grad, loss, s, sms);
    if (e != cudaSuccess) {
        sg::set_last_error(cudaGetErrorString(e));
        return SPGEMM_ERR_CUDA;
    }
    return SPGEMM_OK;
}

spgemm_status spgemm_sizer_train(const float* X, const float* T, const int64_t* order, int64_t N,
                                 int32_t F, float* params, float* adam_m, float* adam_v,
                                 float* grad, int32_t steps, int32_t batch, float lr,
                                 float* loss_trace, void* stream) {
    if (N <= 0 || F < 1 || F > 64 || steps < 0 || batch < 1 || !X || !T || !order || !params ||
        !adam_m || !adam_v || !grad || !loss_trace) {
        sg::set_last_error("sizer_train: bad arguments");
        return SPGEMM_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = (cudaStream_t)stream;
    const int P = sg::sizer_params(F);
    cudaError_t e = cudaMemsetAsync(loss_trace, 0, sizeof(float) * (size_t)steps, s);
    const long long B = std::min<long long>(batch, N);
    for (int t = 0; t < steps && e == cudaSuccess; ++t) {
        const long long s0 = ((long long)t * B) % std::max<long long>(1, N - B + 1);
        e = cudaMemsetAsync(grad, 0, sizeof(float) * P, s);
        if (e == cudaSuccess)
            e = sg::launch_sizer_grad(X, T, (const long long*)order, s0, B, F, (float)B, params,
                                      grad, loss_trace + t, s, sms);
        if (e == cudaSuccess) {
            sg::count_launches(1);
            sg::sizer_adam_kernel<<<(P + 255) / 256, 256, 0, s>>>(P, params, grad, adam_m, adam_v,
                                                                  lr, 0.9f, 0.999f, 1e-8f, t + 1);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        sg::set_last_error(cudaGetErrorString(e));
        return SPGEMM_ERR_CUDA;
    }
    return SPGEMM_OK;
}

spgemm_status spgemm_sizer_targets(const int64_t* rowptrC, int64_t m, float* T, void* stream) {
    if (m < 0 || (m > 0 && (!rowptrC || !T))) {
        sg::set_last_error("sizer_targets: bad arguments");
        return SPGEMM_ERR_INVALID_ARG;
    }
    if (m == 0) return SPGEMM_OK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>((m + 255) / 256, (long long)sms * 8));
    sg::count_launches(1);
    sg::sizer_targets_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(rowptrC, m, T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        sg::set_last_error(cudaGetErrorString(e));
        return SPGEMM_ERR_CUDA;
    }
    return SPGEMM_OK;
}

spgemm_status spgemm_sizer_save(const float* params, int32_t F, void* stream, void* buf,
                                size_t buf_bytes, size_t* bytes_out) {
    if (F < 1 || F > 64 || !bytes_out) {
        sg::set_last_error("sizer_save: bad arguments");
        return SPGEMM_ERR_INVALID_ARG;
    }
    const size_t need = sg::sizer_record_bytes(F);
    *bytes_out = need;
    if (!buf) return SPGEMM_OK;  // size query
    if (buf_bytes < need || !params) {
        sg::set_last_error("sizer_save: buffer smaller than the record, or params NULL");
        return SPGEMM_ERR_INVALID_ARG;
    }
    unsigned char* out = (unsigned char*)buf;
    const uint32_t head[6] = {sg::kSizerVersion, (uint32_t)F, (uint32_t)sg::kSizerH,
                              sg::kSizerFeatureSet, sg::kSizerTarget,
                              (uint32_t)sg::sizer_params(F)};
    std::memcpy(out, sg::kSizerMagic, 8);
    std::memcpy(out + 8, head, sizeof(head));
    const size_t pbytes = sizeof(float) * (size_t)sg::sizer_params(F);
    cudaError_t e = cudaMemcpyAsync(out + sg::kSizerHeader, params, pbytes, cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        sg::set_last_error(cudaGetErrorString(e));
        return SPGEMM_ERR_CUDA;
    }
    const uint64_t h = sg::fnv1a(out, sg::kSizerHeader + pbytes);
    std::memcpy(out + sg::kSizerHeader + pbytes, &h, sizeof(h));
    return SPGEMM_OK;
}

spgemm_status spgemm_sizer_load(const void* buf, size_t buf_bytes, int32_t F, float* params,
                                void* stream) {
    const unsigned char* in = (const unsigned char*)buf;
    if (!in || F < 1 || F > 64) {
        sg::set_last_error("sizer_load: bad arguments");
        return SPGEMM_ERR_INVALID_ARG;
    }
    if (buf_bytes < sg::kSizerHeader || std::memcmp(in, sg::kSizerMagic, 8) != 0) {
        sg::set_last_error("sizer_load: not a predictor record");
        return SPGEMM_ERR_INVALID_ARG;
    }
    uint32_t head[6];
    std::memcpy(head, in + 8, sizeof(head));
    if (head[0] != sg::kSizerVersion) {
        sg::set_last_error("sizer_load: unknown record version");
        return SPGEMM_ERR_NOT_SUPPORTED;
    }
    if (head[1] != (uint32_t)F || head[2] != (uint32_t)sg::kSizerH ||
        head[3] != sg::kSizerFeatureSet || head[4] != sg::kSizerTarget ||
        head[5] != (uint32_t)sg::sizer_params(F)) {
        sg::set_last_error("sizer_load: record is for another network, feature set or target");
        return SPGEMM_ERR_INVALID_ARG;
    }
    const size_t pbytes = sizeof(float) * (size_t)sg::sizer_params(F);
    if (buf_bytes < sg::sizer_record_bytes(F)) {
        sg::set_last_error("sizer_load: record truncated");
        return SPGEMM_ERR_INVALID_ARG;
    }
    uint64_t h = 0;
    std::memcpy(&h, in + sg::kSizerHeader + pbytes, sizeof(h));
    if (h != sg::fnv1a(in, sg::kSizerHeader + pbytes)) {
        sg::set_last_error("sizer_load: record hash mismatch");
        return SPGEMM_ERR_INVALID_ARG;
    }
    if (!params) {
        sg::set_last_error("sizer_load: params is NULL");
        return SPGEMM_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaMemcpyAsync(params, in + sg::kSizerHeader, pbytes, cudaMemcpyHostToDevice,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        sg::set_last_error(cudaGetErrorString(e));
        return SPGEMM_ERR_CUDA;
    }
    return SPGEMM_OK;
}

}  // extern "C"
