// Surrogate network for the critical body force: forward, backward, Gaussian
// negative log-likelihood and Adam as hand-written FP32 CUDA kernels.
//
// Not part of the paper: the network only seeds the bisection brackets of
// lbm_critical_pressure_batch, which alone decides the result.
// Network 5 -> 128 -> 128 -> 128 -> 2 with SiLU hidden units; outputs
// (mu, s) = (predicted log g_crit, log predicted variance); per-sample loss
// 0.5 (exp(-s) (y - mu)^2 + s), averaged over the batch.  Parameters flat:
// W1 [128x5], b1, W2 [128x128], b2, W3 [128x128], b3, W4 [2x128], b4.
//
// The layers are small dense products (batch x 128 x 128 at most); one
// strided shared-memory-tiled FP32 kernel serves the forward product
// (with bias and SiLU in its epilogue), dX = dZ W and dW = dZ^T X.  Each
// output element is summed by one thread in a fixed order, so gradients
// are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace {

constexpr int kLayers = 4;
constexpr int kSizes[kLayers + 1] = {5, 128, 128, 128, 2};
constexpr int kParams = 128 * 5 + 128 + 128 * 128 + 128 + 128 * 128 + 128 + 2 * 128 + 2;   // 34050
constexpr int kMaxBatch = 1 << 16;
constexpr int kTile = 16;

thread_local std::string g_mlp_err;

int mfail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_mlp_err = buf;
    return code;
}

#define MTRY(call)                                                                              \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return mfail(LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int w_off(int k) {
    int o = 0;
    for (int j = 0; j < k; j++) o += kSizes[j + 1] * kSizes[j] + kSizes[j + 1];
    return o;
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]); A(m, k) = A[m*sam + k*sak],
// B(k, n) = B[k*sbk + n*sbn]; C row-major with leading dimension N.
// If Z != nullptr the pre-activation is stored there and C gets SiLU(.).
__global__ void gemm_kernel(const float* __restrict__ A, int sam, int sak, const float* __restrict__ B, int sbk,
                            int sbn, const float* __restrict__ bias, float* __restrict__ C, float* __restrict__ Z,
                            int M, int N, int K) {
    __shared__ float As[kTile][kTile + 1];
    __shared__ float Bs[kTile][kTile + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int m = blockIdx.y * kTile + ty;
    const int n = blockIdx.x * kTile + tx;
    float acc = 0.0f;
    for (int k0 = 0; k0 < K; k0 += kTile) {
        const int ka = k0 + tx, kb = k0 + ty;
        As[ty][tx] = (m < M && ka < K) ? A[(size_t)m * sam + (size_t)ka * sak] : 0.0f;
        Bs[ty][tx] = (kb < K && n < N) ? B[(size_t)kb * sbk + (size_t)n * sbn] : 0.0f;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTile; kk++) acc = fmaf(As[ty][kk], Bs[kk][tx], acc);
        __syncthreads();
    }
    if (m < M && n < N) {
        if (bias) acc += bias[n];
        if (Z) {
            Z[(size_t)m * N + n] = acc;
            C[(size_t)m * N + n] = silu_f(acc);
        } else {
            C[(size_t)m * N + n] = acc;
        }
    }
}

// dOut from the Gaussian NLL; loss summed into *loss (already scaled by 1/B).
__global__ void nll_kernel(const float* __restrict__ out, const float* __restrict__ y, float* __restrict__ dout,
                           float* __restrict__ loss, int B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (i < B) {
        const float mu = out[2 * i], s = out[2 * i + 1];
        const float r = y[i] - mu, e = __expf(-s);
        l = 0.5f * (e * r * r + s) / (float)B;
        dout[2 * i] = -e * r / (float)B;
        dout[2 * i + 1] = 0.5f * (1.0f - e * r * r) / (float)B;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// d <- d * SiLU'(z) elementwise
__global__ void dsilu_kernel(float* __restrict__ d, const float* __restrict__ z, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] *= dsilu_f(z[i]);
}

// db[n] = sum_b dZ[b][n] (one thread per n, fixed order)
__global__ void colsum_kernel(const float* __restrict__ d, float* __restrict__ db, int B, int N) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int b = 0; b < B; b++) s += d[(size_t)b * N + n];
    db[n] = s;
}

__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void gather_kernel(const float* __restrict__ x, const float* __restrict__ y, const int* __restrict__ idx,
                              float* __restrict__ xb, float* __restrict__ yb, int B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const int j = idx[i];
    for (int k = 0; k < 5; k++) xb[5 * i + k] = x[5 * j + k];
    yb[i] = y[j];
}

}  // namespace

struct lbm_mlp_t {
    cudaStream_t stream = nullptr;
    float* theta = nullptr;   // device parameters
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* act[kLayers + 1] = {};   // act[0] = input batch, act[k] = layer k output
    float* pre[kLayers] = {};       // pre-activations of the hidden layers
    float* d0 = nullptr;            // two gradient buffers [B x 128]
    float* d1 = nullptr;
    float* y = nullptr;
    float* loss = nullptr;
    int* idx = nullptr;
    float* data_x = nullptr;        // training set on the device
    float* data_y = nullptr;
    int cap = 0;                    // batch capacity of the buffers
    int ndata = 0;
    long long t = 0;                // Adam step count
};

namespace {

void free_batch(lbm_mlp_t* h) {
    for (auto& p : h->act) cudaFree(p), p = nullptr;
    for (auto& p : h->pre) cudaFree(p), p = nullptr;
    cudaFree(h->d0);
    cudaFree(h->d1);
    cudaFree(h->y);
    cudaFree(h->idx);
    h->d0 = h->d1 = h->y = nullptr;
    h->idx = nullptr;
    h->cap = 0;
}

int ensure_batch(lbm_mlp_t* h, int B) {
    if (B <= h->cap) return LBM_OK;
    free_batch(h);
    for (int k = 0; k <= kLayers; k++) MTRY(cudaMalloc(&h->act[k], sizeof(float) * (size_t)B * kSizes[k]));
    for (int k = 0; k < kLayers; k++) MTRY(cudaMalloc(&h->pre[k], sizeof(float) * (size_t)B * kSizes[k + 1]));
    MTRY(cudaMalloc(&h->d0, sizeof(float) * (size_t)B * 128));
    MTRY(cudaMalloc(&h->d1, sizeof(float) * (size_t)B * 128));
    MTRY(cudaMalloc(&h->y, sizeof(float) * (size_t)B));
    MTRY(cudaMalloc(&h->idx, sizeof(int) * (size_t)B));
    h->cap = B;
    return LBM_OK;
}

void gemm(cudaStream_t st, const float* A, int sam, int sak, const float* B, int sbk, int sbn, const float* bias,
          float* C, float* Z, int M, int N, int K) {
    dim3 blk(kTile, kTile), grd((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
    gemm_kernel<<<grd, blk, 0, st>>>(A, sam, sak, B, sbk, sbn, bias, C, Z, M, N, K);
}

// forward of act[0] (B x 5) through all layers
void forward(lbm_mlp_t* h, int B) {
    for (int k = 0; k < kLayers; k++) {
        const int K = kSizes[k], N = kSizes[k + 1];
        const float* W = h->theta + w_off(k);
        const float* b = W + N * K;
        // Y = X W^T + b: A = X (B x K), B(k, n) = W[n][k]
        gemm(h->stream, h->act[k], K, 1, W, 1, K, b, h->act[k + 1], k < kLayers - 1 ? h->pre[k] : nullptr, B, N, K);
    }
}

// loss and gradient of the batch in act[0] / y into h->grad
void backward(lbm_mlp_t* h, int B) {
    cudaMemsetAsync(h->loss, 0, sizeof(float), h->stream);
    nll_kernel<<<(B + 127) / 128, 128, 0, h->stream>>>(h->act[kLayers], h->y, h->d0, h->loss, B);
    float* d = h->d0;
    float* dn = h->d1;
    for (int k = kLayers - 1; k >= 0; k--) {
        const int K = kSizes[k], N = kSizes[k + 1];
        if (k < kLayers - 1) dsilu_kernel<<<(B * N + 255) / 256, 256, 0, h->stream>>>(d, h->pre[k], B * N);
        float* gW = h->grad + w_off(k);
        float* gb = gW + N * K;
        // dW[n][k] = sum_b dZ[b][n] X[b][k]: A(m=n, kk=b) = d[b*N + n], B(kk=b, n=k) = X[b*K + k]
        gemm(h->stream, d, 1, N, h->act[k], K, 1, nullptr, gW, nullptr, N, K, B);
        colsum_kernel<<<(N + 127) / 128, 128, 0, h->stream>>>(d, gb, B, N);
        if (k > 0) {
            // dX[b][k] = sum_n dZ[b][n] W[n][k]
            const float* W = h->theta + w_off(k);
            gemm(h->stream, d, N, 1, W, K, 1, nullptr, dn, nullptr, B, K, N);
            float* t = d;
            d = dn;
            dn = t;
        }
    }
}

}  // namespace

extern "C" {

int lbm_mlp_create(const float* params, uint64_t seed, void* stream, lbm_mlp_t** out) {
    if (!out) return mfail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_mlp_t* h = new (std::nothrow) lbm_mlp_t();
    if (!h) return mfail(LBM_ENOMEM, "host allocation failed");
    h->stream = (cudaStream_t)stream;
    std::vector<float> init(kParams, 0.0f);
    if (params) {
        memcpy(init.data(), params, sizeof(float) * kParams);
    } else {
        // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
        std::mt19937_64 rng(seed);
        for (int k = 0; k < kLayers; k++) {
            const float lim = 1.0f / std::sqrt((float)kSizes[k]);
            std::uniform_real_distribution<float> u(-lim, lim);
            float* W = init.data() + w_off(k);
            for (int j = 0; j < kSizes[k + 1] * kSizes[k]; j++) W[j] = u(rng);
        }
    }
    auto bail = [&](int rc) {
        lbm_mlp_destroy(h);
        return rc;
    };
    if (cudaMalloc(&h->theta, sizeof(float) * kParams) != cudaSuccess ||
        cudaMalloc(&h->grad, sizeof(float) * kParams) != cudaSuccess ||
        cudaMalloc(&h->m, sizeof(float) * kParams) != cudaSuccess ||
        cudaMalloc(&h->v, sizeof(float) * kParams) != cudaSuccess || cudaMalloc(&h->loss, sizeof(float)) != cudaSuccess)
        return bail(mfail(LBM_ENOMEM, "device allocation failed"));
    if (cudaMemcpy(h->theta, init.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->m, 0, sizeof(float) * kParams) != cudaSuccess ||
        cudaMemset(h->v, 0, sizeof(float) * kParams) != cudaSuccess)
        return bail(mfail(LBM_ECUDA, "parameter upload failed"));
    *out = h;
    return LBM_OK;
}

int lbm_mlp_params(lbm_mlp_t* h, float* out_params, const float* in_params) {
    if (!h) return mfail(LBM_EINVAL, "handle is NULL");
    if (in_params) {
        MTRY(cudaMemcpyAsync(h->theta, in_params, sizeof(float) * kParams, cudaMemcpyHostToDevice, h->stream));
        h->t = 0;
        MTRY(cudaMemsetAsync(h->m, 0, sizeof(float) * kParams, h->stream));
        MTRY(cudaMemsetAsync(h->v, 0, sizeof(float) * kParams, h->stream));
    }
    if (out_params)
        MTRY(cudaMemcpyAsync(out_params, h->theta, sizeof(float) * kParams, cudaMemcpyDeviceToHost, h->stream));
    MTRY(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_mlp_forward(lbm_mlp_t* h, const float* x, int32_t B, float* out) {
    if (!h || !x || !out || B < 1 || B > kMaxBatch) return mfail(LBM_EINVAL, "bad argument");
    int rc = ensure_batch(h, B);
    if (rc) return rc;
    MTRY(cudaMemcpyAsync(h->act[0], x, sizeof(float) * 5 * B, cudaMemcpyHostToDevice, h->stream));
    forward(h, B);
    MTRY(cudaGetLastError());
    MTRY(cudaMemcpyAsync(out, h->act[kLayers], sizeof(float) * 2 * B, cudaMemcpyDeviceToHost, h->stream));
    MTRY(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_mlp_loss_grad(lbm_mlp_t* h, const float* x, const float* y, int32_t B, float* loss, float* grad) {
    if (!h || !x || !y || B < 1 || B > kMaxBatch) return mfail(LBM_EINVAL, "bad argument");
    int rc = ensure_batch(h, B);
    if (rc) return rc;
    MTRY(cudaMemcpyAsync(h->act[0], x, sizeof(float) * 5 * B, cudaMemcpyHostToDevice, h->stream));
    MTRY(cudaMemcpyAsync(h->y, y, sizeof(float) * B, cudaMemcpyHostToDevice, h->stream));
    forward(h, B);
    backward(h, B);
    MTRY(cudaGetLastError());
    if (loss) MTRY(cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (grad) MTRY(cudaMemcpyAsync(grad, h->grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost, h->stream));
    MTRY(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_mlp_adam(lbm_mlp_t* h, float lr) {
    if (!h) return mfail(LBM_EINVAL, "handle is NULL");
    h->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)h->t), c2 = 1.0f - std::pow(b2, (float)h->t);
    adam_kernel<<<(kParams + 255) / 256, 256, 0, h->stream>>>(h->theta, h->grad, h->m, h->v, kParams, lr, b1, b2,
                                                               1e-8f, c1, c2);
    MTRY(cudaGetLastError());
    return LBM_OK;
}

int lbm_mlp_train(lbm_mlp_t* h, const float* x, const float* y, int32_t n, int32_t epochs, int32_t batch, float lr,
                  uint64_t seed, float* last_loss) {
    if (!h || !x || !y || n < 1 || epochs < 0 || batch < 1 || batch > kMaxBatch)
        return mfail(LBM_EINVAL, "bad argument");
    int rc = ensure_batch(h, batch);
    if (rc) return rc;
    if (n > h->ndata) {
        cudaFree(h->data_x);
        cudaFree(h->data_y);
        h->data_x = h->data_y = nullptr;
        MTRY(cudaMalloc(&h->data_x, sizeof(float) * 5 * (size_t)n));
        MTRY(cudaMalloc(&h->data_y, sizeof(float) * (size_t)n));
        h->ndata = n;
    }
    MTRY(cudaMemcpyAsync(h->data_x, x, sizeof(float) * 5 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    MTRY(cudaMemcpyAsync(h->data_y, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    std::mt19937_64 rng(seed);
    std::vector<int> perm(n);
    for (int i = 0; i < n; i++) perm[i] = i;
    std::vector<int> order;
    for (int e = 0; e < epochs; e++) {
        std::shuffle(perm.begin(), perm.end(), rng);
        for (int s = 0; s + batch <= n || (s == 0 && n < batch); s += batch) {
            const int B = std::min(batch, n - s);
            MTRY(cudaMemcpyAsync(h->idx, perm.data() + s, sizeof(int) * B, cudaMemcpyHostToDevice, h->stream));
            gather_kernel<<<(B + 127) / 128, 128, 0, h->stream>>>(h->data_x, h->data_y, h->idx, h->act[0], h->y, B);
            forward(h, B);
            backward(h, B);
            rc = lbm_mlp_adam(h, lr);
            if (rc) return rc;
            // the index upload reads perm on the host: keep it alive until used
            MTRY(cudaStreamSynchronize(h->stream));
            if (n < batch) break;
        }
    }
    MTRY(cudaGetLastError());
    if (last_loss) MTRY(cudaMemcpyAsync(last_loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    MTRY(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

void lbm_mlp_destroy(lbm_mlp_t* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_batch(h);
    cudaFree(h->theta);
    cudaFree(h->grad);
    cudaFree(h->m);
    cudaFree(h->v);
    cudaFree(h->loss);
    cudaFree(h->data_x);
    cudaFree(h->data_y);
    delete h;
}

const char* lbm_mlp_last_error(void) { return g_mlp_err.c_str(); }

}  // extern "C"
