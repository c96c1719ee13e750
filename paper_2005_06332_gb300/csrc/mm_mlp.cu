// mm_mlp.cu -- the learned cost model: a 16 -> 64 -> 64 -> 1 MLP (ReLU),
// BF16 weights, FP32 accumulation, trained with Adam on FP32 master
// weights, by hand-written kernels.
//
// It predicts a neuron's per-step solve time from its morphology features
// so that the work queue can take the longest items first (the paper's
// priority(size) and sorting by size, Sec. 4, with a learned key).
//
// Parameters, flat, in this order (MM_MLP_PARAMS = 5313 values):
//   W1 [64 x 16] row-major, b1 [64], W2 [64 x 64], b2 [64], W3 [1 x 64], b3 [1].
// Inputs are standardised with per-feature mean / std, targets with mean /
// std, both taken from the training set by mm_mlp_train.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "mm.h"

namespace {

constexpr int kIn = MM_N_FEATURES, kH = 64;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kParams = kOffB3 + 1;
static_assert(kParams == MM_MLP_PARAMS, "parameter count");

// y[s, u] = act(sum_k x[s, k] W[u, k] + b[u]) for one dense layer; one thread
// per (sample, unit); BF16 weights and bias widened to FP32.
__global__ void dense_fwd_kernel(const float *__restrict__ x, int K, const __nv_bfloat16 *__restrict__ W,
                                 const __nv_bfloat16 *__restrict__ b, int U, int64_t n, int relu,
                                 float *__restrict__ y)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * U; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t / U;
        const int u = (int)(t - s * U);
        float acc = __bfloat162float(b[u]);
        const float *xs = x + s * K;
        const __nv_bfloat16 *wu = W + (int64_t)u * K;
        for (int k = 0; k < K; ++k) acc = fmaf(xs[k], __bfloat162float(wu[k]), acc);
        y[t] = relu ? fmaxf(acc, 0.0f) : acc;
    }
}

// dW[u, k] = sum_s dy[s, u] x[s, k], db[u] = sum_s dy[s, u]; one thread per
// weight (k == K: the bias), FP32 accumulation over the samples.
__global__ void dense_wgrad_kernel(const float *__restrict__ x, int K, const float *__restrict__ dy, int U,
                                   int64_t n, float *__restrict__ dW, float *__restrict__ db)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= U * (K + 1)) return;
    const int u = t / (K + 1), k = t - u * (K + 1);
    float acc = 0.0f;
    if (k < K) {
        for (int64_t s = 0; s < n; ++s) acc = fmaf(dy[s * U + u], x[s * K + k], acc);
        dW[(int64_t)u * K + k] = acc;
    } else {
        for (int64_t s = 0; s < n; ++s) acc += dy[s * U + u];
        db[u] = acc;
    }
}

// dx[s, k] = (sum_u dy[s, u] W[u, k]) * [x[s, k] > 0]  (ReLU of the layer below)
__global__ void dense_xgrad_kernel(const float *__restrict__ dy, int U, const __nv_bfloat16 *__restrict__ W, int K,
                                   const float *__restrict__ xact, int64_t n, float *__restrict__ dx)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * K; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t / K;
        const int k = (int)(t - s * K);
        float acc = 0.0f;
        for (int u = 0; u < U; ++u) acc = fmaf(dy[s * U + u], __bfloat162float(W[(int64_t)u * K + k]), acc);
        dx[t] = xact[t] > 0.0f ? acc : 0.0f;
    }
}

// Mean squared error of y vs target, and dL/dy = 2 (y - t) / n.
__global__ void mse_kernel(const float *__restrict__ y, const float *__restrict__ tgt, int64_t n,
                           float *__restrict__ dy, float *__restrict__ loss)
{
    __shared__ float part[256];
    float acc = 0.0f;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const float e = y[s] - tgt[s];
        dy[s] = 2.0f * e / (float)n;
        acc = fmaf(e, e, acc);
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, part[0] / (float)n);
}

// (x - mean) / std per feature
__global__ void standardise_kernel(const float *__restrict__ x, int64_t n, const float *__restrict__ mu,
                                   const float *__restrict__ sd, float *__restrict__ out)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * kIn; t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t % kIn);
        out[t] = (x[t] - mu[k]) / sd[k];
    }
}

// Adam on the FP32 master weights; refreshes the BF16 compute copy.
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, int n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
}

__global__ void to_bf16_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

int blocks_for(int64_t n, int t)
{
    int64_t b = (n + t - 1) / t;
    return (int)(b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b));
}

}  // namespace

struct mm_mlp {
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, gradient, Adam moments
    __nv_bfloat16 *wb = nullptr;                                  // BF16 compute copy
    float *mu = nullptr, *sd = nullptr;                           // feature standardisation (device)
    float y_mu = 0.0f, y_sd = 1.0f;                               // target standardisation
    int64_t steps = 0;                                            // Adam steps taken
    // work buffers for n samples
    int64_t cap = 0;
    float *x = nullptr, *h1 = nullptr, *h2 = nullptr, *y = nullptr, *t = nullptr, *dy = nullptr, *dh2 = nullptr,
          *dh1 = nullptr, *loss = nullptr;
};

namespace {

void free_work(mm_mlp *p)
{
    for (float *q : {p->x, p->h1, p->h2, p->y, p->t, p->dy, p->dh2, p->dh1, p->loss}) cudaFree(q);
    p->x = p->h1 = p->h2 = p->y = p->t = p->dy = p->dh2 = p->dh1 = p->loss = nullptr;
    p->cap = 0;
}

mm_status ensure_work(mm_mlp *p, int64_t n)
{
    if (n <= p->cap) return MM_OK;
    free_work(p);
    const size_t f = sizeof(float);
    if (cudaMalloc(&p->x, (size_t)n * kIn * f) != cudaSuccess || cudaMalloc(&p->h1, (size_t)n * kH * f) != cudaSuccess ||
        cudaMalloc(&p->h2, (size_t)n * kH * f) != cudaSuccess || cudaMalloc(&p->y, (size_t)n * f) != cudaSuccess ||
        cudaMalloc(&p->t, (size_t)n * f) != cudaSuccess || cudaMalloc(&p->dy, (size_t)n * f) != cudaSuccess ||
        cudaMalloc(&p->dh2, (size_t)n * kH * f) != cudaSuccess || cudaMalloc(&p->dh1, (size_t)n * kH * f) != cudaSuccess ||
        cudaMalloc(&p->loss, f) != cudaSuccess) {
        cudaGetLastError();
        free_work(p);
        return MM_ENOMEM;
    }
    p->cap = n;
    return MM_OK;
}

// forward on p->x (already standardised) -> p->h1, p->h2, p->y
void forward(mm_mlp *p, int64_t n)
{
    dense_fwd_kernel<<<blocks_for(n * kH, 256), 256>>>(p->x, kIn, p->wb + kOffW1, p->wb + kOffB1, kH, n, 1, p->h1);
    dense_fwd_kernel<<<blocks_for(n * kH, 256), 256>>>(p->h1, kH, p->wb + kOffW2, p->wb + kOffB2, kH, n, 1, p->h2);
    dense_fwd_kernel<<<blocks_for(n, 256), 256>>>(p->h2, kH, p->wb + kOffW3, p->wb + kOffB3, 1, n, 0, p->y);
}

// loss and gradient (into p->g) for targets in p->t
void backward(mm_mlp *p, int64_t n)
{
    cudaMemsetAsync(p->loss, 0, sizeof(float));
    mse_kernel<<<blocks_for(n, 256), 256>>>(p->y, p->t, n, p->dy, p->loss);
    dense_wgrad_kernel<<<blocks_for(1 * (kH + 1), 256), 256>>>(p->h2, kH, p->dy, 1, n, p->g + kOffW3, p->g + kOffB3);
    dense_xgrad_kernel<<<blocks_for(n * kH, 256), 256>>>(p->dy, 1, p->wb + kOffW3, kH, p->h2, n, p->dh2);
    dense_wgrad_kernel<<<blocks_for(kH * (kH + 1), 256), 256>>>(p->h1, kH, p->dh2, kH, n, p->g + kOffW2, p->g + kOffB2);
    dense_xgrad_kernel<<<blocks_for(n * kH, 256), 256>>>(p->dh2, kH, p->wb + kOffW2, kH, p->h1, n, p->dh1);
    dense_wgrad_kernel<<<blocks_for(kH * (kIn + 1), 256), 256>>>(p->x, kIn, p->dh1, kH, n, p->g + kOffW1, p->g + kOffB1);
}

mm_status upload_x(mm_mlp *p, const float *X, int64_t n)
{
    // raw features -> device, then standardised in place
    if (cudaMemcpy(p->dh1, X, (size_t)n * kIn * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return MM_ECUDA;
    standardise_kernel<<<blocks_for(n * kIn, 256), 256>>>(p->dh1, n, p->mu, p->sd, p->x);
    return cudaGetLastError() == cudaSuccess ? MM_OK : MM_ECUDA;
}

}  // namespace

extern "C" {

mm_status mm_mlp_create(uint64_t seed, mm_mlp **out)
{
    if (!out) return MM_EINVAL;
    *out = nullptr;
    mm_mlp *p = new (std::nothrow) mm_mlp();
    if (!p) return MM_ENOMEM;
    const size_t f = sizeof(float);
    if (cudaMalloc(&p->w, kParams * f) != cudaSuccess || cudaMalloc(&p->g, kParams * f) != cudaSuccess ||
        cudaMalloc(&p->m, kParams * f) != cudaSuccess || cudaMalloc(&p->v, kParams * f) != cudaSuccess ||
        cudaMalloc(&p->wb, kParams * sizeof(__nv_bfloat16)) != cudaSuccess || cudaMalloc(&p->mu, kIn * f) != cudaSuccess ||
        cudaMalloc(&p->sd, kIn * f) != cudaSuccess) {
        cudaGetLastError();
        mm_mlp_destroy(p);
        return MM_ENOMEM;
    }
    // He-uniform initial weights, zero biases (host generator, seeded)
    std::vector<float> w(kParams, 0.0f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int rows, int cols) {
        const float a = std::sqrt(6.0f / (float)cols);
        std::uniform_real_distribution<float> U(-a, a);
        for (int i = 0; i < rows * cols; ++i) w[(size_t)(off + i)] = U(rng);
    };
    fill(kOffW1, kH, kIn);
    fill(kOffW2, kH, kH);
    fill(kOffW3, 1, kH);
    std::vector<float> ones(kIn, 1.0f), zeros(kIn, 0.0f);
    mm_status st = mm_mlp_set_params(p, w.data(), kParams);
    if (st == MM_OK && (cudaMemcpy(p->mu, zeros.data(), kIn * f, cudaMemcpyHostToDevice) != cudaSuccess ||
                        cudaMemcpy(p->sd, ones.data(), kIn * f, cudaMemcpyHostToDevice) != cudaSuccess))
        st = MM_ECUDA;
    if (st != MM_OK) {
        mm_mlp_destroy(p);
        return st;
    }
    *out = p;
    return MM_OK;
}

mm_status mm_mlp_set_params(mm_mlp *p, const float *params, int64_t n)
{
    if (!p || !params || n != kParams) return MM_EINVAL;
    if (cudaMemcpy(p->w, params, kParams * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return MM_ECUDA;
    if (cudaMemset(p->m, 0, kParams * sizeof(float)) != cudaSuccess ||
        cudaMemset(p->v, 0, kParams * sizeof(float)) != cudaSuccess)
        return MM_ECUDA;
    to_bf16_kernel<<<blocks_for(kParams, 256), 256>>>(p->w, p->wb, kParams);
    p->steps = 0;
    return cudaDeviceSynchronize() == cudaSuccess ? MM_OK : MM_ECUDA;
}

mm_status mm_mlp_get_params(mm_mlp *p, float *params, int64_t n)
{
    if (!p || !params || n < kParams) return MM_EINVAL;
    return cudaMemcpy(params, p->w, kParams * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? MM_OK : MM_ECUDA;
}

mm_status mm_mlp_set_normalisation(mm_mlp *p, const float *mu, const float *sd, float y_mu, float y_sd)
{
    if (!p || !mu || !sd || !(y_sd > 0.0f)) return MM_EINVAL;
    for (int k = 0; k < kIn; ++k)
        if (!(sd[k] > 0.0f)) return MM_EINVAL;
    if (cudaMemcpy(p->mu, mu, kIn * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->sd, sd, kIn * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return MM_ECUDA;
    p->y_mu = y_mu;
    p->y_sd = y_sd;
    return MM_OK;
}

mm_status mm_mlp_loss_grad(mm_mlp *p, const float *X, const float *y, int64_t n, float *loss, float *grad,
                           int64_t grad_cap)
{
    if (!p || !X || !y || n < 1 || !loss || (grad && grad_cap < kParams)) return MM_EINVAL;
    mm_status st = ensure_work(p, n);
    if (st != MM_OK) return st;
    if ((st = upload_x(p, X, n)) != MM_OK) return st;
    std::vector<float> ty((size_t)n);
    for (int64_t s = 0; s < n; ++s) ty[(size_t)s] = (y[s] - p->y_mu) / p->y_sd;
    if (cudaMemcpy(p->t, ty.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return MM_ECUDA;
    forward(p, n);
    backward(p, n);
    if (cudaMemcpy(loss, p->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MM_ECUDA;
    if (grad && cudaMemcpy(grad, p->g, kParams * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MM_ECUDA;
    return cudaGetLastError() == cudaSuccess ? MM_OK : MM_ECUDA;
}

mm_status mm_mlp_train(mm_mlp *p, const float *X, const float *y, int64_t n, int32_t epochs, float lr,
                       float *loss_per_epoch)
{
    if (!p || !X || !y || n < 2 || epochs < 0 || !(lr > 0.0f)) return MM_EINVAL;
    // standardisation from the training set
    float mu[kIn], sd[kIn];
    for (int k = 0; k < kIn; ++k) {
        double s1 = 0.0, s2 = 0.0;
        for (int64_t s = 0; s < n; ++s) {
            const double v = X[s * kIn + k];
            s1 += v;
            s2 += v * v;
        }
        const double m = s1 / (double)n, var = s2 / (double)n - m * m;
        mu[k] = (float)m;
        sd[k] = (float)(var > 1e-12 ? std::sqrt(var) : 1.0);
    }
    double t1 = 0.0, t2 = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        t1 += y[s];
        t2 += (double)y[s] * y[s];
    }
    const double ym = t1 / (double)n, yv = t2 / (double)n - ym * ym;
    mm_status st = mm_mlp_set_normalisation(p, mu, sd, (float)ym, (float)(yv > 1e-24 ? std::sqrt(yv) : 1.0));
    if (st != MM_OK) return st;
    if ((st = ensure_work(p, n)) != MM_OK) return st;
    if ((st = upload_x(p, X, n)) != MM_OK) return st;
    std::vector<float> ty((size_t)n);
    for (int64_t s = 0; s < n; ++s) ty[(size_t)s] = (y[s] - p->y_mu) / p->y_sd;
    if (cudaMemcpy(p->t, ty.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return MM_ECUDA;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int32_t e = 0; e < epochs; ++e) {
        forward(p, n);
        backward(p, n);
        p->steps++;
        const float c1 = 1.0f - std::pow(b1, (float)p->steps), c2 = 1.0f - std::pow(b2, (float)p->steps);
        adam_kernel<<<blocks_for(kParams, 256), 256>>>(p->w, p->g, p->m, p->v, p->wb, kParams, lr, b1, b2, eps, c1, c2);
        if (loss_per_epoch &&
            cudaMemcpy(&loss_per_epoch[e], p->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
            return MM_ECUDA;
    }
    return cudaDeviceSynchronize() == cudaSuccess && cudaGetLastError() == cudaSuccess ? MM_OK : MM_ECUDA;
}

mm_status mm_mlp_predict(mm_mlp *p, const float *X, int64_t n, float *out)
{
    if (!p || !X || !out || n < 1) return MM_EINVAL;
    mm_status st = ensure_work(p, n);
    if (st != MM_OK) return st;
    if ((st = upload_x(p, X, n)) != MM_OK) return st;
    forward(p, n);
    if (cudaMemcpy(out, p->y, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MM_ECUDA;
    for (int64_t s = 0; s < n; ++s) out[s] = out[s] * p->y_sd + p->y_mu;
    return MM_OK;
}

void mm_mlp_destroy(mm_mlp *p)
{
    if (!p) return;
    free_work(p);
    for (void *q : {(void *)p->w, (void *)p->g, (void *)p->m, (void *)p->v, (void *)p->wb, (void *)p->mu, (void *)p->sd})
        cudaFree(q);
    delete p;
}

}  // extern "C"
