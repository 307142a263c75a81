// pgg_mlp.cu -- the surrogate network: a 202-128-128-2 MLP with BF16 parameters and FP32
// accumulation, trained on the GPU by hand-written forward, backward and Adam kernels.
//
// Input: the first 200 samples of rho_C(t) of a run and its normalised (r, K); output:
// p = sigmoid(z0), the probability that the run falls into the absorbing all-defector state,
// and rho = sigmoid(z1), its stationary cooperator fraction (Eq. (4)). The loss of a batch of
// B samples is mean BCE(p, y_abs) + mean(mask * (rho - y_rho)^2); Adam (bias corrected)
// updates an FP32 master copy, whose round-to-nearest-even BF16 image is what the forward
// and backward passes read.
//
// Every kernel accumulates in a fixed order (one thread per output, sequential sums), so the
// results are deterministic; the hidden layers' forward and weight-gradient kernels stage their
// operands through shared memory for coalesced reads and keep that order. The whole training step is about 20 MFLOP for B = 256, far too
// small for tensor cores to matter: plain FMA kernels keep it simple and exact to reason about.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>

#include "pgg.h"
#include "pgg_internal.h"

namespace {

constexpr int kIn = 202, kHid = 128, kOut = 2;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid, kParams = kOffB3 + kOut;

__global__ void k_quantize(const float *__restrict__ master, __nv_bfloat16 *__restrict__ q, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        q[i] = __float2bfloat16_rn(master[i]);
}

// A[b][o] = bias[o] + sum_i W[o][i] X[b][i]; H = max(A, 0) if H is not NULL.
__global__ void k_dense(const float *__restrict__ X, const __nv_bfloat16 *__restrict__ W,
                        const __nv_bfloat16 *__restrict__ bias, float *__restrict__ A, float *__restrict__ H,
                        int B, int n_in, int n_out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * n_out) return;
    const int b = idx / n_out, o = idx - b * n_out;
    const float *x = X + static_cast<size_t>(b) * n_in;
    const __nv_bfloat16 *w = W + static_cast<size_t>(o) * n_in;
    float acc = __bfloat162float(bias[o]);
    for (int i = 0; i < n_in; ++i) acc = fmaf(__bfloat162float(w[i]), x[i], acc);
    A[idx] = acc;
    if (H) H[idx] = fmaxf(acc, 0.0f);
}

// The same for n_out % 32 == 0 through shared memory: a 256-thread block computes 32 outputs
// (lane) of 8 rows (warp); W and X pass through shared memory in chunks of 32 inputs, read with
// consecutive addresses across the lanes (a thread of k_dense walks its own weight row, so a warp's
// weight loads lie n_in elements apart). Each thread sums its output over the inputs in the same
// order as k_dense, with the same operands, so the results are the same bit for bit.
__global__ void __launch_bounds__(256) k_dense_tiled(const float *__restrict__ X, const __nv_bfloat16 *__restrict__ W,
                                                     const __nv_bfloat16 *__restrict__ bias, float *__restrict__ A,
                                                     float *__restrict__ H, int B, int n_in, int n_out) {
    __shared__ float ws[32][33];  // [output][input], padded: lanes read a column without conflicts
    __shared__ float xs[8][32];   // [row][input]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int o0 = blockIdx.y * 32, o = o0 + lane, b = blockIdx.x * 8 + warp;  // rows in x: up to 2^20 of them
    float acc = __bfloat162float(bias[o]);
    for (int i0 = 0; i0 < n_in; i0 += 32) {
        const int ni = min(32, n_in - i0);
        for (int rr = warp; rr < 32; rr += 8)
            ws[rr][lane] = lane < ni ? __bfloat162float(W[static_cast<size_t>(o0 + rr) * n_in + i0 + lane]) : 0.0f;
        xs[warp][lane] = b < B && lane < ni ? X[static_cast<size_t>(b) * n_in + i0 + lane] : 0.0f;
        __syncthreads();
        if (b < B)
            for (int ii = 0; ii < ni; ++ii) acc = fmaf(ws[lane][ii], xs[warp][ii], acc);
        __syncthreads();
    }
    if (b < B) {
        A[static_cast<size_t>(b) * n_out + o] = acc;
        if (H) H[static_cast<size_t>(b) * n_out + o] = fmaxf(acc, 0.0f);
    }
}

__device__ __forceinline__ float sigmoidf(float z) { return 1.0f / (1.0f + expf(-z)); }

// Heads: out[b] = (sigmoid(z0), sigmoid(z1)).
__global__ void k_heads(const float *__restrict__ Z, float *__restrict__ out, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    out[2 * b] = sigmoidf(Z[2 * b]);
    out[2 * b + 1] = sigmoidf(Z[2 * b + 1]);
}

// Loss and its gradient with respect to z (one block; fixed reduction order).
__global__ void k_loss(const float *__restrict__ Z, const float *__restrict__ Y, float *__restrict__ dZ,
                       float *__restrict__ loss, int B) {
    __shared__ float part[256];
    float acc = 0.0f;
    const float invB = 1.0f / static_cast<float>(B);
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float z0 = Z[2 * b], z1 = Z[2 * b + 1];
        const float y = Y[3 * b], yr = Y[3 * b + 1], m = Y[3 * b + 2];
        const float p = sigmoidf(z0), rho = sigmoidf(z1);
        // BCE written through z: max(z, 0) - y z + log(1 + exp(-|z|))
        const float bce = fmaxf(z0, 0.0f) - y * z0 + log1pf(expf(-fabsf(z0)));
        const float d = rho - yr;
        acc += bce + m * d * d;
        dZ[2 * b] = (p - y) * invB;
        dZ[2 * b + 1] = m * 2.0f * d * rho * (1.0f - rho) * invB;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = part[0] * invB;
}

// dAprev[b][i] = (sum_o dA[b][o] W[o][i]) * (Aprev[b][i] > 0)
__global__ void k_dense_bwd_data(const float *__restrict__ dA, const __nv_bfloat16 *__restrict__ W,
                                 const float *__restrict__ Aprev, float *__restrict__ dAprev, int B, int n_in,
                                 int n_out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * n_in) return;
    const int b = idx / n_in, i = idx - b * n_in;
    float acc = 0.0f;
    for (int o = 0; o < n_out; ++o) acc = fmaf(dA[static_cast<size_t>(b) * n_out + o], __bfloat162float(W[static_cast<size_t>(o) * n_in + i]), acc);
    dAprev[idx] = Aprev[idx] > 0.0f ? acc : 0.0f;
}

// gW[o][i] = sum_b dA[b][o] Xin[b][i] and gb[o] = sum_b dA[b][o]: a 256-thread block computes 8
// outputs (warp) by 32 inputs (lane), input n_in standing for the bias (a column of ones:
// fmaf(d, 1, acc) rounds exactly as acc + d does). dA and Xin pass through shared memory in chunks
// of 32 rows, read with consecutive addresses; each thread sums its own output over the rows
// b = 0 .. B-1 in order, one fmaf per row, so the result does not depend on the launch shape.
__global__ void __launch_bounds__(256) k_dense_bwd_weight_tiled(const float *__restrict__ dA, const float *__restrict__ Xin,
                                                                float *__restrict__ gW, float *__restrict__ gb, int B,
                                                                int n_in, int n_out) {
    __shared__ float das[32][8];   // [row][output]
    __shared__ float xs[32][32];   // [row][input]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int o0 = blockIdx.y * 8, i = blockIdx.x * 32 + lane, o = o0 + warp;
    float acc = 0.0f;
    for (int b0 = 0; b0 < B; b0 += 32) {
        const int nb = min(32, B - b0);
        const int bb_l = threadIdx.x >> 3, oo_l = threadIdx.x & 7;  // 32 rows x 8 outputs
        das[bb_l][oo_l] = bb_l < nb && o0 + oo_l < n_out ? dA[static_cast<size_t>(b0 + bb_l) * n_out + o0 + oo_l] : 0.0f;
        for (int bb = warp; bb < 32; bb += 8)
            xs[bb][lane] = bb >= nb || i > n_in ? 0.0f : i == n_in ? 1.0f : Xin[static_cast<size_t>(b0 + bb) * n_in + i];
        __syncthreads();
        for (int bb = 0; bb < nb; ++bb) acc = fmaf(das[bb][warp], xs[bb][lane], acc);
        __syncthreads();
    }
    if (o < n_out && i < n_in) gW[static_cast<size_t>(o) * n_in + i] = acc;
    if (o < n_out && i == n_in) gb[o] = acc;
}

__global__ void k_adam(float *__restrict__ master, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, __nv_bfloat16 *__restrict__ q, int n, float lr, float beta1,
                       float beta2, float eps, float bc1, float bc2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
        const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / bc1, vh = vi / bc2;
        const float w = master[i] - lr * mh / (sqrtf(vh) + eps);
        master[i] = w;
        q[i] = __float2bfloat16_rn(w);
    }
}

int mfail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return pgg::record_error(code, buf);
}

#define PGG_MCUDA(call)                                                                           \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return mfail(PGG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int blocks_for(long n, int t) { return static_cast<int>((n + t - 1) / t); }

}  // namespace

struct pgg_mlp {
    int max_batch = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __nv_bfloat16 *q = nullptr;
    float *a1 = nullptr, *h1 = nullptr, *a2 = nullptr, *h2 = nullptr, *z = nullptr;
    float *dz = nullptr, *da2 = nullptr, *da1 = nullptr, *loss = nullptr;
    long t = 0;  // Adam step counter
};

namespace {

// Forward pass over B rows of X into the saved activations.
int forward(pgg_mlp *n, const float *X, int B) {
    const int T = 256;
    const __nv_bfloat16 *q = n->q;
    static_assert(kHid % 32 == 0, "hidden layers go through k_dense_tiled");
    const dim3 grid(static_cast<unsigned>((B + 7) / 8), kHid / 32);
    k_dense_tiled<<<grid, 256, 0, n->stream>>>(X, q + kOffW1, q + kOffB1, n->a1, n->h1, B, kIn, kHid);
    k_dense_tiled<<<grid, 256, 0, n->stream>>>(n->h1, q + kOffW2, q + kOffB2, n->a2, n->h2, B, kHid, kHid);
    k_dense<<<blocks_for(long(B) * kOut, T), T, 0, n->stream>>>(n->h2, q + kOffW3, q + kOffB3, n->z, nullptr, B, kHid, kOut);
    PGG_MCUDA(cudaGetLastError());
    return PGG_OK;
}

// Loss and full parameter gradient into n->grad.
int backward(pgg_mlp *n, const float *X, const float *Y, int B) {
    const int T = 256;
    const __nv_bfloat16 *q = n->q;
    float *g = n->grad;
    k_loss<<<1, 256, 0, n->stream>>>(n->z, Y, n->dz, n->loss, B);
    // weight and bias gradients: 8 outputs x 32 inputs (the last one the bias) per block
    const dim3 gw3((kHid + 1 + 31) / 32, (kOut + 7) / 8), gw2((kHid + 1 + 31) / 32, kHid / 8), gw1((kIn + 1 + 31) / 32, kHid / 8);
    k_dense_bwd_weight_tiled<<<gw3, 256, 0, n->stream>>>(n->dz, n->h2, g + kOffW3, g + kOffB3, B, kHid, kOut);
    k_dense_bwd_data<<<blocks_for(long(B) * kHid, T), T, 0, n->stream>>>(n->dz, q + kOffW3, n->a2, n->da2, B, kHid, kOut);
    k_dense_bwd_weight_tiled<<<gw2, 256, 0, n->stream>>>(n->da2, n->h1, g + kOffW2, g + kOffB2, B, kHid, kHid);
    k_dense_bwd_data<<<blocks_for(long(B) * kHid, T), T, 0, n->stream>>>(n->da2, q + kOffW2, n->a1, n->da1, B, kHid, kHid);
    k_dense_bwd_weight_tiled<<<gw1, 256, 0, n->stream>>>(n->da1, X, g + kOffW1, g + kOffB1, B, kIn, kHid);
    PGG_MCUDA(cudaGetLastError());
    return PGG_OK;
}

}  // namespace

extern "C" {

int pgg_mlp_info(int *n_in, int *n_hidden, int *n_out, int *n_params) {
    if (n_in) *n_in = kIn;
    if (n_hidden) *n_hidden = kHid;
    if (n_out) *n_out = kOut;
    if (n_params) *n_params = kParams;
    return PGG_OK;
}

int pgg_mlp_create(pgg_mlp **out, int max_batch, void *cuda_stream) {
    pgg::clear_error();
    if (!out) return mfail(PGG_ERR_ARG, "pgg_mlp_create: out is NULL");
    *out = nullptr;
    if (max_batch < 1 || max_batch > (1 << 20)) return mfail(PGG_ERR_ARG, "pgg_mlp_create: max_batch in [1, 2^20]");
    pgg_mlp *n = new (std::nothrow) pgg_mlp();
    if (!n) return mfail(PGG_ERR_OOM, "pgg_mlp_create: host allocation failed");
    n->max_batch = max_batch;
    n->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&n->device);
    const size_t P = kParams * sizeof(float), Bh = size_t(max_batch) * kHid * sizeof(float);
    if (e == cudaSuccess) e = cudaMalloc(&n->master, P);
    if (e == cudaSuccess) e = cudaMalloc(&n->m, P);
    if (e == cudaSuccess) e = cudaMalloc(&n->v, P);
    if (e == cudaSuccess) e = cudaMalloc(&n->grad, P);
    if (e == cudaSuccess) e = cudaMalloc(&n->q, kParams * sizeof(__nv_bfloat16));
    for (float **p : {&n->a1, &n->h1, &n->a2, &n->h2, &n->da2, &n->da1})
        if (e == cudaSuccess) e = cudaMalloc(p, Bh);
    if (e == cudaSuccess) e = cudaMalloc(&n->z, size_t(max_batch) * kOut * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->dz, size_t(max_batch) * kOut * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(n->master, 0, P, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, P, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, P, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->q, 0, kParams * sizeof(__nv_bfloat16), n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) {
        pgg_mlp_destroy(n);
        return mfail(PGG_ERR_OOM, "pgg_mlp_create: %s", cudaGetErrorString(e));
    }
    *out = n;
    return PGG_OK;
}

int pgg_mlp_set_params(pgg_mlp *n, const float *host_master) {
    pgg::clear_error();
    if (!n || !host_master) return mfail(PGG_ERR_ARG, "pgg_mlp_set_params: NULL argument");
    PGG_MCUDA(cudaSetDevice(n->device));
    PGG_MCUDA(cudaMemcpyAsync(n->master, host_master, kParams * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    PGG_MCUDA(cudaMemsetAsync(n->m, 0, kParams * sizeof(float), n->stream));
    PGG_MCUDA(cudaMemsetAsync(n->v, 0, kParams * sizeof(float), n->stream));
    k_quantize<<<blocks_for(kParams, 256), 256, 0, n->stream>>>(n->master, n->q, kParams);
    PGG_MCUDA(cudaGetLastError());
    PGG_MCUDA(cudaStreamSynchronize(n->stream));
    n->t = 0;
    return PGG_OK;
}

int pgg_mlp_get_params(pgg_mlp *n, float *host_master, uint16_t *host_bf16) {
    pgg::clear_error();
    if (!n) return mfail(PGG_ERR_ARG, "pgg_mlp_get_params: NULL network");
    PGG_MCUDA(cudaSetDevice(n->device));
    if (host_master)
        PGG_MCUDA(cudaMemcpyAsync(host_master, n->master, kParams * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    if (host_bf16)
        PGG_MCUDA(cudaMemcpyAsync(host_bf16, n->q, kParams * sizeof(uint16_t), cudaMemcpyDeviceToHost, n->stream));
    PGG_MCUDA(cudaStreamSynchronize(n->stream));
    return PGG_OK;
}

int pgg_mlp_forward(pgg_mlp *n, const float *X, int B, float *out) {
    pgg::clear_error();
    if (!n || !X || !out) return mfail(PGG_ERR_ARG, "pgg_mlp_forward: NULL argument");
    if (B < 1 || B > n->max_batch) return mfail(PGG_ERR_ARG, "pgg_mlp_forward: B = %d not in [1, %d]", B, n->max_batch);
    PGG_MCUDA(cudaSetDevice(n->device));
    int rc = forward(n, X, B);
    if (rc) return rc;
    k_heads<<<blocks_for(B, 256), 256, 0, n->stream>>>(n->z, out, B);
    PGG_MCUDA(cudaGetLastError());
    return PGG_OK;
}

int pgg_mlp_loss_grad(pgg_mlp *n, const float *X, const float *Y, int B, float *loss_out, float *grad_out) {
    pgg::clear_error();
    if (!n || !X || !Y) return mfail(PGG_ERR_ARG, "pgg_mlp_loss_grad: NULL argument");
    if (B < 1 || B > n->max_batch) return mfail(PGG_ERR_ARG, "pgg_mlp_loss_grad: B = %d not in [1, %d]", B, n->max_batch);
    PGG_MCUDA(cudaSetDevice(n->device));
    int rc = forward(n, X, B);
    if (!rc) rc = backward(n, X, Y, B);
    if (rc) return rc;
    if (loss_out) PGG_MCUDA(cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
    if (grad_out) PGG_MCUDA(cudaMemcpyAsync(grad_out, n->grad, kParams * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
    return PGG_OK;
}

int pgg_mlp_train_step(pgg_mlp *n, const float *X, const float *Y, int B, float lr, float *loss_out) {
    pgg::clear_error();
    if (!n || !X || !Y) return mfail(PGG_ERR_ARG, "pgg_mlp_train_step: NULL argument");
    if (B < 1 || B > n->max_batch) return mfail(PGG_ERR_ARG, "pgg_mlp_train_step: B = %d not in [1, %d]", B, n->max_batch);
    if (!(lr > 0.0f)) return mfail(PGG_ERR_ARG, "pgg_mlp_train_step: lr must be > 0");
    PGG_MCUDA(cudaSetDevice(n->device));
    int rc = forward(n, X, B);
    if (!rc) rc = backward(n, X, Y, B);
    if (rc) return rc;
    n->t += 1;
    const double beta1 = 0.9, beta2 = 0.999;
    const float bc1 = static_cast<float>(1.0 - std::pow(beta1, double(n->t)));
    const float bc2 = static_cast<float>(1.0 - std::pow(beta2, double(n->t)));
    k_adam<<<blocks_for(kParams, 256), 256, 0, n->stream>>>(n->master, n->grad, n->m, n->v, n->q, kParams, lr, 0.9f,
                                                             0.999f, 1e-8f, bc1, bc2);
    PGG_MCUDA(cudaGetLastError());
    if (loss_out) PGG_MCUDA(cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
    return PGG_OK;
}

void pgg_mlp_destroy(pgg_mlp *n) {
    if (!n) return;
    cudaSetDevice(n->device);
    cudaStreamSynchronize(n->stream);
    for (void *p : {static_cast<void *>(n->master), static_cast<void *>(n->m), static_cast<void *>(n->v),
                    static_cast<void *>(n->grad), static_cast<void *>(n->q), static_cast<void *>(n->a1),
                    static_cast<void *>(n->h1), static_cast<void *>(n->a2), static_cast<void *>(n->h2),
                    static_cast<void *>(n->z), static_cast<void *>(n->dz), static_cast<void *>(n->da2),
                    static_cast<void *>(n->da1), static_cast<void *>(n->loss)})
        if (p) cudaFree(p);
    delete n;
}

}  // extern "C"
