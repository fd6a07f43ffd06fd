// The cost model's network: 3-layer tanh perceptron, FP32, with hand-written
// forward, backward and Adam kernels (see tsm_mlp.h for the maths and the
// parameter layout).  Sizes are tiny (a few thousand parameters, thousands
// of samples), so the kernels favour a fixed, reproducible order over speed:
// one thread per sample for the activations and their gradients, one thread
// per parameter for the sums over samples (taken in sample order).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "tsm_internal.h"
#include "tsm_mlp.h"

struct tsm_mlp {
    int D, H, max_batch, P;
    float* params;  // device
    float* grads;
    float* m;
    float* v;
    float* act;     // max_batch x 2H   (h1, h2)
    float* dtmp;    // max_batch x (1 + 2H)  (dy, dh2, dh1)
    float* sqerr;   // max_batch
    int64_t step;
};

namespace tsm {
namespace mlp {

struct Off {
    int W1, b1, W2, b2, w3, b3, P;
};
__host__ __device__ inline Off offsets(int D, int H) {
    Off o;
    o.W1 = 0;
    o.b1 = H * D;
    o.W2 = o.b1 + H;
    o.b2 = o.W2 + H * H;
    o.w3 = o.b2 + H;
    o.b3 = o.w3 + H;
    o.P = o.b3 + 1;
    return o;
}

__global__ void k_forward(const float* __restrict__ p, int D, int H, const float* __restrict__ X, int n,
                          float* __restrict__ y, float* __restrict__ act) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Off o = offsets(D, H);
    float x[TSM_MLP_MAX_IN], h1[TSM_MLP_MAX_HIDDEN], h2[TSM_MLP_MAX_HIDDEN];
    for (int k = 0; k < D; ++k) x[k] = X[(int64_t)i * D + k];
    for (int j = 0; j < H; ++j) {
        float s = p[o.b1 + j];
        for (int k = 0; k < D; ++k) s = fmaf(p[o.W1 + j * D + k], x[k], s);
        h1[j] = tanhf(s);
    }
    for (int j = 0; j < H; ++j) {
        float s = p[o.b2 + j];
        for (int k = 0; k < H; ++k) s = fmaf(p[o.W2 + j * H + k], h1[k], s);
        h2[j] = tanhf(s);
    }
    float s = p[o.b3];
    for (int k = 0; k < H; ++k) s = fmaf(p[o.w3 + k], h2[k], s);
    y[i] = s;
    if (act) {
        for (int j = 0; j < H; ++j) {
            act[(int64_t)i * 2 * H + j] = h1[j];
            act[(int64_t)i * 2 * H + H + j] = h2[j];
        }
    }
}

// Per sample: dL/dy, dL/d(pre-activation of layer 2) and of layer 1.
__global__ void k_backward_samples(const float* __restrict__ p, int D, int H, const float* __restrict__ t, int n,
                                   const float* __restrict__ y, const float* __restrict__ act,
                                   float* __restrict__ dtmp, float* __restrict__ sqerr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Off o = offsets(D, H);
    const float e = y[i] - t[i];
    sqerr[i] = e * e;
    const float dy = 2.0f * e / (float)n;
    const float* h1 = act + (int64_t)i * 2 * H;
    const float* h2 = h1 + H;
    float* d = dtmp + (int64_t)i * (1 + 2 * H);
    d[0] = dy;
    float dh2[TSM_MLP_MAX_HIDDEN];
    for (int j = 0; j < H; ++j) {
        dh2[j] = dy * p[o.w3 + j] * (1.0f - h2[j] * h2[j]);
        d[1 + j] = dh2[j];
    }
    for (int k = 0; k < H; ++k) {
        float s = 0.0f;
        for (int j = 0; j < H; ++j) s = fmaf(p[o.W2 + j * H + k], dh2[j], s);
        d[1 + H + k] = s * (1.0f - h1[k] * h1[k]);
    }
}

// Per parameter: the sum over samples of its gradient terms, in sample order.
__global__ void k_backward_params(int D, int H, const float* __restrict__ X, int n, const float* __restrict__ act,
                                  const float* __restrict__ dtmp, float* __restrict__ g) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const Off o = offsets(D, H);
    if (q >= o.P) return;
    const int S = 1 + 2 * H;
    float s = 0.0f;
    if (q < o.b1) {  // W1[j][k] : dh1_j * x_k
        const int j = q / D, k = q - j * D;
        for (int i = 0; i < n; ++i) s = fmaf(dtmp[(int64_t)i * S + 1 + H + j], X[(int64_t)i * D + k], s);
    } else if (q < o.W2) {  // b1[j]
        const int j = q - o.b1;
        for (int i = 0; i < n; ++i) s += dtmp[(int64_t)i * S + 1 + H + j];
    } else if (q < o.b2) {  // W2[j][k] : dh2_j * h1_k
        const int r = q - o.W2, j = r / H, k = r - j * H;
        for (int i = 0; i < n; ++i) s = fmaf(dtmp[(int64_t)i * S + 1 + j], act[(int64_t)i * 2 * H + k], s);
    } else if (q < o.w3) {  // b2[j]
        const int j = q - o.b2;
        for (int i = 0; i < n; ++i) s += dtmp[(int64_t)i * S + 1 + j];
    } else if (q < o.b3) {  // w3[j] : dy * h2_j
        const int j = q - o.w3;
        for (int i = 0; i < n; ++i) s = fmaf(dtmp[(int64_t)i * S], act[(int64_t)i * 2 * H + H + j], s);
    } else {  // b3
        for (int i = 0; i < n; ++i) s += dtmp[(int64_t)i * S];
    }
    g[q] = s;
}

__global__ void k_loss(const float* __restrict__ sqerr, int n, float* loss) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += sqerr[i];
    *loss = (float)(s / n);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int P, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.0f - b1) * gq;
    const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace mlp
}  // namespace tsm

using namespace tsm;

extern "C" {

tsm_status tsm_mlp_create(int in_dim, int hidden, int max_batch, uint64_t seed, tsm_mlp** out) {
    if (!out || in_dim < 1 || in_dim > TSM_MLP_MAX_IN || hidden < 1 || hidden > TSM_MLP_MAX_HIDDEN ||
        max_batch < 1)
        return TSM_ERR_INVALID_VALUE;
    *out = nullptr;
    tsm_mlp* m = (tsm_mlp*)calloc(1, sizeof(tsm_mlp));
    if (!m) return TSM_ERR_ALLOC;
    const mlp::Off o = mlp::offsets(in_dim, hidden);
    m->D = in_dim;
    m->H = hidden;
    m->max_batch = max_batch;
    m->P = o.P;
    const size_t pb = sizeof(float) * o.P;
    bool ok = cudaMalloc(&m->params, pb) == cudaSuccess && cudaMalloc(&m->grads, pb) == cudaSuccess &&
              cudaMalloc(&m->m, pb) == cudaSuccess && cudaMalloc(&m->v, pb) == cudaSuccess &&
              cudaMalloc(&m->act, sizeof(float) * (size_t)max_batch * 2 * hidden) == cudaSuccess &&
              cudaMalloc(&m->dtmp, sizeof(float) * (size_t)max_batch * (1 + 2 * hidden)) == cudaSuccess &&
              cudaMalloc(&m->sqerr, sizeof(float) * (size_t)max_batch) == cudaSuccess;
    if (!ok) {
        tsm_mlp_destroy(m);
        return TSM_ERR_ALLOC;
    }
    std::vector<float> h(o.P, 0.0f);
    uint64_t s = seed;
    auto uni = [&](float bound) {
        return (float)(((double)(mlp::splitmix(s) >> 11) * 0x1p-53 * 2.0 - 1.0) * bound);
    };
    for (int i = 0; i < hidden * in_dim; ++i) h[o.W1 + i] = uni(1.0f / sqrtf((float)in_dim));
    for (int i = 0; i < hidden * hidden; ++i) h[o.W2 + i] = uni(1.0f / sqrtf((float)hidden));
    for (int i = 0; i < hidden; ++i) h[o.w3 + i] = uni(1.0f / sqrtf((float)hidden));
    if (cudaMemcpy(m->params, h.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->grads, 0, pb) != cudaSuccess || cudaMemset(m->m, 0, pb) != cudaSuccess ||
        cudaMemset(m->v, 0, pb) != cudaSuccess) {
        tsm_mlp_destroy(m);
        return TSM_ERR_LAUNCH;
    }
    *out = m;
    return TSM_OK;
}

void tsm_mlp_destroy(tsm_mlp* m) {
    if (!m) return;
    cudaFree(m->params);
    cudaFree(m->grads);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->act);
    cudaFree(m->dtmp);
    cudaFree(m->sqerr);
    free(m);
}

int tsm_mlp_param_count(const tsm_mlp* m) { return m ? m->P : -1; }

tsm_status tsm_mlp_set_params(tsm_mlp* m, const float* host) {
    if (!m || !host) return TSM_ERR_INVALID_VALUE;
    if (cudaMemcpy(m->params, host, sizeof(float) * m->P, cudaMemcpyHostToDevice) != cudaSuccess)
        return TSM_ERR_LAUNCH;
    // a new parameter vector restarts the optimiser
    if (cudaMemset(m->m, 0, sizeof(float) * m->P) != cudaSuccess ||
        cudaMemset(m->v, 0, sizeof(float) * m->P) != cudaSuccess)
        return TSM_ERR_LAUNCH;
    m->step = 0;
    return TSM_OK;
}

tsm_status tsm_mlp_get_params(const tsm_mlp* m, float* host) {
    if (!m || !host) return TSM_ERR_INVALID_VALUE;
    return cudaMemcpy(host, m->params, sizeof(float) * m->P, cudaMemcpyDeviceToHost) == cudaSuccess
               ? TSM_OK
               : TSM_ERR_LAUNCH;
}

tsm_status tsm_mlp_get_grads(const tsm_mlp* m, float* host) {
    if (!m || !host) return TSM_ERR_INVALID_VALUE;
    return cudaMemcpy(host, m->grads, sizeof(float) * m->P, cudaMemcpyDeviceToHost) == cudaSuccess
               ? TSM_OK
               : TSM_ERR_LAUNCH;
}

tsm_status tsm_mlp_forward(tsm_mlp* m, const float* X, int n, float* y, tsm_stream_t stream) {
    if (!m || !X || !y || n < 1 || n > m->max_batch) return TSM_ERR_INVALID_VALUE;
    mlp::k_forward<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(m->params, m->D, m->H, X, n, y, nullptr);
    return cudaGetLastError() == cudaSuccess ? TSM_OK : TSM_ERR_LAUNCH;
}

tsm_status tsm_mlp_backward(tsm_mlp* m, const float* X, const float* t, int n, float* loss,
                            tsm_stream_t stream) {
    if (!m || !X || !t || !loss || n < 1 || n > m->max_batch) return TSM_ERR_INVALID_VALUE;
    cudaStream_t s = (cudaStream_t)stream;
    // predictions go to the per-sample error buffer first, then become errors
    float* y = m->sqerr;
    mlp::k_forward<<<(n + 127) / 128, 128, 0, s>>>(m->params, m->D, m->H, X, n, y, m->act);
    mlp::k_backward_samples<<<(n + 127) / 128, 128, 0, s>>>(m->params, m->D, m->H, t, n, y, m->act, m->dtmp,
                                                            m->sqerr);
    mlp::k_backward_params<<<(m->P + 127) / 128, 128, 0, s>>>(m->D, m->H, X, n, m->act, m->dtmp, m->grads);
    mlp::k_loss<<<1, 1, 0, s>>>(m->sqerr, n, loss);
    return cudaGetLastError() == cudaSuccess ? TSM_OK : TSM_ERR_LAUNCH;
}

tsm_status tsm_mlp_adam(tsm_mlp* m, float lr, float beta1, float beta2, float eps, tsm_stream_t stream) {
    if (!m || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
        !(eps > 0.0f))
        return TSM_ERR_INVALID_VALUE;
    m->step += 1;
    const float c1 = 1.0f - powf(beta1, (float)m->step);
    const float c2 = 1.0f - powf(beta2, (float)m->step);
    mlp::k_adam<<<(m->P + 127) / 128, 128, 0, (cudaStream_t)stream>>>(m->params, m->grads, m->m, m->v, m->P, lr,
                                                                      beta1, beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? TSM_OK : TSM_ERR_LAUNCH;
}

}  // extern "C"
