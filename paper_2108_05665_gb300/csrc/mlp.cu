// Learned cost model of plans: a small fully connected network (ReLU hidden
// layers, one linear output) mapping plan features to log2 of the measured
// step time, with hand-written forward, backward and Adam kernels.
//
// Parameters live in one device buffer, layer by layer: W_l (out x in,
// row-major) then b_l (out).  Gradients and the two Adam moments use the same
// layout in their own buffers.  Inputs are normalised on the device with the
// stored per-feature mean and scale before the first layer.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <random>
#include <string>
#include <vector>

#include "plan.h"
#include "xeb.h"

struct xeb_mlp_s {
    int n_in = 0, n_hidden = 0, n_layers = 0;   // n_layers hidden layers + one output layer
    std::vector<int> dims;                        // n_in, H, ..., H, 1
    std::vector<size_t> w_off, b_off;             // float offsets of W_l, b_l
    size_t n_params = 0;
    float* params = nullptr;                      // device
    float* grads = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    float* norm = nullptr;                        // device: mean[n_in], scale[n_in]
    float* act = nullptr;                         // device activations of the last batch
    float* dact = nullptr;
    int cap = 0;                                  // batch capacity of act / dact
    int64_t step = 0;
};

namespace {

xeb_status mfail(xeb_status s, const std::string& m) {
    xebp::set_last_error(m);
    return s;
}
#define XEB_MCUDA(x)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (x);                                                                 \
        if (e_ != cudaSuccess) return mfail(XEB_ECUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
    } while (0)

constexpr int kT = 16;   // tile edge of the small GEMM kernels

// Y[b][o] = act(sum_i X[b][i] W[o][i] + bias[o]); X is n x in, Y n x out.
// relu = 1: ReLU; the pre-activation is not kept (ReLU's derivative is read
// from Y itself).
__global__ void k_dense_fwd(const float* __restrict__ X, const float* __restrict__ W, const float* __restrict__ bias,
                            float* __restrict__ Y, int n, int in, int out, int relu) {
    __shared__ float xs[kT][kT + 1], ws[kT][kT + 1];
    const int o = blockIdx.x * kT + threadIdx.x, b = blockIdx.y * kT + threadIdx.y;
    float acc = 0.f;
    for (int i0 = 0; i0 < in; i0 += kT) {
        const int ix = i0 + threadIdx.x, iw = i0 + threadIdx.y;
        xs[threadIdx.y][threadIdx.x] = (b < n && ix < in) ? X[size_t(b) * in + ix] : 0.f;
        ws[threadIdx.x][threadIdx.y] = (blockIdx.x * kT + threadIdx.x < out && iw < in)
                                           ? W[size_t(blockIdx.x * kT + threadIdx.x) * in + iw] : 0.f;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kT; ++t) acc = fmaf(xs[threadIdx.y][t], ws[threadIdx.x][t], acc);
        __syncthreads();
    }
    if (b < n && o < out) {
        const float v = acc + bias[o];
        Y[size_t(b) * out + o] = relu ? fmaxf(v, 0.f) : v;
    }
}

// dX[b][i] = sum_o dY[b][o] W[o][i], then masked by ReLU'(X) when mask = 1
// (X is the layer's input, itself a ReLU output).
__global__ void k_dense_bwd_x(const float* __restrict__ dY, const float* __restrict__ W, const float* __restrict__ X,
                              float* __restrict__ dX, int n, int in, int out, int mask) {
    __shared__ float ds[kT][kT + 1], ws[kT][kT + 1];
    const int i = blockIdx.x * kT + threadIdx.x, b = blockIdx.y * kT + threadIdx.y;
    float acc = 0.f;
    for (int o0 = 0; o0 < out; o0 += kT) {
        const int od = o0 + threadIdx.x, ow = o0 + threadIdx.y;
        ds[threadIdx.y][threadIdx.x] = (b < n && od < out) ? dY[size_t(b) * out + od] : 0.f;
        ws[threadIdx.y][threadIdx.x] = (ow < out && i < in) ? W[size_t(ow) * in + i] : 0.f;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kT; ++t) acc = fmaf(ds[threadIdx.y][t], ws[t][threadIdx.x], acc);
        __syncthreads();
    }
    if (b < n && i < in) dX[size_t(b) * in + i] = (mask && X[size_t(b) * in + i] <= 0.f) ? 0.f : acc;
}

// dW[o][i] = sum_b dY[b][o] X[b][i] / scale; db[o] = sum_b dY[b][o] / scale
__global__ void k_dense_bwd_w(const float* __restrict__ dY, const float* __restrict__ X, float* __restrict__ dW,
                              float* __restrict__ db, int n, int in, int out, float scale) {
    __shared__ float ds[kT][kT + 1], xs[kT][kT + 1];
    const int i = blockIdx.x * kT + threadIdx.x, o = blockIdx.y * kT + threadIdx.y;
    float acc = 0.f, accb = 0.f;
    for (int b0 = 0; b0 < n; b0 += kT) {
        const int bd = b0 + threadIdx.x, bx = b0 + threadIdx.y;
        ds[threadIdx.y][threadIdx.x] = (bd < n && blockIdx.y * kT + threadIdx.y < out)
                                           ? dY[size_t(bd) * out + blockIdx.y * kT + threadIdx.y] : 0.f;
        xs[threadIdx.y][threadIdx.x] = (bx < n && i < in) ? X[size_t(bx) * in + i] : 0.f;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kT; ++t) {
            acc = fmaf(ds[threadIdx.y][t], xs[t][threadIdx.x], acc);
            accb += ds[threadIdx.y][t];
        }
        __syncthreads();
    }
    if (o < out && i < in) dW[size_t(o) * in + i] = acc / scale;
    if (o < out && blockIdx.x == 0 && threadIdx.x == 0) db[o] = accb / scale;
}

// normalised input: Xn[b][i] = (X[b][i] - mean[i]) * scale[i]
__global__ void k_normalise(const float* __restrict__ X, const float* __restrict__ norm, float* __restrict__ Xn, int n,
                            int in) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * in; e += gridDim.x * blockDim.x) {
        const int i = e % in;
        Xn[e] = (X[e] - norm[i]) * norm[in + i];
    }
}

// dY of the squared-error loss L = mean_b (y_b - t_b)^2 (the 2/n factor goes
// into the weight gradient's scale); partial sums of L per block
__global__ void k_loss_grad(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy, int n,
                            float* __restrict__ loss) {
    __shared__ float s[256];
    float acc = 0.f;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        const float d = y[b] - t[b];
        dy[b] = 2.f * d;
        acc += d * d;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) atomicAdd(loss, s[0] / float(n));
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1, float* __restrict__ m2,
                       size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x) {
        const float gi = g[e];
        const float a = b1 * m1[e] + (1.f - b1) * gi;
        const float v = b2 * m2[e] + (1.f - b2) * gi * gi;
        m1[e] = a;
        m2[e] = v;
        p[e] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

size_t act_floats(const xeb_mlp_s* m, int n) {
    size_t s = 0;
    for (int d : m->dims) s += size_t(n) * size_t(d);
    return s;
}

xeb_status ensure_cap(xeb_mlp_s* m, int n) {
    if (n <= m->cap) return XEB_OK;
    if (m->act) cudaFree(m->act);
    if (m->dact) cudaFree(m->dact);
    m->act = m->dact = nullptr;
    XEB_MCUDA(cudaMalloc(&m->act, act_floats(m, n) * 4));
    XEB_MCUDA(cudaMalloc(&m->dact, act_floats(m, n) * 4));
    m->cap = n;
    return XEB_OK;
}

// activations of layer l (l = 0: normalised input) for a batch of n
float* act_of(xeb_mlp_s* m, float* base, int n, int l) {
    size_t s = 0;
    for (int j = 0; j < l; ++j) s += size_t(n) * size_t(m->dims[j]);
    return base + s;
}

xeb_status forward(xeb_mlp_s* m, const float* X, int n, cudaStream_t st) {
    xeb_status s = ensure_cap(m, n);
    if (s != XEB_OK) return s;
    k_normalise<<<(n * m->n_in + 255) / 256, 256, 0, st>>>(X, m->norm, act_of(m, m->act, n, 0), n, m->n_in);
    const int L = int(m->dims.size()) - 1;
    for (int l = 0; l < L; ++l) {
        const int in = m->dims[l], out = m->dims[l + 1];
        dim3 grid((out + kT - 1) / kT, (n + kT - 1) / kT), block(kT, kT);
        k_dense_fwd<<<grid, block, 0, st>>>(act_of(m, m->act, n, l), m->params + m->w_off[l], m->params + m->b_off[l],
                                            act_of(m, m->act, n, l + 1), n, in, out, l < L - 1);
    }
    XEB_MCUDA(cudaGetLastError());
    return XEB_OK;
}

// gradients of the mean squared error into m->grads (after forward)
xeb_status backward(xeb_mlp_s* m, const float* t, int n, float* loss, cudaStream_t st) {
    const int L = int(m->dims.size()) - 1;
    float* dy = act_of(m, m->dact, n, L);
    k_loss_grad<<<(n + 255) / 256 < 64 ? (n + 255) / 256 : 64, 256, 0, st>>>(act_of(m, m->act, n, L), t, dy, n, loss);
    for (int l = L - 1; l >= 0; --l) {
        const int in = m->dims[l], out = m->dims[l + 1];
        dim3 gw((in + kT - 1) / kT, (out + kT - 1) / kT), block(kT, kT);
        k_dense_bwd_w<<<gw, block, 0, st>>>(act_of(m, m->dact, n, l + 1), act_of(m, m->act, n, l),
                                             m->grads + m->w_off[l], m->grads + m->b_off[l], n, in, out, float(n));
        if (l > 0) {
            dim3 gx((in + kT - 1) / kT, (n + kT - 1) / kT);
            k_dense_bwd_x<<<gx, block, 0, st>>>(act_of(m, m->dact, n, l + 1), m->params + m->w_off[l],
                                                 act_of(m, m->act, n, l), act_of(m, m->dact, n, l), n, in, out, 1);
        }
    }
    XEB_MCUDA(cudaGetLastError());
    return XEB_OK;
}

}  // namespace

extern "C" {

xeb_status xeb_mlp_create(int n_in, int n_hidden, int n_layers, uint64_t seed, xeb_mlp_s** out) {
    if (!out) return mfail(XEB_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_in < 1 || n_in > 1024 || n_hidden < 1 || n_hidden > 1024 || n_layers < 0 || n_layers > 8)
        return mfail(XEB_EINVAL, "mlp sizes out of range");
    std::unique_ptr<xeb_mlp_s> m(new xeb_mlp_s());
    m->n_in = n_in;
    m->n_hidden = n_hidden;
    m->n_layers = n_layers;
    m->dims.push_back(n_in);
    for (int l = 0; l < n_layers; ++l) m->dims.push_back(n_hidden);
    m->dims.push_back(1);
    size_t off = 0;
    for (size_t l = 0; l + 1 < m->dims.size(); ++l) {
        m->w_off.push_back(off);
        off += size_t(m->dims[l]) * m->dims[l + 1];
        m->b_off.push_back(off);
        off += size_t(m->dims[l + 1]);
    }
    m->n_params = off;
    // He-uniform initial weights (ReLU layers), zero biases
    std::vector<float> h(off, 0.f);
    std::mt19937_64 rng(seed);
    for (size_t l = 0; l + 1 < m->dims.size(); ++l) {
        const float lim = std::sqrt(6.f / float(m->dims[l]));
        std::uniform_real_distribution<float> u(-lim, lim);
        for (size_t e = 0; e < size_t(m->dims[l]) * m->dims[l + 1]; ++e) h[m->w_off[l] + e] = u(rng);
    }
    std::vector<float> norm(2 * size_t(n_in), 0.f);
    for (int i = 0; i < n_in; ++i) norm[n_in + i] = 1.f;
    XEB_MCUDA(cudaMalloc(&m->params, off * 4));
    XEB_MCUDA(cudaMalloc(&m->grads, off * 4));
    XEB_MCUDA(cudaMalloc(&m->m1, off * 4));
    XEB_MCUDA(cudaMalloc(&m->m2, off * 4));
    XEB_MCUDA(cudaMalloc(&m->norm, norm.size() * 4));
    XEB_MCUDA(cudaMemcpy(m->params, h.data(), off * 4, cudaMemcpyHostToDevice));
    XEB_MCUDA(cudaMemset(m->grads, 0, off * 4));
    XEB_MCUDA(cudaMemset(m->m1, 0, off * 4));
    XEB_MCUDA(cudaMemset(m->m2, 0, off * 4));
    XEB_MCUDA(cudaMemcpy(m->norm, norm.data(), norm.size() * 4, cudaMemcpyHostToDevice));
    *out = m.release();
    return XEB_OK;
}

void xeb_mlp_destroy(xeb_mlp_s* m) {
    if (!m) return;
    cudaFree(m->params);
    cudaFree(m->grads);
    cudaFree(m->m1);
    cudaFree(m->m2);
    cudaFree(m->norm);
    cudaFree(m->act);
    cudaFree(m->dact);
    delete m;
}

size_t xeb_mlp_n_params(xeb_mlp_s* m) { return m ? m->n_params : 0; }

xeb_status xeb_mlp_weights(xeb_mlp_s* m, float* host, int set) {
    if (!m || !host) return mfail(XEB_EINVAL, "NULL argument");
    if (set) {
        XEB_MCUDA(cudaMemcpy(m->params, host, m->n_params * 4, cudaMemcpyHostToDevice));
        XEB_MCUDA(cudaMemset(m->m1, 0, m->n_params * 4));
        XEB_MCUDA(cudaMemset(m->m2, 0, m->n_params * 4));
        m->step = 0;
    } else {
        XEB_MCUDA(cudaMemcpy(host, m->params, m->n_params * 4, cudaMemcpyDeviceToHost));
    }
    return XEB_OK;
}

xeb_status xeb_mlp_set_norm(xeb_mlp_s* m, const float* mean, const float* scale) {
    if (!m || !mean || !scale) return mfail(XEB_EINVAL, "NULL argument");
    std::vector<float> h(2 * size_t(m->n_in));
    std::memcpy(h.data(), mean, size_t(m->n_in) * 4);
    std::memcpy(h.data() + m->n_in, scale, size_t(m->n_in) * 4);
    XEB_MCUDA(cudaMemcpy(m->norm, h.data(), h.size() * 4, cudaMemcpyHostToDevice));
    return XEB_OK;
}

xeb_status xeb_mlp_forward(xeb_mlp_s* m, const float* x_dev, int n, float* y_dev, uintptr_t stream) {
    if (!m || !x_dev || !y_dev || n < 1) return mfail(XEB_EINVAL, "bad mlp forward arguments");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    xeb_status s = forward(m, x_dev, n, st);
    if (s != XEB_OK) return s;
    XEB_MCUDA(cudaMemcpyAsync(y_dev, act_of(m, m->act, n, int(m->dims.size()) - 1), size_t(n) * 4,
                              cudaMemcpyDeviceToDevice, st));
    return XEB_OK;
}

xeb_status xeb_mlp_gradients(xeb_mlp_s* m, const float* x_dev, const float* t_dev, int n, float* grad_host,
                             float* loss_host, uintptr_t stream) {
    if (!m || !x_dev || !t_dev || n < 1) return mfail(XEB_EINVAL, "bad mlp gradient arguments");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    xeb_status s = forward(m, x_dev, n, st);
    if (s != XEB_OK) return s;
    float* dl = nullptr;
    XEB_MCUDA(cudaMalloc(&dl, 4));
    XEB_MCUDA(cudaMemsetAsync(dl, 0, 4, st));
    s = backward(m, t_dev, n, dl, st);
    if (s == XEB_OK && grad_host)
        if (cudaMemcpyAsync(grad_host, m->grads, m->n_params * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            s = mfail(XEB_ECUDA, "gradient copy");
    if (s == XEB_OK && loss_host)
        if (cudaMemcpyAsync(loss_host, dl, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) s = mfail(XEB_ECUDA, "loss copy");
    cudaStreamSynchronize(st);
    cudaFree(dl);
    return s;
}

xeb_status xeb_mlp_train_step(xeb_mlp_s* m, const float* x_dev, const float* t_dev, int n, float lr, float* loss_dev,
                              uintptr_t stream) {
    if (!m || !x_dev || !t_dev || n < 1) return mfail(XEB_EINVAL, "bad mlp training arguments");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    xeb_status s = forward(m, x_dev, n, st);
    if (s == XEB_OK) s = backward(m, t_dev, n, loss_dev, st);
    if (s != XEB_OK) return s;
    ++m->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, float(m->step)), c2 = 1.f - std::pow(b2, float(m->step));
    k_adam<<<int((m->n_params + 255) / 256 < 1024 ? (m->n_params + 255) / 256 : 1024), 256, 0, st>>>(
        m->params, m->grads, m->m1, m->m2, m->n_params, lr, b1, b2, 1e-8f, c1, c2);
    XEB_MCUDA(cudaGetLastError());
    return XEB_OK;
}

}  // extern "C"
