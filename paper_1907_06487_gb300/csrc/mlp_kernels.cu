// The RACE-parameter predictor: a 16 -> 64 -> 64 -> 3 perceptron (ReLU,
// linear output) trained with mean squared error and Adam, all in FP32 on
// the device, plus the host feature extractor.
//
// Parameters are one packed FP32 array:
//   W1[64][16] b1[64] W2[64][64] b2[64] W3[3][64] b3[3]   (row-major, out x in)
// Activations of a batch (caller-owned scratch, race_mlp_act_size floats):
//   z1[B][64] h1[B][64] z2[B][64] h2[B][64] y[B][3]
// The network is small (5,312 multiply-adds per sample): one thread per
// output element, latency-bound, no tensor cores.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "race_internal.h"

namespace race_mlp {

constexpr int kIn = 16, kH = 64, kOut = 3;
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kOut * kH, kParams = ob3 + kOut;

// y[b][o] = act(sum_i W[o][i] x[b][i] + bias[o]); also stores the pre-activation
__global__ void k_dense(int batch, int in, int out, const float* __restrict__ W, const float* __restrict__ bias,
                        const float* __restrict__ x, float* __restrict__ z, float* __restrict__ h, int relu) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<int64_t>(batch) * out) return;
    const int b = static_cast<int>(t / out), o = static_cast<int>(t % out);
    float acc = bias[o];
    for (int i = 0; i < in; ++i) acc += W[o * in + i] * x[static_cast<int64_t>(b) * in + i];
    if (z) z[t] = acc;
    h[t] = relu ? fmaxf(acc, 0.f) : acc;
}

// dz[b][o] = dh[b][o] * (z > 0) for ReLU layers (in place on dh)
__global__ void k_relu_back(int64_t count, const float* __restrict__ z, float* __restrict__ dh) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < count && z[t] <= 0.f) dh[t] = 0.f;
}

// dW[o][i] = sum_b dz[b][o] x[b][i];  db[o] = sum_b dz[b][o]
__global__ void k_dense_grad_w(int batch, int in, int out, const float* __restrict__ dz, const float* __restrict__ x,
                               float* __restrict__ dW, float* __restrict__ db) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < out * in) {
        const int o = t / in, i = t % in;
        float acc = 0.f;
        for (int b = 0; b < batch; ++b) acc += dz[static_cast<int64_t>(b) * out + o] * x[static_cast<int64_t>(b) * in + i];
        dW[t] = acc;
    } else if (t < out * in + out) {
        const int o = t - out * in;
        float acc = 0.f;
        for (int b = 0; b < batch; ++b) acc += dz[static_cast<int64_t>(b) * out + o];
        db[o] = acc;
    }
}

// dx[b][i] = sum_o W[o][i] dz[b][o]
__global__ void k_dense_grad_x(int batch, int in, int out, const float* __restrict__ W, const float* __restrict__ dz,
                               float* __restrict__ dx) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<int64_t>(batch) * in) return;
    const int b = static_cast<int>(t / in), i = static_cast<int>(t % in);
    float acc = 0.f;
    for (int o = 0; o < out; ++o) acc += W[o * in + i] * dz[static_cast<int64_t>(b) * out + o];
    dx[t] = acc;
}

// loss gradient of L = 1/(2B) sum_b sum_k w_k (y - t)^2; per-sample loss terms
__global__ void k_mse_grad(int batch, const float* __restrict__ y, const float* __restrict__ target,
                           const float* __restrict__ wk, float* __restrict__ dy, float* __restrict__ lossterm) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= batch * kOut) return;
    const float d = y[t] - target[t], w = wk[t % kOut];
    dy[t] = w * d / static_cast<float>(batch);
    lossterm[t] = 0.5f * w * d * d / static_cast<float>(batch);
}

__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float beta1, float beta2, float eps, float c1, float c2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gi = g[t];
    const float mi = beta1 * m[t] + (1.f - beta1) * gi;
    const float vi = beta2 * v[t] + (1.f - beta2) * gi * gi;
    m[t] = mi;
    v[t] = vi;
    p[t] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline int blocks(int64_t n) { return static_cast<int>((n + 255) / 256); }

}  // namespace race_mlp

using namespace race_mlp;

extern "C" {

int32_t race_mlp_param_count(void) { return kParams; }

int64_t race_mlp_act_size(int32_t batch) { return static_cast<int64_t>(batch) * (4 * kH + kOut); }

int race_mlp_forward(const float* params_d, int32_t batch, const float* x_d, float* act_d, float* y_d, void* stream) {
    if (!params_d || !x_d || !act_d || batch < 1) {
        race_set_detail("race_mlp_forward: bad argument");
        return RACE_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* z1 = act_d;
    float* h1 = z1 + static_cast<int64_t>(batch) * kH;
    float* z2 = h1 + static_cast<int64_t>(batch) * kH;
    float* h2 = z2 + static_cast<int64_t>(batch) * kH;
    float* y = h2 + static_cast<int64_t>(batch) * kH;
    k_dense<<<blocks(static_cast<int64_t>(batch) * kH), 256, 0, st>>>(batch, kIn, kH, params_d + oW1, params_d + ob1,
                                                                      x_d, z1, h1, 1);
    k_dense<<<blocks(static_cast<int64_t>(batch) * kH), 256, 0, st>>>(batch, kH, kH, params_d + oW2, params_d + ob2,
                                                                      h1, z2, h2, 1);
    k_dense<<<blocks(static_cast<int64_t>(batch) * kOut), 256, 0, st>>>(batch, kH, kOut, params_d + oW3,
                                                                        params_d + ob3, h2, nullptr, y, 0);
    if (y_d) cudaMemcpyAsync(y_d, y, sizeof(float) * batch * kOut, cudaMemcpyDeviceToDevice, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        race_set_detail(std::string("race_mlp_forward: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}

int race_mlp_backward(const float* params_d, int32_t batch, const float* x_d, float* act_d, const float* target_d,
                      const float* out_weight_d, float* grad_d, float* work_d, float* loss_terms_d, void* stream) {
    if (!params_d || !x_d || !act_d || !target_d || !out_weight_d || !grad_d || !work_d || !loss_terms_d ||
        batch < 1) {
        race_set_detail("race_mlp_backward: bad argument");
        return RACE_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t B = batch;
    float* z1 = act_d;
    float* h1 = z1 + B * kH;
    float* z2 = h1 + B * kH;
    float* h2 = z2 + B * kH;
    float* y = h2 + B * kH;
    float* dy = work_d;              // B x 3
    float* dh2 = dy + B * kOut;      // B x 64
    float* dh1 = dh2 + B * kH;       // B x 64
    k_mse_grad<<<blocks(B * kOut), 256, 0, st>>>(batch, y, target_d, out_weight_d, dy, loss_terms_d);
    k_dense_grad_w<<<blocks(kOut * kH + kOut), 256, 0, st>>>(batch, kH, kOut, dy, h2, grad_d + oW3, grad_d + ob3);
    k_dense_grad_x<<<blocks(B * kH), 256, 0, st>>>(batch, kH, kOut, params_d + oW3, dy, dh2);
    k_relu_back<<<blocks(B * kH), 256, 0, st>>>(B * kH, z2, dh2);
    k_dense_grad_w<<<blocks(kH * kH + kH), 256, 0, st>>>(batch, kH, kH, dh2, h1, grad_d + oW2, grad_d + ob2);
    k_dense_grad_x<<<blocks(B * kH), 256, 0, st>>>(batch, kH, kH, params_d + oW2, dh2, dh1);
    k_relu_back<<<blocks(B * kH), 256, 0, st>>>(B * kH, z1, dh1);
    k_dense_grad_w<<<blocks(kH * kIn + kH), 256, 0, st>>>(batch, kIn, kH, dh1, x_d, grad_d + oW1, grad_d + ob1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        race_set_detail(std::string("race_mlp_backward: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}

int64_t race_mlp_work_size(int32_t batch) { return static_cast<int64_t>(batch) * (kOut + 2 * kH); }

int race_mlp_adam(float* params_d, const float* grad_d, float* m_d, float* v_d, float lr, float beta1, float beta2,
                  float eps, int32_t step, void* stream) {
    if (!params_d || !grad_d || !m_d || !v_d || step < 1) {
        race_set_detail("race_mlp_adam: bad argument");
        return RACE_ERR_INVALID;
    }
    const float c1 = 1.f - std::pow(beta1, static_cast<float>(step));
    const float c2 = 1.f - std::pow(beta2, static_cast<float>(step));
    k_adam<<<blocks(kParams), 256, 0, static_cast<cudaStream_t>(stream)>>>(kParams, params_d, grad_d, m_d, v_d, lr,
                                                                           beta1, beta2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        race_set_detail(std::string("race_mlp_adam: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}

}  // extern "C"
