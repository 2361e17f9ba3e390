// Learned impedance network of the step's trace_mode 3 (Sec. III-B: K(q) and D(q) may be
// learned instead of set by the heuristic): evaluation at a batch of feature vectors, and its
// fit by full-batch Adam on the mean squared error against a target (the log ratio of the
// exact diagonal impedance to the heuristic's, captured by the step kernel).
//
// The network is tiny (4 inputs, 8 tanh units, 49 parameters), so the fit is a plain
// reduction: every thread accumulates the loss and all 49 gradient terms of its samples in
// registers, each CTA reduces them with warp shuffles into one partial row, and a single CTA
// sums the rows in a fixed order and applies the Adam update.  Results do not depend on
// scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "cf_internal.cuh"

using namespace cf;

namespace {

constexpr int kFitBlocks = 304;                 // 2 CTAs per SM of a 152-SM part
constexpr int kFitThreads = 256;
constexpr int kRow = kImpParams + 1;            // 49 gradient terms + the summed squared error

struct Net {
  float W1[kImpHidden][kImpIn], b1[kImpHidden], w2[kImpHidden], b2;
};

__device__ __forceinline__ void load_net(const float* __restrict__ th, Net& n) {
#pragma unroll
  for (int h = 0; h < kImpHidden; ++h) {
#pragma unroll
    for (int i = 0; i < kImpIn; ++i) n.W1[h][i] = __ldg(th + h * kImpIn + i);
    n.b1[h] = __ldg(th + kImpHidden * kImpIn + h);
    n.w2[h] = __ldg(th + kImpHidden * kImpIn + kImpHidden + h);
  }
  n.b2 = __ldg(th + kImpParams - 1);
}

__global__ void __launch_bounds__(kFitThreads) impnet_eval_kernel(const float* __restrict__ th,
                                                                  const float* __restrict__ x, int n,
                                                                  float* __restrict__ g) {
  Net net;
  load_net(th, net);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 xi = reinterpret_cast<const float4*>(x)[i];
    const float xv[kImpIn] = {xi.x, xi.y, xi.z, xi.w};
    float out = net.b2;
#pragma unroll
    for (int h = 0; h < kImpHidden; ++h) {
      float a = net.b1[h];
#pragma unroll
      for (int k = 0; k < kImpIn; ++k) a = fmaf(net.W1[h][k], xv[k], a);
      out = fmaf(net.w2[h], tanhf(a), out);
    }
    g[i] = out;
  }
}

// Per-CTA partial sums of sum_i (g(x_i) - y_i)^2 and of its gradient 2 (g - y) dg/dtheta.
__global__ void __launch_bounds__(kFitThreads) impnet_grad_kernel(const float* __restrict__ th,
                                                                  const float* __restrict__ x,
                                                                  const float* __restrict__ y, int n,
                                                                  float* __restrict__ partial) {
  Net net;
  load_net(th, net);
  float acc[kRow];
#pragma unroll
  for (int p = 0; p < kRow; ++p) acc[p] = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 xi = reinterpret_cast<const float4*>(x)[i];
    const float xv[kImpIn] = {xi.x, xi.y, xi.z, xi.w};
    float hid[kImpHidden];
    float g = net.b2;
#pragma unroll
    for (int h = 0; h < kImpHidden; ++h) {
      float a = net.b1[h];
#pragma unroll
      for (int k = 0; k < kImpIn; ++k) a = fmaf(net.W1[h][k], xv[k], a);
      hid[h] = tanhf(a);
      g = fmaf(net.w2[h], hid[h], g);
    }
    const float e = g - __ldg(y + i);
    const float dg = 2.f * e;
    acc[kImpParams] = fmaf(e, e, acc[kImpParams]);
    acc[kImpParams - 1] += dg;
#pragma unroll
    for (int h = 0; h < kImpHidden; ++h) {
      acc[kImpHidden * kImpIn + kImpHidden + h] = fmaf(dg, hid[h], acc[kImpHidden * kImpIn + kImpHidden + h]);
      const float da = dg * net.w2[h] * (1.f - hid[h] * hid[h]);
      acc[kImpHidden * kImpIn + h] += da;
#pragma unroll
      for (int k = 0; k < kImpIn; ++k) acc[h * kImpIn + k] = fmaf(da, xv[k], acc[h * kImpIn + k]);
    }
  }
  __shared__ float red[kFitThreads / 32][kRow];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < kRow; ++p) {
    float v = acc[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][p] = v;
  }
  __syncthreads();
  if (threadIdx.x < kRow) {
    float v = 0.f;
    for (int w = 0; w < kFitThreads / 32; ++w) v += red[w][threadIdx.x];
    partial[blockIdx.x * kRow + threadIdx.x] = v;
  }
}

// Sum the CTA rows in order; write the mean loss and gradient, and (adam != 0) take one Adam
// step (Kingma and Ba 2015: beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected moments) at step
// number t (1-based).
__global__ void impnet_update_kernel(float* __restrict__ th, float* __restrict__ mom, const float* __restrict__ partial,
                                     int n, int adam, int t, float lr, float* __restrict__ grad_out,
                                     float* __restrict__ loss_out) {
  const int p = threadIdx.x;
  if (p >= kRow) return;
  float s = 0.f;
  for (int b = 0; b < kFitBlocks; ++b) s += partial[b * kRow + p];
  const float inv_n = 1.f / (float)n;
  if (p == kImpParams) {
    if (loss_out) *loss_out = s * inv_n;
    return;
  }
  const float g = s * inv_n;
  if (grad_out) grad_out[p] = g;
  if (!adam) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float m = b1 * mom[p] + (1.f - b1) * g;
  const float v = b2 * mom[kImpParams + p] + (1.f - b2) * g * g;
  mom[p] = m;
  mom[kImpParams + p] = v;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  th[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

cf_status ifail(cf_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

cf_status launched(const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CF_OK : ifail(CF_ERR_CUDA, what);
}

}  // namespace

extern "C" size_t cf_impnet_state_floats(void) { return 2 * kImpParams + (size_t)kFitBlocks * kRow; }

extern "C" cf_status cf_impnet_eval(const float* theta, const float* x, int32_t n, float* g, void* stream) {
  if (n == 0) return CF_OK;
  if (!theta || !x || !g || n < 0 || !aligned16(x))
    return ifail(CF_ERR_INVALID_ARGUMENT, "impnet eval: null pointer, negative count or x not 16-byte aligned");
  const int grid = std::min((n + kFitThreads - 1) / kFitThreads, 8 * kFitBlocks);
  impnet_eval_kernel<<<grid, kFitThreads, 0, (cudaStream_t)stream>>>(theta, x, n, g);
  return launched("impnet eval launch");
}

extern "C" cf_status cf_impnet_loss_grad(const float* theta, const float* x, const float* y, int32_t n, float* state,
                                         float* grad, float* loss, void* stream) {
  if (!theta || !x || !y || !state || n < 1 || !aligned16(x))
    return ifail(CF_ERR_INVALID_ARGUMENT, "impnet loss: null pointer, empty data or x not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  float* partial = state + 2 * kImpParams;
  impnet_grad_kernel<<<kFitBlocks, kFitThreads, 0, s>>>(theta, x, y, n, partial);
  impnet_update_kernel<<<1, 64, 0, s>>>(nullptr, state, partial, n, 0, 0, 0.f, grad, loss);
  return launched("impnet loss launch");
}

extern "C" cf_status cf_impnet_fit(float* theta, float* state, int32_t step0, const float* x, const float* y,
                                   int32_t n, int32_t iters, float lr, float* losses, void* stream) {
  if (!theta || !state || !x || !y || n < 1 || iters < 0 || step0 < 0 || !(lr > 0.f) || !aligned16(x))
    return ifail(CF_ERR_INVALID_ARGUMENT, "impnet fit: null pointer, empty data, bad step or rate, or x not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  float* partial = state + 2 * kImpParams;
  for (int it = 0; it < iters; ++it) {
    impnet_grad_kernel<<<kFitBlocks, kFitThreads, 0, s>>>(theta, x, y, n, partial);
    impnet_update_kernel<<<1, 64, 0, s>>>(theta, state, partial, n, 1, step0 + it + 1, lr, nullptr,
                                          losses ? losses + it : nullptr);
  }
  return launched("impnet fit launch");
}
