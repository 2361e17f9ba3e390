// Sampling MPC (MPPI, Williams et al. 2017, as used in Sec. V of ComFree-Sim) around the batched
// step: control sampling (optionally mixed with a learned Gaussian proposal), the exponential
// cost weighting and weighted-mean update, state broadcast to the rollout worlds, and the
// proposal's input features.  Random normals are inputs (drawn by the caller).
#include <cuda_runtime.h>

#include <cmath>

#include "comfree.h"
#include "cf_internal.cuh"

namespace cf {

// sample k < n_prop from the proposal N(pm, exp(pls)^2), the rest from N(mean, sigma^2);
// clip to [-limit, limit]; write the rollout controls ctrl[h][k * nu + j] and samples[k][h][j]
__global__ void mppi_sample_kernel(int N, int H, int nu, const float* mean, const float* eps, float sigma, float limit,
                                   const float* pm, const float* pls, int n_prop, float* ctrl, float* samples) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int total = N * H * nu;
  if (i >= total) return;
  int k = i / (H * nu), r = i % (H * nu), h = r / nu, j = r % nu;
  float u;
  if (k < n_prop) u = pm[r] + expf(pls[r]) * eps[i];
  else u = mean[r] + sigma * eps[i];
  u = fminf(fmaxf(u, -limit), limit);
  samples[i] = u;
  ctrl[(size_t)h * N * nu + (size_t)k * nu + j] = u;
}

// weights w_k = exp(-(J_k - min J) / lambda); mean <- sum_k w_k U_k / sum_k w_k.
// A rollout whose cost is not finite (its state blew up) gets weight 0; if no rollout is finite
// the mean is left unchanged.  One CTA; stats = (min cost, mean finite cost, effective sample size).
__global__ void mppi_update_kernel(int N, int H, int nu, const float* cost, const float* samples, float lambda,
                                   float* mean, float* stats) {
  extern __shared__ float w[];
  __shared__ float red[32];
  __shared__ float s_min, s_sum, s_mean, s_sq;
  const int tid = threadIdx.x, nt = blockDim.x;
  float mn = 3.0e38f, sm = 0.f;
  for (int k = tid; k < N; k += nt) {
    float c = cost[k];
    if (isfinite(c)) {
      mn = fminf(mn, c);
      sm += c;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
    sm += __shfl_down_sync(0xffffffffu, sm, o);
  }
  if ((tid & 31) == 0) { red[tid >> 5] = mn; w[N + (tid >> 5)] = sm; }
  __syncthreads();
  if (tid == 0) {
    float a = red[0], b = w[N];
    for (int i = 1; i < (nt + 31) / 32; ++i) { a = fminf(a, red[i]); b += w[N + i]; }
    s_min = a;
    s_mean = b / N;
  }
  __syncthreads();
  float ws = 0.f, wq = 0.f;
  for (int k = tid; k < N; k += nt) {
    float c = cost[k];
    float e = isfinite(c) ? expf(-(c - s_min) / lambda) : 0.f;
    w[k] = e;
    ws += e;
    wq += e * e;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ws += __shfl_down_sync(0xffffffffu, ws, o);
    wq += __shfl_down_sync(0xffffffffu, wq, o);
  }
  __syncthreads();
  if ((tid & 31) == 0) { red[tid >> 5] = ws; w[N + (tid >> 5)] = wq; }
  __syncthreads();
  if (tid == 0) {
    float a = 0.f, b = 0.f;
    for (int i = 0; i < (nt + 31) / 32; ++i) { a += red[i]; b += w[N + i]; }
    s_sum = a;
    s_sq = b;
  }
  __syncthreads();
  const int M = H * nu;
  if (s_sum > 0.f && isfinite(s_sum)) {
    for (int r = tid; r < M; r += nt) {
      float acc = 0.f;
      for (int k = 0; k < N; ++k) acc = fmaf(w[k], samples[(size_t)k * M + r], acc);
      mean[r] = acc / s_sum;
    }
  }
  if (tid == 0 && stats) {
    stats[0] = s_min;
    stats[1] = s_mean;
    stats[2] = s_sum * s_sum / s_sq;
  }
}

// copy one world's state (q0[nq], v0[nv]) into W back-to-back worlds
__global__ void broadcast_kernel(const float* q0, const float* v0, int nq, int nv, int W, float* q, float* v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < W * nq) q[i] = q0[i % nq];
  if (i < W * nv) v[i] = v0[i % nv];
}

// shift a plan by one step (the receding horizon): mean[h] <- mean[h + 1], last step kept
__global__ void shift_kernel(int H, int nu, float* mean) {
  int j = threadIdx.x;
  if (j >= nu) return;
  for (int h = 0; h + 1 < H; ++h) mean[h * nu + j] = mean[(h + 1) * nu + j];
}

// out = base + scale * delta (the learned warm start: the proposal's correction of a plan)
__global__ void blend_kernel(int n, const float* base, const float* delta, float scale, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = fmaf(scale, delta[i], base[i]);
}

}  // namespace cf

using namespace cf;

static cf_status mp_fail(cf_status s, const char* m) {
  set_last_error(m);
  return s;
}

extern "C" cf_status cf_mppi_sample(int32_t N, int32_t H, int32_t nu, const float* mean, const float* noise, float sigma,
                                    float limit, const float* prop_mean, const float* prop_logstd, int32_t n_prop,
                                    float* ctrl, float* samples, void* stream) {
  if (N < 1 || H < 1 || nu < 1 || !mean || !noise || !ctrl || !samples || n_prop < 0 || n_prop > N ||
      (n_prop > 0 && (!prop_mean || !prop_logstd)) || !(limit > 0.f) || !(sigma >= 0.f))
    return mp_fail(CF_ERR_INVALID_ARGUMENT, "bad mppi sample arguments");
  int total = N * H * nu;
  mppi_sample_kernel<<<(total + 255) / 256, 256, 0, (cudaStream_t)stream>>>(N, H, nu, mean, noise, sigma, limit,
                                                                            prop_mean, prop_logstd, n_prop, ctrl,
                                                                            samples);
  return cudaGetLastError() == cudaSuccess ? CF_OK : mp_fail(CF_ERR_CUDA, "mppi sample launch");
}

extern "C" cf_status cf_mppi_update(int32_t N, int32_t H, int32_t nu, const float* costs, const float* samples,
                                    float lambda, float* mean, float* stats, void* stream) {
  if (N < 1 || N > 16384 || H < 1 || nu < 1 || !costs || !samples || !mean || !(lambda > 0.f))
    return mp_fail(CF_ERR_INVALID_ARGUMENT, "bad mppi update arguments (1 <= N <= 16384)");
  size_t smem = sizeof(float) * (N + 32);
  mppi_update_kernel<<<1, 1024, smem, (cudaStream_t)stream>>>(N, H, nu, costs, samples, lambda, mean, stats);
  return cudaGetLastError() == cudaSuccess ? CF_OK : mp_fail(CF_ERR_CUDA, "mppi update launch");
}

extern "C" cf_status cf_mppi_shift(int32_t H, int32_t nu, float* mean, void* stream) {
  if (H < 1 || nu < 1 || nu > 1024 || !mean) return mp_fail(CF_ERR_INVALID_ARGUMENT, "bad shift arguments");
  shift_kernel<<<1, nu, 0, (cudaStream_t)stream>>>(H, nu, mean);
  return cudaGetLastError() == cudaSuccess ? CF_OK : mp_fail(CF_ERR_CUDA, "shift launch");
}

extern "C" cf_status cf_mppi_blend(int32_t n, const float* base, const float* delta, float scale, float* out,
                                   void* stream) {
  if (n < 0 || (n > 0 && (!base || !delta || !out))) return mp_fail(CF_ERR_INVALID_ARGUMENT, "bad blend arguments");
  if (n == 0) return CF_OK;
  blend_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, base, delta, scale, out);
  return cudaGetLastError() == cudaSuccess ? CF_OK : mp_fail(CF_ERR_CUDA, "blend launch");
}

extern "C" cf_status cf_broadcast_state(const float* q0, const float* v0, int32_t nq, int32_t nv, int32_t W, float* q,
                                        float* v, void* stream) {
  if (!q0 || !v0 || !q || !v || nq < 1 || nv < 1 || W < 1) return mp_fail(CF_ERR_INVALID_ARGUMENT, "bad broadcast");
  int n = W * (nq > nv ? nq : nv);
  broadcast_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(q0, v0, nq, nv, W, q, v);
  return cudaGetLastError() == cudaSuccess ? CF_OK : mp_fail(CF_ERR_CUDA, "broadcast launch");
}

namespace cf {
__global__ void concat_kernel(const float* a, int na, const float* b, int nb, float bscale, const float* c, int nc,
                              float clamp, float* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float x;
  if (i < na) x = a[i];
  else if (i < na + nb) x = bscale * b[i - na];
  else if (i < na + nb + nc) x = c[i - na - nb];
  else return;
  out[i] = fminf(fmaxf(x, -clamp), clamp);
}
}  // namespace cf

extern "C" cf_status cf_mppi_features(const float* q, int32_t nq, const float* v, int32_t nv, float v_scale,
                                      const float* goal, int32_t ngoal, float clamp, float* out, void* stream) {
  if (!q || !v || !out || nq < 0 || nv < 0 || ngoal < 0 || (ngoal && !goal) || !(clamp > 0.f))
    return mp_fail(CF_ERR_INVALID_ARGUMENT, "bad feature arguments");
  int n = nq + nv + ngoal;
  concat_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(q, nq, v, nv, v_scale, goal, ngoal, clamp, out);
  return cudaGetLastError() == cudaSuccess ? CF_OK : mp_fail(CF_ERR_CUDA, "features launch");
}
