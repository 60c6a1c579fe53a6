// proposal.cu -- the learned proposer: a small 1-D convolutional network that
// reads the incoherent dedispersed power (trial DMs as channels, filterbank
// samples as time) and scores every (DM, time) cell, so the coherent path can
// be run only where the score is high.  Training and inference run entirely
// in the kernels below (FP32 storage and arithmetic):
//   conv forward (+ bias, + ReLU), backward to the input (the forward kernel
//   on flipped, transposed weights), backward to weights and biases, class-
//   weighted BCE with logits, Adam, per-DM z-score normalisation and window
//   maxima for the proposal mask.
//
//   h1 = relu(conv(x, W1, b1, K1/2)), h2 = relu(conv(h1, W2, b2, K2/2)),
//   z = conv(h2, W3, b3, 0) with K3 = 1;
//   conv(x, W, b, pad)[b, o, t] = b[o] + sum_{i,k} W[o, i, k] x[b, i, t + k - pad].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/chirp_gb300.h"
#include "internal.h"

namespace {

constexpr int kOT = 32;    // output channels per CTA
constexpr int kTT = 64;    // time samples per CTA
constexpr int kIC = 16;    // input channels per staged chunk
constexpr int kKMAX = 15;  // largest kernel width
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_conv_fwd(const float* __restrict__ in,
                                                       const float* __restrict__ W,
                                                       const float* __restrict__ bias,
                                                       float* __restrict__ out, int C, int O,
                                                       int T, int K, int pad, int relu) {
  __shared__ float s_in[kIC][kTT + kKMAX - 1];
  __shared__ float s_w[kOT][kIC * kKMAX];
  const int b = blockIdx.z, o0 = blockIdx.y * kOT, t0 = blockIdx.x * kTT;
  const int ol = threadIdx.x / 8, tg = threadIdx.x % 8;
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; j++) acc[j] = 0.f;
  const int span = kTT + K - 1;
  for (int i0 = 0; i0 < C; i0 += kIC) {
    for (int idx = threadIdx.x; idx < kIC * span; idx += kThreads) {
      const int ii = idx / span, tt = idx % span;
      const int ci = i0 + ii, t = t0 + tt - pad;
      s_in[ii][tt] = (ci < C && t >= 0 && t < T) ? in[((long long)b * C + ci) * T + t] : 0.f;
    }
    for (int idx = threadIdx.x; idx < kOT * kIC * K; idx += kThreads) {
      const int oo = idx / (kIC * K), r = idx % (kIC * K);
      const int ii = r / K, kk = r % K;
      const int o = o0 + oo, ci = i0 + ii;
      s_w[oo][ii * K + kk] = (o < O && ci < C) ? W[((long long)o * C + ci) * K + kk] : 0.f;
    }
    __syncthreads();
    for (int ii = 0; ii < kIC; ii++)
      for (int kk = 0; kk < K; kk++) {
        const float w = s_w[ol][ii * K + kk];
#pragma unroll
        for (int j = 0; j < 8; j++) acc[j] = fmaf(w, s_in[ii][tg + 8 * j + kk], acc[j]);
      }
    __syncthreads();
  }
  const int o = o0 + ol;
  if (o >= O) return;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int t = t0 + tg + 8 * j;
    if (t >= T) continue;
    float v = acc[j] + (bias ? bias[o] : 0.f);
    if (relu) v = fmaxf(v, 0.f);
    out[((long long)b * O + o) * T + t] = v;
  }
}

// Wt[i][o][K-1-k] = W[o][i][k]: the backward-to-input convolution is a forward
// convolution of the output gradient with these weights and pad K-1-pad.
__global__ void k_flip_transpose(const float* __restrict__ W, float* __restrict__ Wt, int O,
                                 int C, int K) {
  const long long n = (long long)O * C * K;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(idx / ((long long)C * K)), r = (int)(idx % ((long long)C * K));
    const int i = r / K, k = r % K;
    Wt[((long long)i * O + o) * K + (K - 1 - k)] = W[idx];
  }
}

// g *= (h > 0): gradient through a ReLU whose output is h
__global__ void k_relu_bwd(float* __restrict__ g, const float* __restrict__ h, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!(h[i] > 0.f)) g[i] = 0.f;
}

// dW[o][i][k] = sum_{b,t} g[b][o][t] x[b][i][t + k - pad]; one CTA per (i, o)
__global__ void __launch_bounds__(kThreads) k_conv_wgrad(const float* __restrict__ x,
                                                         const float* __restrict__ g,
                                                         float* __restrict__ dW, int B, int C,
                                                         int O, int T, int K, int pad) {
  __shared__ float red[kKMAX][kThreads];
  const int i = blockIdx.x, o = blockIdx.y;
  float acc[kKMAX];
#pragma unroll
  for (int k = 0; k < kKMAX; k++) acc[k] = 0.f;
  const long long n = (long long)B * T;
  for (long long bt = threadIdx.x; bt < n; bt += kThreads) {
    const int b = (int)(bt / T), t = (int)(bt % T);
    const float gv = g[((long long)b * O + o) * T + t];
    const float* xr = x + ((long long)b * C + i) * T;
#pragma unroll
    for (int k = 0; k < kKMAX; k++) {
      const int tt = t + k - pad;
      if (k < K && tt >= 0 && tt < T) acc[k] = fmaf(gv, xr[tt], acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < kKMAX; k++) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < K; k++) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < K) dW[((long long)o * C + i) * K + threadIdx.x] = red[threadIdx.x][0];
}

// db[o] = sum_{b,t} g[b][o][t]; one CTA per o
__global__ void __launch_bounds__(kThreads) k_bias_grad(const float* __restrict__ g,
                                                        float* __restrict__ db, int B, int O,
                                                        int T) {
  __shared__ float red[kThreads];
  const int o = blockIdx.x;
  float acc = 0.f;
  const long long n = (long long)B * T;
  for (long long bt = threadIdx.x; bt < n; bt += kThreads) {
    const int b = (int)(bt / T), t = (int)(bt % T);
    acc += g[((long long)b * O + o) * T + t];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[o] = red[0];
}

__device__ __forceinline__ float softplusf(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

// class-weighted BCE with logits: dz and per-CTA partial losses (mean over n)
__global__ void __launch_bounds__(kThreads) k_bce(const float* __restrict__ z,
                                                  const float* __restrict__ y,
                                                  float* __restrict__ dz, long long n, float pw,
                                                  float* __restrict__ partial) {
  __shared__ float red[kThreads];
  float acc = 0.f;
  const float inv = 1.0f / (float)n;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (long long)gridDim.x * kThreads) {
    const float zi = z[i], yi = y[i];
    acc += pw * yi * softplusf(-zi) + (1.f - yi) * softplusf(zi);
    const float s = 1.f / (1.f + expf(-zi));
    dz[i] = (-pw * yi * (1.f - s) + (1.f - yi) * s) * inv;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0] * inv;
}

__global__ void k_sum(const float* __restrict__ partial, int n, float* __restrict__ out) {
  __shared__ float red[kThreads];
  float acc = 0.f;
  for (int i = threadIdx.x; i < n; i += kThreads) acc += partial[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Adam: m, v moments; theta -= lr (m / c1) / (sqrt(v / c2) + eps), c = 1 - beta^step
__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, long long n, float lr,
                       float b1, float b2, float c1, float c2, float eps) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// x[d][t] = (D[d][t] - mean_d) / std_d over the DM's nonzero (valid) samples;
// samples outside the valid range stay 0.  One CTA per DM row.
__global__ void __launch_bounds__(kThreads) k_zscore(const float* __restrict__ D,
                                                     float* __restrict__ x, long long T) {
  __shared__ double red[3][kThreads];
  const float* row = D + (long long)blockIdx.x * T;
  float* xo = x + (long long)blockIdx.x * T;
  double s0 = 0, s1 = 0, s2 = 0;
  for (long long t = threadIdx.x; t < T; t += kThreads) {
    const double v = row[t];
    if (v != 0.0) {
      s0 += 1.0;
      s1 += v;
      s2 += v * v;
    }
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  red[2][threadIdx.x] = s2;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 3; q++) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  const double n = red[0][0];
  const double mean = n > 0 ? red[1][0] / n : 0.0;
  const double var = n > 1 ? (red[2][0] - n * mean * mean) / (n - 1) : 0.0;
  const float inv = var > 0 ? (float)(1.0 / sqrt(var)) : 0.f;
  for (long long t = threadIdx.x; t < T; t += kThreads) {
    const float v = row[t];
    xo[t] = v != 0.f ? (float)((v - mean) * inv) : 0.f;
  }
}

// mask[d][w] = 1 if max over window w of the logits exceeds thr
__global__ void k_windows(const float* __restrict__ z, long long T, int win, long long n_win,
                          float thr, int* __restrict__ mask) {
  const int d = blockIdx.y;
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < n_win;
       w += (long long)gridDim.x * blockDim.x) {
    float mx = -INFINITY;
    for (int i = 0; i < win; i++) {
      const long long t = w * win + i;
      if (t < T) mx = fmaxf(mx, z[(long long)d * T + t]);
    }
    mask[(long long)d * n_win + w] = mx > thr ? 1 : 0;
  }
}

unsigned grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

struct chirp_propnet {
  int C, H, K1, K2, maxB, T;
  cudaStream_t st;
  long long n_par;
  long long off[6], len[6];  // W1 b1 W2 b2 W3 b3 inside the flat vectors
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  float *h1 = nullptr, *h2 = nullptr, *z = nullptr;        // activations
  float *gz = nullptr, *g2 = nullptr, *g1 = nullptr;       // gradients
  float *wt = nullptr;                                     // flipped weights
  float *partial = nullptr, *loss = nullptr;
  long long step = 0;
};

namespace {
thread_local char p_err[256];
int perr(int code, const char* msg) {
  snprintf(p_err, sizeof p_err, "%s", msg);
  return chirp_report_error(code, p_err);
}
#define PK(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return perr(CHIRP_ECUDA, cudaGetErrorString(e_));        \
  } while (0)

void free_net(chirp_propnet* n) {
  for (float* p : {n->theta, n->grad, n->m, n->v, n->h1, n->h2, n->z, n->gz, n->g2, n->g1, n->wt,
                   n->partial, n->loss})
    cudaFree(p);
}

int conv(chirp_propnet* n, const float* in, const float* W, const float* b, float* out, int B,
         int C, int O, int K, int pad, int relu) {
  dim3 grid((n->T + kTT - 1) / kTT, (O + kOT - 1) / kOT, B);
  k_conv_fwd<<<grid, kThreads, 0, n->st>>>(in, W, b, out, C, O, n->T, K, pad, relu);
  PK(cudaGetLastError());
  return CHIRP_OK;
}

// grad of a conv layer: weights, bias and (if gin) input
int conv_bwd(chirp_propnet* n, const float* x, const float* W, const float* g, float* dW,
             float* db, float* gin, int B, int C, int O, int K, int pad) {
  k_conv_wgrad<<<dim3(C, O), kThreads, 0, n->st>>>(x, g, dW, B, C, O, n->T, K, pad);
  PK(cudaGetLastError());
  k_bias_grad<<<O, kThreads, 0, n->st>>>(g, db, B, O, n->T);
  PK(cudaGetLastError());
  if (gin) {
    k_flip_transpose<<<grid_for((long long)O * C * K), kThreads, 0, n->st>>>(W, n->wt, O, C, K);
    PK(cudaGetLastError());
    int rc = conv(n, g, n->wt, nullptr, gin, B, O, C, K, K - 1 - pad, 0);
    if (rc) return rc;
  }
  return CHIRP_OK;
}

int forward(chirp_propnet* n, const float* x, int B, float* z) {
  const float* th = n->theta;
  int rc = conv(n, x, th + n->off[0], th + n->off[1], n->h1, B, n->C, n->H, n->K1, n->K1 / 2, 1);
  if (!rc) rc = conv(n, n->h1, th + n->off[2], th + n->off[3], n->h2, B, n->H, n->H, n->K2, n->K2 / 2, 1);
  if (!rc) rc = conv(n, n->h2, th + n->off[4], th + n->off[5], z, B, n->H, n->C, 1, 0, 0);
  return rc;
}

int backward(chirp_propnet* n, const float* x, const float* y, int B, float pw, float* loss_host) {
  int rc = forward(n, x, B, n->z);
  if (rc) return rc;
  const long long nz = (long long)B * n->C * n->T;
  const unsigned gb = grid_for(nz);
  k_bce<<<gb, kThreads, 0, n->st>>>(n->z, y, n->gz, nz, pw, n->partial);
  PK(cudaGetLastError());
  k_sum<<<1, kThreads, 0, n->st>>>(n->partial, (int)gb, n->loss);
  PK(cudaGetLastError());
  float* gr = n->grad;
  const float* th = n->theta;
  rc = conv_bwd(n, n->h2, th + n->off[4], n->gz, gr + n->off[4], gr + n->off[5], n->g2, B, n->H,
                n->C, 1, 0);
  if (rc) return rc;
  const long long nh = (long long)B * n->H * n->T;
  k_relu_bwd<<<grid_for(nh), kThreads, 0, n->st>>>(n->g2, n->h2, nh);
  PK(cudaGetLastError());
  rc = conv_bwd(n, n->h1, th + n->off[2], n->g2, gr + n->off[2], gr + n->off[3], n->g1, B, n->H,
                n->H, n->K2, n->K2 / 2);
  if (rc) return rc;
  k_relu_bwd<<<grid_for(nh), kThreads, 0, n->st>>>(n->g1, n->h1, nh);
  PK(cudaGetLastError());
  rc = conv_bwd(n, x, th + n->off[0], n->g1, gr + n->off[0], gr + n->off[1], nullptr, B, n->C,
                n->H, n->K1, n->K1 / 2);
  if (rc) return rc;
  if (loss_host) {
    PK(cudaMemcpyAsync(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->st));
    PK(cudaStreamSynchronize(n->st));
  }
  return CHIRP_OK;
}

int check_batch(const chirp_propnet* n, int B) {
  if (B < 1 || B > n->maxB) return perr(CHIRP_EINVAL, "batch must be in 1..max_batch");
  return CHIRP_OK;
}

}  // namespace

extern "C" {

int chirp_propnet_create(chirp_propnet** out, int n_dm, int hidden, int k1, int k2, int max_batch,
                         int n_time, void* stream) {
  if (!out) return perr(CHIRP_EINVAL, "net pointer is NULL");
  *out = nullptr;
  if (n_dm < 1 || hidden < 1 || max_batch < 1 || n_time < 1)
    return perr(CHIRP_EINVAL, "propnet sizes must be positive");
  if (k1 < 1 || k1 > kKMAX || k2 < 1 || k2 > kKMAX || !(k1 & 1) || !(k2 & 1))
    return perr(CHIRP_EINVAL, "kernel widths must be odd and <= 15");
  chirp_propnet* n = new (std::nothrow) chirp_propnet();
  if (!n) return perr(CHIRP_ENOMEM, "host allocation failed");
  n->C = n_dm;
  n->H = hidden;
  n->K1 = k1;
  n->K2 = k2;
  n->maxB = max_batch;
  n->T = n_time;
  n->st = (cudaStream_t)stream;
  n->len[0] = (long long)hidden * n_dm * k1;
  n->len[1] = hidden;
  n->len[2] = (long long)hidden * hidden * k2;
  n->len[3] = hidden;
  n->len[4] = (long long)n_dm * hidden;
  n->len[5] = n_dm;
  long long o = 0;
  for (int i = 0; i < 6; i++) {
    n->off[i] = o;
    o += n->len[i];
  }
  n->n_par = o;
  const long long nh = (long long)max_batch * hidden * n_time;
  const long long nc = (long long)max_batch * n_dm * n_time;
  const long long nw = std::max({n->len[0], n->len[2], n->len[4]});
  struct A { float** p; long long n; } allocs[] = {
      {&n->theta, o}, {&n->grad, o}, {&n->m, o}, {&n->v, o}, {&n->h1, nh}, {&n->h2, nh},
      {&n->z, nc}, {&n->gz, nc}, {&n->g2, nh}, {&n->g1, nh}, {&n->wt, nw}, {&n->partial, 4096},
      {&n->loss, 1}};
  for (auto& a : allocs) {
    if (cudaMalloc((void**)a.p, (size_t)a.n * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      free_net(n);
      delete n;
      return perr(CHIRP_ENOMEM, "device allocation for the proposal net failed");
    }
  }
  cudaMemsetAsync(n->theta, 0, (size_t)o * sizeof(float), n->st);
  cudaMemsetAsync(n->m, 0, (size_t)o * sizeof(float), n->st);
  cudaMemsetAsync(n->v, 0, (size_t)o * sizeof(float), n->st);
  *out = n;
  return CHIRP_OK;
}

void chirp_propnet_destroy(chirp_propnet* n) {
  if (!n) return;
  cudaStreamSynchronize(n->st);
  free_net(n);
  delete n;
}

long long chirp_propnet_param_count(const chirp_propnet* n) { return n ? n->n_par : -1; }

int chirp_propnet_set_params(chirp_propnet* n, const float* params) {
  if (!n || !params) return perr(CHIRP_EINVAL, "NULL argument");
  PK(cudaMemcpyAsync(n->theta, params, (size_t)n->n_par * sizeof(float), cudaMemcpyHostToDevice,
                     n->st));
  PK(cudaMemsetAsync(n->m, 0, (size_t)n->n_par * sizeof(float), n->st));
  PK(cudaMemsetAsync(n->v, 0, (size_t)n->n_par * sizeof(float), n->st));
  PK(cudaStreamSynchronize(n->st));
  n->step = 0;
  return CHIRP_OK;
}

int chirp_propnet_get_params(const chirp_propnet* n, float* params) {
  if (!n || !params) return perr(CHIRP_EINVAL, "NULL argument");
  PK(cudaMemcpyAsync(params, n->theta, (size_t)n->n_par * sizeof(float), cudaMemcpyDeviceToHost,
                     n->st));
  PK(cudaStreamSynchronize(n->st));
  return CHIRP_OK;
}

int chirp_propnet_get_state(const chirp_propnet* n, float* params, float* m, float* v,
                            long long* step) {
  if (!n || !params || !m || !v || !step) return perr(CHIRP_EINVAL, "NULL argument");
  const size_t bytes = (size_t)n->n_par * sizeof(float);
  PK(cudaMemcpyAsync(params, n->theta, bytes, cudaMemcpyDeviceToHost, n->st));
  PK(cudaMemcpyAsync(m, n->m, bytes, cudaMemcpyDeviceToHost, n->st));
  PK(cudaMemcpyAsync(v, n->v, bytes, cudaMemcpyDeviceToHost, n->st));
  PK(cudaStreamSynchronize(n->st));
  *step = n->step;
  return CHIRP_OK;
}

int chirp_propnet_set_state(chirp_propnet* n, const float* params, const float* m,
                            const float* v, long long step) {
  if (!n || !params || !m || !v) return perr(CHIRP_EINVAL, "NULL argument");
  if (step < 0) return perr(CHIRP_EINVAL, "negative Adam step");
  const size_t bytes = (size_t)n->n_par * sizeof(float);
  PK(cudaMemcpyAsync(n->theta, params, bytes, cudaMemcpyHostToDevice, n->st));
  PK(cudaMemcpyAsync(n->m, m, bytes, cudaMemcpyHostToDevice, n->st));
  PK(cudaMemcpyAsync(n->v, v, bytes, cudaMemcpyHostToDevice, n->st));
  PK(cudaStreamSynchronize(n->st));
  n->step = step;
  return CHIRP_OK;
}

int chirp_propnet_get_grads(const chirp_propnet* n, float* grads) {
  if (!n || !grads) return perr(CHIRP_EINVAL, "NULL argument");
  PK(cudaMemcpyAsync(grads, n->grad, (size_t)n->n_par * sizeof(float), cudaMemcpyDeviceToHost,
                     n->st));
  PK(cudaStreamSynchronize(n->st));
  return CHIRP_OK;
}

int chirp_propnet_forward(chirp_propnet* n, const float* x, int batch, float* logits) {
  if (!n || !x || !logits) return perr(CHIRP_EINVAL, "NULL argument");
  int rc = check_batch(n, batch);
  return rc ? rc : forward(n, x, batch, logits);
}

int chirp_propnet_backward(chirp_propnet* n, const float* x, const float* y, int batch,
                           float pos_weight, float* loss_host) {
  if (!n || !x || !y) return perr(CHIRP_EINVAL, "NULL argument");
  int rc = check_batch(n, batch);
  return rc ? rc : backward(n, x, y, batch, pos_weight, loss_host);
}

int chirp_propnet_train_step(chirp_propnet* n, const float* x, const float* y, int batch,
                             float pos_weight, float lr, float* loss_host) {
  int rc = chirp_propnet_backward(n, x, y, batch, pos_weight, nullptr);
  if (rc) return rc;
  n->step++;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)n->step));
  const float c2 = (float)(1.0 - std::pow(0.999, (double)n->step));
  k_adam<<<grid_for(n->n_par), kThreads, 0, n->st>>>(n->theta, n->grad, n->m, n->v, n->n_par, lr,
                                                     b1, b2, c1, c2, eps);
  PK(cudaGetLastError());
  if (loss_host) {
    PK(cudaMemcpyAsync(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->st));
    PK(cudaStreamSynchronize(n->st));
  }
  return CHIRP_OK;
}

int chirp_propnet_normalize(const float* D, int n_dm, long long n_time, float* x, void* stream) {
  if (!D || !x || n_dm < 1 || n_time < 1) return perr(CHIRP_EINVAL, "bad argument");
  k_zscore<<<n_dm, kThreads, 0, (cudaStream_t)stream>>>(D, x, n_time);
  PK(cudaGetLastError());
  return CHIRP_OK;
}

int chirp_propose_windows(const float* logits, int n_dm, long long n_time, int win, float thr,
                          int* mask, void* stream) {
  if (!logits || !mask || n_dm < 1 || n_time < 1 || win < 1) return perr(CHIRP_EINVAL, "bad argument");
  const long long n_win = (n_time + win - 1) / win;
  dim3 grid(grid_for(n_win), n_dm);
  k_windows<<<grid, kThreads, 0, (cudaStream_t)stream>>>(logits, n_time, win, n_win, thr, mask);
  PK(cudaGetLastError());
  return CHIRP_OK;
}

}  // extern "C"
