// incoherent.cu -- the cheap antenna-incoherent search that proposes where
// the coherent path should look: power-beam filterbank (Sec. 2.4.1 power
// beams, channelised as in Sec. 2.3.1) and incoherent shift-and-sum
// dedispersion over a DM grid (Sec. 2.3.1).
//
//   S[c][tau] = sum_a sum_{i < n_int} |X_{a, tau n_int + i}[k(c)]|^2,
//     X_{a,b} = DFT of samples [b L, (b+1) L) of antenna a (L = n_chan),
//     k(c) = (c + L/2) mod L (ascending frequency f_c = f0 + (c - L/2) B / L);
//   D[d][t] = sum_c S[c][t + s_c(d)], s_c = floor(k DM (f_c^-2 - f0^-2) / t_fb + 1/2),
//     t_fb = L n_int / B, valid for t in [-min s, T - max s), zero elsewhere.
#include <cuda_runtime.h>

#include "fft.cuh"
#include "internal.h"

namespace chirp {

// In-place forward FFTs of length L over rows of every antenna's series:
// row r of antenna q is data[q seq_stride + r L .. + L).
template <int L>
__global__ void __launch_bounds__(256) k_fb_fft(float2* __restrict__ data, long long seq_stride,
                                                long long n_rows, TwiddlePtrs twp) {
  constexpr int C = 4096 / L;
  constexpr int T = L / 16;
  __shared__ float2 sm[FftTile<L, C>::SLOTS];
  const Twiddles tw{twp.coarse, twp.fine, twp.stage};
  const int jt = threadIdx.x % T, s = threadIdx.x / T;
  const long long r = (long long)blockIdx.x * C + s;
  const bool act = r < n_rows;
  float2* p = data + (long long)blockIdx.y * seq_stride + r * L;
  float2 v[16];
#pragma unroll
  for (int k = 0; k < 16; k++) v[k] = act ? p[jt + k * T] : make_float2(0.f, 0.f);
  fft_core<L, C, true, false>(v, sm, s, jt, tw);
  if (!act) return;
#pragma unroll
  for (int k = 0; k < 16; k++) p[jt + k * T] = v[k];
}

// S[c][tau]: one thread per (channel, filterbank sample); two-level FP32 sum
__global__ void k_fb_power(const float2* __restrict__ X, long long seq_stride, int n_ant, int L,
                           int n_int, long long T_fb, float* __restrict__ S) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L) return;
  const int k = (c + L / 2) % L;
  for (long long tau = blockIdx.y; tau < T_fb; tau += gridDim.y) {
    float total = 0.f;
    for (int a = 0; a < n_ant; a++) {
      const float2* base = X + (long long)a * seq_stride + (tau * n_int) * L + k;
      float part = 0.f;
      for (int i = 0; i < n_int; i++) {
        const float2 z = base[(long long)i * L];
        part = fmaf(z.x, z.x, fmaf(z.y, z.y, part));
      }
      total += part;
    }
    S[(long long)c * T_fb + tau] = total;
  }
}

// D[d][t] = sum_c S[c][t + shift[d][c]] over the DM's valid range, else 0
__global__ void k_incoherent(const float* __restrict__ S, int n_chan, long long T_fb,
                             const int* __restrict__ shift, float* __restrict__ D) {
  extern __shared__ int ssh[];  // shifts of this DM
  const int d = blockIdx.y;
  int s_min = 0, s_max = 0;
  for (int c = threadIdx.x; c < n_chan; c += blockDim.x) ssh[c] = shift[(long long)d * n_chan + c];
  __syncthreads();
  for (int c = 0; c < n_chan; c++) {
    s_min = c == 0 || ssh[c] < s_min ? ssh[c] : s_min;
    s_max = c == 0 || ssh[c] > s_max ? ssh[c] : s_max;
  }
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < T_fb;
       t += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    if (t >= -s_min && t < T_fb - s_max)
      for (int c = 0; c < n_chan; c++) acc += S[(long long)c * T_fb + t + ssh[c]];
    D[(long long)d * T_fb + t] = acc;
  }
}

__global__ void k_unpack_ci8(const char2* __restrict__ x, const float* __restrict__ scale,
                             long long n_samp, long long total, float2* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float sc = scale ? scale[i / n_samp] : 1.0f;
    const char2 z = x[i];
    y[i] = make_float2(__fmul_rn((float)z.x, sc), __fmul_rn((float)z.y, sc));
  }
}

cudaError_t launch_unpack_ci8(const void* x, const float* scale, int n_ant, long long n_samp,
                              float2* y, cudaStream_t st) {
  const long long total = (long long)n_ant * n_samp;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_unpack_ci8<<<(unsigned)blocks, 256, 0, st>>>((const char2*)x, scale, n_samp, total, y);
  return cudaGetLastError();
}

cudaError_t launch_incoherent(float2* scratch, long long seq_stride, int n_ant, int n_chan,
                              int n_int, long long T_fb, const int* shift, int n_dm, float* S,
                              float* D, TwiddlePtrs tw, cudaStream_t st) {
  if (T_fb <= 0) return cudaSuccess;
  const long long n_rows = T_fb * n_int;
  const int C = 4096 / n_chan;
  dim3 g1((unsigned)((n_rows + C - 1) / C), (unsigned)n_ant);
  switch (n_chan) {
#define X(L) \
  case L: k_fb_fft<L><<<g1, 256, 0, st>>>(scratch, seq_stride, n_rows, tw); break;
    X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)
#undef X
    default: return cudaErrorInvalidValue;
  }
  const int tb = n_chan < 256 ? n_chan : 256;
  dim3 g2((n_chan + tb - 1) / tb, (unsigned)(T_fb < 65535 ? T_fb : 65535));
  k_fb_power<<<g2, tb, 0, st>>>(scratch, seq_stride, n_ant, n_chan, n_int, T_fb, S);
  long long bx = (T_fb + 255) / 256;
  if (bx > 1024) bx = 1024;
  dim3 g3((unsigned)bx, (unsigned)n_dm);
  k_incoherent<<<g3, 256, (size_t)n_chan * sizeof(int), st>>>(S, n_chan, T_fb, shift, D);
  return cudaGetLastError();
}

}  // namespace chirp
