// backends.cu -- CUDA-core back-ends that consume dedispersed voltages.
//
// Chirpolator (correlate): per dump m the zero-lag products
//   V_pq = sum_{t in dump} y_p(t) y_q(t)^*   (p <= q, autos included),
// the pair mixing x_pq = s_p s_q^* of Eq. xpq integrated and dumped.
// Chimageator, plain FP32 form: per dump and pixel
//   P = sum_{t in dump} |sum_a W_pa y_a(t)|^2
// (direct beamforming, Sec. 2.4.2, detected and integrated).
//
// Both accumulate in FP32 with a two-level sum (a short inner run, then the
// running total) so that a 4096-sample dump stays within the 1e-5 relative
// budget of the FP32 path.
#include <cuda_runtime.h>

#include "internal.h"

namespace chirp {

// ------------------------------------------------------------------ correlate
// One CTA per dump.  The M x M product is cut into 4 x 4 antenna tiles; each
// thread owns one tile on or above the diagonal and a slice of the dump's
// samples, so every staged sample value it loads feeds four complex MACs.
// Slices are summed through shared memory at the end.
constexpr int kCorrThreads = 256;
constexpr int kCorrTile = 4;

__global__ void __launch_bounds__(kCorrThreads) k_correlate(const float2* __restrict__ y,
                                                             long long n_samp, int M, int L,
                                                             long long first, long long last,
                                                             float2* __restrict__ vis,
                                                             int chunk) {
  extern __shared__ float2 sy[];  // [Mp][chunk] staged voltages, Mp = M rounded up to 4
  const long long m = blockIdx.x;
  const int n_pair = M * (M + 1) / 2;
  float2* out = vis + m * n_pair;
  if (m < first || m > last) {
    for (int i = threadIdx.x; i < n_pair; i += blockDim.x) out[i] = make_float2(0.f, 0.f);
    return;
  }
  const int nt = (M + kCorrTile - 1) / kCorrTile;          // tiles per side
  const int n_tiles = nt * (nt + 1) / 2;                   // tiles with ti <= tj
  const int n_slice = kCorrThreads / n_tiles;              // >= 1 for M <= 84
  const int tile = threadIdx.x % n_tiles, slice = threadIdx.x / n_tiles;
  const bool worker = slice < n_slice;
  int ti = 0, rem = tile;
  while (rem >= nt - ti) {
    rem -= nt - ti;
    ti++;
  }
  const int tj = ti + rem;
  const int Mp = nt * kCorrTile;
  float2 acc[kCorrTile][kCorrTile];
#pragma unroll
  for (int a = 0; a < kCorrTile; a++)
#pragma unroll
    for (int b = 0; b < kCorrTile; b++) acc[a][b] = make_float2(0.f, 0.f);
  const long long t0 = m * L;
  for (int c0 = 0; c0 < L; c0 += chunk) {
    const int len = (L - c0) < chunk ? (L - c0) : chunk;
    __syncthreads();
    for (int i = threadIdx.x; i < Mp * len; i += blockDim.x) {
      int a = i / len, t = i % len;
      sy[a * chunk + t] = a < M ? y[(long long)a * n_samp + t0 + c0 + t] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (worker) {
      float2 part[kCorrTile][kCorrTile];
#pragma unroll
      for (int a = 0; a < kCorrTile; a++)
#pragma unroll
        for (int b = 0; b < kCorrTile; b++) part[a][b] = make_float2(0.f, 0.f);
      for (int t = slice; t < len; t += n_slice) {
        float2 u[kCorrTile], w[kCorrTile];
#pragma unroll
        for (int a = 0; a < kCorrTile; a++) {
          u[a] = sy[(ti * kCorrTile + a) * chunk + t];
          w[a] = sy[(tj * kCorrTile + a) * chunk + t];
        }
#pragma unroll
        for (int a = 0; a < kCorrTile; a++)
#pragma unroll
          for (int b = 0; b < kCorrTile; b++) {  // u_a * conj(w_b)
            part[a][b].x = fmaf(u[a].x, w[b].x, fmaf(u[a].y, w[b].y, part[a][b].x));
            part[a][b].y = fmaf(u[a].y, w[b].x, fmaf(-u[a].x, w[b].y, part[a][b].y));
          }
      }
#pragma unroll
      for (int a = 0; a < kCorrTile; a++)
#pragma unroll
        for (int b = 0; b < kCorrTile; b++) {
          acc[a][b].x += part[a][b].x;
          acc[a][b].y += part[a][b].y;
        }
    }
  }
  // reduce the slices: red[slice][tile][4][4] in the staging buffer
  __syncthreads();
  float2* red = sy;
  if (worker)
#pragma unroll
    for (int a = 0; a < kCorrTile; a++)
#pragma unroll
      for (int b = 0; b < kCorrTile; b++)
        red[((slice * n_tiles + tile) * kCorrTile + a) * kCorrTile + b] = acc[a][b];
  __syncthreads();
  for (int k = threadIdx.x; k < n_pair; k += blockDim.x) {
    int p = 0, r2 = k;  // row-major upper-triangle index k -> (p, q)
    while (r2 >= M - p) {
      r2 -= M - p;
      p++;
    }
    const int q = p + r2;
    const int pi = p / kCorrTile, qi = q / kCorrTile;  // pi <= qi
    const int tk = pi * nt - pi * (pi - 1) / 2 + (qi - pi);
    const int a = p % kCorrTile, b = q % kCorrTile;
    float2 s = make_float2(0.f, 0.f);
    for (int sl = 0; sl < n_slice; sl++) {
      float2 v = red[((sl * n_tiles + tk) * kCorrTile + a) * kCorrTile + b];
      s.x += v.x;
      s.y += v.y;
    }
    out[k] = s;
  }
}

cudaError_t launch_correlate(const float2* y, long long n_samp, int n_ant, int dump_len,
                             long long n_dump, long long first, long long last, float2* vis,
                             cudaStream_t st) {
  const int nt = (n_ant + kCorrTile - 1) / kCorrTile;
  const int n_tiles = nt * (nt + 1) / 2;
  if (n_tiles > kCorrThreads) return cudaErrorInvalidValue;
  const int n_slice = kCorrThreads / n_tiles;
  const int Mp = nt * kCorrTile;
  // staging chunk: at most 32 KB of voltages; the reduction reuses the buffer
  int chunk = (32 * 1024) / (8 * Mp);
  if (chunk > dump_len) chunk = dump_len;
  if (chunk < 1) chunk = 1;
  size_t stage = (size_t)Mp * chunk * sizeof(float2);
  size_t redb = (size_t)n_slice * n_tiles * kCorrTile * kCorrTile * sizeof(float2);
  size_t smem = stage > redb ? stage : redb;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_correlate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (n_dump <= 0) return cudaSuccess;
  k_correlate<<<(unsigned)n_dump, kCorrThreads, smem, st>>>(y, n_samp, n_ant, dump_len, first,
                                                             last, vis, chunk);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ beams from visibilities
// Exact identity: sum_t |sum_a W_pa y_a(t)|^2 = sum_{a,b} W_pa W_pb^* V_ab with
// V_ab = sum_t y_a y_b^* (the correlator's output), i.e. for the packed upper
// triangle  P_p = sum_{a<=b} Re(w_p,ab V_ab),  w_p,ab = c_ab W_pa W_pb^*,
// c = 1 on the diagonal, 2 above it.  wpair is [n_pair][n_pix] (pixel-fastest).
constexpr int kVisPix = 128;
constexpr int kVisDumps = 16;

__global__ void __launch_bounds__(kVisPix) k_beam_from_vis(const float2* __restrict__ V,
                                                           const float2* __restrict__ wpair,
                                                           int n_pair, int n_pix, long long first,
                                                           long long last,
                                                           float* __restrict__ pow) {
  extern __shared__ float2 sv[];  // [kVisDumps][n_pair]
  const long long m0 = first + (long long)blockIdx.x * kVisDumps;
  const int nd = (int)((last + 1 - m0) < kVisDumps ? (last + 1 - m0) : kVisDumps);
  const int p = blockIdx.y * kVisPix + threadIdx.x;
  for (int i = threadIdx.x; i < nd * n_pair; i += blockDim.x) sv[i] = V[m0 * n_pair + i];
  __syncthreads();
  if (p >= n_pix) return;
  float acc[kVisDumps];
#pragma unroll
  for (int d = 0; d < kVisDumps; d++) acc[d] = 0.f;
  for (int k = 0; k < n_pair; k++) {
    const float2 w = wpair[(long long)k * n_pix + p];
#pragma unroll
    for (int d = 0; d < kVisDumps; d++) {
      const float2 v = sv[d * n_pair + k < nd * n_pair ? d * n_pair + k : 0];
      acc[d] = fmaf(w.x, v.x, fmaf(-w.y, v.y, acc[d]));
    }
  }
  for (int d = 0; d < nd; d++) pow[(m0 + d) * n_pix + p] = acc[d];
}

cudaError_t launch_beam_from_vis(const float2* V, const float2* wpair, int n_ant, int n_pix,
                                 long long first, long long last, float* pow, cudaStream_t st) {
  if (last < first || n_pix <= 0) return cudaSuccess;
  const int n_pair = n_ant * (n_ant + 1) / 2;
  const size_t smem = (size_t)kVisDumps * n_pair * sizeof(float2);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_beam_from_vis,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long n = last - first + 1;
  dim3 grid((unsigned)((n + kVisDumps - 1) / kVisDumps), (n_pix + kVisPix - 1) / kVisPix);
  k_beam_from_vis<<<grid, kVisPix, smem, st>>>(V, wpair, n_pair, n_pix, first, last, pow);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ beamform
// One CTA per (dump, 128 pixels).  Weights of the CTA's pixels live in shared
// memory antenna-major; a chunk of every antenna's voltages is staged and each
// thread forms its pixel's beam sample by sample.
constexpr int kBeamPix = 128;
constexpr int kBeamChunk = 128;

__global__ void __launch_bounds__(kBeamPix) k_beamform_simt(const float2* __restrict__ y,
                                                            long long n_samp, int M, int L,
                                                            long long first, long long last,
                                                            const float2* __restrict__ W,
                                                            int n_pix, float* __restrict__ pow) {
  extern __shared__ float2 smem[];
  float2* sw = smem;                   // [M][kBeamPix]
  float2* sy = smem + M * kBeamPix;    // [M][kBeamChunk]
  const long long m = blockIdx.x;
  const int p = blockIdx.y * kBeamPix + threadIdx.x;
  float* out = pow + m * n_pix;
  if (m < first || m > last) {
    if (p < n_pix) out[p] = 0.f;
    return;
  }
  for (int a = 0; a < M; a++)
    sw[a * kBeamPix + threadIdx.x] = (p < n_pix) ? W[(long long)p * M + a] : make_float2(0.f, 0.f);
  float total = 0.f;
  const long long t0 = m * L;
  for (int c0 = 0; c0 < L; c0 += kBeamChunk) {
    const int len = (L - c0) < kBeamChunk ? (L - c0) : kBeamChunk;
    __syncthreads();
    for (int i = threadIdx.x; i < M * len; i += blockDim.x) {
      int a = i / len, t = i % len;
      sy[a * kBeamChunk + t] = y[(long long)a * n_samp + t0 + c0 + t];
    }
    __syncthreads();
    float part = 0.f;
    for (int t = 0; t < len; t++) {
      float br = 0.f, bi = 0.f;
      for (int a = 0; a < M; a++) {
        float2 w = sw[a * kBeamPix + threadIdx.x];
        float2 v = sy[a * kBeamChunk + t];
        br = fmaf(w.x, v.x, fmaf(-w.y, v.y, br));
        bi = fmaf(w.x, v.y, fmaf(w.y, v.x, bi));
      }
      part = fmaf(br, br, fmaf(bi, bi, part));
    }
    total += part;
  }
  if (p < n_pix) out[p] = total;
}

cudaError_t launch_beamform_simt(const float2* y, long long n_samp, int n_ant, int dump_len,
                                 long long n_dump, long long first, long long last,
                                 const float2* W, int n_pix, float* pow, cudaStream_t st) {
  size_t smem = (size_t)n_ant * (kBeamPix + kBeamChunk) * sizeof(float2);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_beamform_simt,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (n_dump <= 0 || n_pix <= 0) return cudaSuccess;
  dim3 grid((unsigned)n_dump, (n_pix + kBeamPix - 1) / kBeamPix);
  k_beamform_simt<<<grid, kBeamPix, smem, st>>>(y, n_samp, n_ant, dump_len, first, last, W,
                                                n_pix, pow);
  return cudaGetLastError();
}

}  // namespace chirp
