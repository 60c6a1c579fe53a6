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
// One CTA per dump.  Threads = (pair slot, time slice); each thread walks
// the pairs slot, slot + n_slot, ... over its slice of every staged chunk.
constexpr int kCorrThreads = 256;
constexpr int kCorrMaxPairsPerThread = 16;  // n_pair <= 4096 -> n_ant <= 90

__global__ void __launch_bounds__(kCorrThreads) k_correlate(const float2* __restrict__ y,
                                                             long long n_samp, int M, int L,
                                                             long long first, long long last,
                                                             float2* __restrict__ vis,
                                                             int chunk) {
  extern __shared__ float2 sy[];  // [M][chunk]
  const long long m = blockIdx.x;
  const int n_pair = M * (M + 1) / 2;
  float2* out = vis + m * n_pair;
  if (m < first || m > last) {
    for (int i = threadIdx.x; i < n_pair; i += blockDim.x) out[i] = make_float2(0.f, 0.f);
    return;
  }
  const int n_slot = n_pair < kCorrThreads ? n_pair : kCorrThreads;
  const int n_slice = kCorrThreads / n_slot;
  const int slot = threadIdx.x % n_slot, slice = threadIdx.x / n_slot;
  const bool worker = slice < n_slice;
  float2 acc[kCorrMaxPairsPerThread];
  int pp_p[kCorrMaxPairsPerThread], pp_q[kCorrMaxPairsPerThread];
  int n_mine = 0;
  for (int k = slot; k < n_pair && n_mine < kCorrMaxPairsPerThread; k += n_slot) {
    // invert the row-major upper-triangle index k -> (p, q)
    int p = 0, rem = k;
    while (rem >= M - p) {
      rem -= M - p;
      p++;
    }
    pp_p[n_mine] = p;
    pp_q[n_mine] = p + rem;
    acc[n_mine] = make_float2(0.f, 0.f);
    n_mine++;
  }
  const long long t0 = m * L;
  for (int c0 = 0; c0 < L; c0 += chunk) {
    const int len = (L - c0) < chunk ? (L - c0) : chunk;
    __syncthreads();
    for (int i = threadIdx.x; i < M * len; i += blockDim.x) {
      int a = i / len, t = i % len;
      sy[a * chunk + t] = y[(long long)a * n_samp + t0 + c0 + t];
    }
    __syncthreads();
    if (worker) {
      for (int j = 0; j < n_mine; j++) {
        const float2* yp = sy + pp_p[j] * chunk;
        const float2* yq = sy + pp_q[j] * chunk;
        float2 part = make_float2(0.f, 0.f);
        for (int t = slice; t < len; t += n_slice) {
          float2 u = yp[t], w = yq[t];
          // u * conj(w)
          part.x = fmaf(u.x, w.x, fmaf(u.y, w.y, part.x));
          part.y = fmaf(u.y, w.x, fmaf(-u.x, w.y, part.y));
        }
        acc[j].x += part.x;
        acc[j].y += part.y;
      }
    }
  }
  // reduce over slices through shared memory (reuse the staging buffer)
  __syncthreads();
  float2* red = sy;  // [n_slice][n_pair]
  if (worker)
    for (int j = 0; j < n_mine; j++) {
      int k = slot + j * n_slot;
      red[slice * n_pair + k] = acc[j];
    }
  __syncthreads();
  for (int k = threadIdx.x; k < n_pair; k += blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int sl = 0; sl < n_slice; sl++) {
      s.x += red[sl * n_pair + k].x;
      s.y += red[sl * n_pair + k].y;
    }
    out[k] = s;
  }
}

cudaError_t launch_correlate(const float2* y, long long n_samp, int n_ant, int dump_len,
                             long long n_dump, long long first, long long last, float2* vis,
                             cudaStream_t st) {
  const int n_pair = n_ant * (n_ant + 1) / 2;
  const int n_slot = n_pair < kCorrThreads ? n_pair : kCorrThreads;
  if ((n_pair + n_slot - 1) / n_slot > kCorrMaxPairsPerThread) return cudaErrorInvalidValue;
  const int n_slice = kCorrThreads / n_slot;
  // staging chunk: at most 32 KB of voltages; the reduction reuses the buffer
  int chunk = (32 * 1024) / (8 * n_ant);
  if (chunk > dump_len) chunk = dump_len;
  if (chunk < 1) chunk = 1;
  size_t stage = (size_t)n_ant * chunk * sizeof(float2);
  size_t redb = (size_t)n_slice * n_pair * sizeof(float2);
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
