// detect.cu -- candidate detection on the Chimageator's dump powers
// (thresholding of the detection metric, Sec. 3.3 after Eq. eth; the best of
// a bank of trial filters over DM, time and direction, App. A.3).
//
// Per (DM d, pixel p) series x_m = P[d][m][p] over the DM's valid dumps:
//   med = median(x) (even count: (a + b) * 0.5),  sigma = 1.4826f * median(|x - med|),
//   S/N = (x - med) / sigma   (0 when sigma == 0),
// every operation one IEEE-rounded FP32 step (no contraction), so that the
// S/N values and hence the threshold and local-maximum decisions are exact.
// A candidate is a valid cell with S/N >= snr_min that no valid neighbour
// (d +- 1, m +- 1, p +- 1) exceeds.
//
// Kernels:
//   k_series_stats  one CTA per (DM, 32 consecutive pixels): exact medians by
//                   radix selection on order-preserving 32-bit keys (four
//                   8-bit digit passes over the series, histograms in shared
//                   memory) plus, for even counts, one pass for the next
//                   order statistic; the same for the absolute deviations.
//                   Reads are coalesced: a warp reads 32 pixels of one dump.
//   k_peak_count    per chunk of 2048 cells (in (d, m, p) order) the number
//                   of candidates;
//   k_peak_scan     exclusive scan of the chunk counts (one CTA);
//   k_peak_write    re-evaluates its chunk and writes the candidates at their
//                   scanned positions, so the list comes out in (d, m, p)
//                   order without sorting.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/chirp_gb300.h"
#include "internal.h"

namespace chirp {

namespace {

constexpr int kSeriesPerCta = 32;
constexpr int kStatsThreads = 256;
constexpr int kCellsPerThread = 8;
constexpr int kPeakThreads = 256;
constexpr int kCellsPerChunk = kCellsPerThread * kPeakThreads;

__device__ __forceinline__ uint32_t order_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_value(uint32_t k) {
  const uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(b);
}

__global__ void __launch_bounds__(kStatsThreads) k_series_stats(const float* __restrict__ P,
                                                                long long n_dump, int n_pix,
                                                                const long long* __restrict__ first,
                                                                const long long* __restrict__ last,
                                                                float2* __restrict__ stats) {
  __shared__ uint32_t hist[kSeriesPerCta][257];
  __shared__ uint32_t prefix[kSeriesPerCta], mask[kSeriesPerCta], krem[kSeriesPerCta];
  __shared__ uint32_t cnt_le[kSeriesPerCta], min_gt[kSeriesPerCta];
  __shared__ float center[kSeriesPerCta];
  const int d = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kStatsThreads / 32;
  const int p = blockIdx.x * kSeriesPerCta + lane;
  const bool pv = p < n_pix;
  const long long f = first[d], n = last[d] - first[d] + 1;
  if (n <= 0) {
    if (warp == 0 && pv) stats[(long long)d * n_pix + p] = make_float2(0.f, 0.f);
    return;
  }
  const float* base = P + ((long long)d * n_dump + f) * n_pix + p;
  const long long k1 = (n - 1) / 2;
  const bool even = (n % 2) == 0;
  if (warp == 0) center[lane] = 0.f;
  float med = 0.f, result = 0.f;
  for (int kind = 0; kind < 2; kind++) {  // 0: the values, 1: |value - med|
    if (warp == 0) {
      prefix[lane] = 0u;
      mask[lane] = 0u;
      krem[lane] = (uint32_t)k1;
    }
    __syncthreads();
    for (int pass = 0; pass < 4; pass++) {
      const int shift = 24 - 8 * pass;
      for (int i = threadIdx.x; i < kSeriesPerCta * 257; i += kStatsThreads)
        (&hist[0][0])[i] = 0u;
      __syncthreads();
      if (pv) {
        const uint32_t pre = prefix[lane], msk = mask[lane];
        const float c = center[lane];
        for (long long m = warp; m < n; m += NW) {
          const float x = base[m * n_pix];
          const float v = kind ? fabsf(__fsub_rn(x, c)) : x;
          const uint32_t key = order_key(v);
          if ((key & msk) == pre) atomicAdd(&hist[lane][(key >> shift) & 255u], 1u);
        }
      }
      __syncthreads();
      if (warp == 0 && pv) {
        uint32_t k = krem[lane], cum = 0u;
        int digit = 255;
        for (int b = 0; b < 256; b++) {
          const uint32_t c = hist[lane][b];
          if (k < cum + c) {
            digit = b;
            break;
          }
          cum += c;
        }
        krem[lane] = k - cum;
        prefix[lane] |= (uint32_t)digit << shift;
        mask[lane] |= 0xFFu << shift;
      }
      __syncthreads();
    }
    // prefix now holds the key of order statistic k1
    float v1 = key_value(prefix[lane]), v2 = v1;
    if (even) {
      if (warp == 0) {
        cnt_le[lane] = 0u;
        min_gt[lane] = 0xFFFFFFFFu;
      }
      __syncthreads();
      if (pv) {
        const uint32_t kk = prefix[lane];
        const float c = center[lane];
        uint32_t le = 0u, gt = 0xFFFFFFFFu;
        for (long long m = warp; m < n; m += NW) {
          const float x = base[m * n_pix];
          const float v = kind ? fabsf(__fsub_rn(x, c)) : x;
          const uint32_t key = order_key(v);
          if (key <= kk) le++;
          else if (key < gt) gt = key;
        }
        atomicAdd(&cnt_le[lane], le);
        atomicMin(&min_gt[lane], gt);
      }
      __syncthreads();
      v2 = cnt_le[lane] >= (uint32_t)(k1 + 2) ? v1 : key_value(min_gt[lane]);
    }
    const float mid = even ? __fmul_rn(__fadd_rn(v1, v2), 0.5f) : v1;
    if (kind == 0) {
      med = mid;
      __syncthreads();
      if (warp == 0) center[lane] = med;
      __syncthreads();
    } else {
      result = __fmul_rn(1.4826f, mid);
    }
  }
  if (warp == 0 && pv) stats[(long long)d * n_pix + p] = make_float2(med, result);
}

struct PeakArgs {
  const float* P;
  const float2* stats;
  const long long* first;
  const long long* last;
  long long n_dump;
  long long total;  // n_dm * n_dump * n_pix
  int n_dm, n_pix;
  float snr_min;
};

__device__ __forceinline__ bool snr_of(const PeakArgs& a, int d, long long m, int p, float* s) {
  if (d < 0 || d >= a.n_dm || p < 0 || p >= a.n_pix) return false;
  if (m < a.first[d] || m > a.last[d]) return false;
  const float2 st = a.stats[(long long)d * a.n_pix + p];
  if (!(st.y > 0.f)) {
    *s = 0.f;
    return true;
  }
  *s = __fdiv_rn(__fsub_rn(a.P[((long long)d * a.n_dump + m) * a.n_pix + p], st.x), st.y);
  return true;
}

__device__ bool is_candidate(const PeakArgs& a, long long i, float* snr) {
  const int p = (int)(i % a.n_pix);
  const long long dm_ = i / a.n_pix;
  const long long m = dm_ % a.n_dump;
  const int d = (int)(dm_ / a.n_dump);
  float s;
  if (!snr_of(a, d, m, p, &s) || !(s >= a.snr_min)) return false;
  for (int dd = -1; dd <= 1; dd++)
    for (int dm = -1; dm <= 1; dm++)
      for (int dp = -1; dp <= 1; dp++) {
        if (!dd && !dm && !dp) continue;
        float t;
        if (snr_of(a, d + dd, m + dm, p + dp, &t) && t > s) return false;
      }
  *snr = s;
  return true;
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[kPeakThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kPeakThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kPeakThreads / 32) warp_sums[lane] = w;
  }
  __syncthreads();
  const int before = warp ? warp_sums[warp - 1] : 0;
  *total = warp_sums[kPeakThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_count(PeakArgs a, int* __restrict__ counts) {
  const long long c0 = (long long)blockIdx.x * kCellsPerChunk + (long long)threadIdx.x * kCellsPerThread;
  int c = 0;
  for (int j = 0; j < kCellsPerThread; j++) {
    float s;
    if (c0 + j < a.total && is_candidate(a, c0 + j, &s)) c++;
  }
  int total;
  block_exclusive_scan(c, &total);
  if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// offsets[i] = sum of counts[0 .. i); *n_total = sum of all
__global__ void __launch_bounds__(1024) k_peak_scan(const int* __restrict__ counts, long long n,
                                                    long long* __restrict__ offsets,
                                                    long long* __restrict__ n_total) {
  __shared__ long long part[1024];
  long long carry = 0;
  for (long long b = 0; b < n; b += 1024) {
    const long long i = b + threadIdx.x;
    const long long v = i < n ? counts[i] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const long long y = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < n) offsets[i] = carry + part[threadIdx.x] - v;
    carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_total = carry;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_write(PeakArgs a,
                                                             const long long* __restrict__ offsets,
                                                             chirp_candidate* __restrict__ out,
                                                             long long max_out) {
  const long long c0 = (long long)blockIdx.x * kCellsPerChunk + (long long)threadIdx.x * kCellsPerThread;
  unsigned flags = 0u;
  float snr[kCellsPerThread];
  int c = 0;
#pragma unroll
  for (int j = 0; j < kCellsPerThread; j++) {
    snr[j] = 0.f;
    if (c0 + j < a.total && is_candidate(a, c0 + j, &snr[j])) {
      flags |= 1u << j;
      c++;
    }
  }
  int total;
  long long pos = offsets[blockIdx.x] + block_exclusive_scan(c, &total);
#pragma unroll
  for (int j = 0; j < kCellsPerThread; j++) {
    if (!(flags & (1u << j))) continue;
    if (pos < max_out) {
      const long long i = c0 + j;
      chirp_candidate cd;
      cd.pix = (int)(i % a.n_pix);
      cd.dump = (i / a.n_pix) % a.n_dump;
      cd.dm = (int)(i / a.n_pix / a.n_dump);
      cd.snr = snr[j];
      cd.power = a.P[i];
      out[pos] = cd;
    }
    pos++;
  }
}

}  // namespace

long long detect_chunks(int n_dm, long long n_dump, int n_pix) {
  const long long total = (long long)n_dm * n_dump * n_pix;
  return (total + kCellsPerChunk - 1) / kCellsPerChunk;
}

cudaError_t launch_detect(const float* P, int n_dm, long long n_dump, int n_pix,
                          const long long* first, const long long* last, float snr_min,
                          float2* stats, int* counts, long long* offsets, long long* n_total,
                          chirp_candidate* out, long long max_out, cudaStream_t st) {
  dim3 g1((n_pix + kSeriesPerCta - 1) / kSeriesPerCta, n_dm);
  k_series_stats<<<g1, kStatsThreads, 0, st>>>(P, n_dump, n_pix, first, last, stats);
  PeakArgs a;
  a.P = P;
  a.stats = stats;
  a.first = first;
  a.last = last;
  a.n_dump = n_dump;
  a.total = (long long)n_dm * n_dump * n_pix;
  a.n_dm = n_dm;
  a.n_pix = n_pix;
  a.snr_min = snr_min;
  const long long nc = detect_chunks(n_dm, n_dump, n_pix);
  if (nc > 0x7FFFFFFFLL) return cudaErrorInvalidConfiguration;
  k_peak_count<<<(unsigned)nc, kPeakThreads, 0, st>>>(a, counts);
  k_peak_scan<<<1, 1024, 0, st>>>(counts, nc, offsets, n_total);
  k_peak_write<<<(unsigned)nc, kPeakThreads, 0, st>>>(a, offsets, out, max_out);
  return cudaGetLastError();
}

}  // namespace chirp
