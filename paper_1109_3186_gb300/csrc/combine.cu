// combine.cu -- combination of coarse channels searched separately.
//
// A wide band searched as C coarse channels gives, per channel, dump powers
// whose time reference is the arrival at that channel's own centre f_c
// (dedispersion about the band centre, Sec. 2.3.2).  A pulse reaches channel
// c later than the top channel (f_ref = max f_c) by the Eq. 1 delay
// k DM (f_c^-2 - f_ref^-2), i.e. s_c = rint(k DM (f_c^-2 - f_ref^-2) B / L)
// dumps, so the channels are aligned to the top channel and added
// incoherently:
//     E[d][m][pix] = sum_c P_c[d][m + s_c(d)][pix]
// wherever every channel's dump m + s_c(d) exists and is valid for DM d, and
// E = 0 elsewhere.  The shifts and the valid range of m are integers formed
// on the host in FP64; the kernel is a gather-add bound by HBM bandwidth
// (C reads and one write of 4 bytes per output cell).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/chirp_gb300.h"
#include "internal.h"

namespace {

constexpr int kMaxChan = CHIRP_MAX_CHANNELS;

struct ChanPtrs {
  const float* p[kMaxChan];
};

// One CTA per (dump m, DM d) row, threads over pixels (float4 when the rows
// are 16-byte aligned).  info[d] = {m_lo, m_hi} of the combined valid dumps;
// shift[d * C + c] = s_c(d).
template <bool VEC>
__global__ void __launch_bounds__(256) k_combine(ChanPtrs P, int C, long long n_dump, int n_pix,
                                                 const long long* __restrict__ info,
                                                 const int* __restrict__ shift,
                                                 float* __restrict__ E) {
  const long long m = blockIdx.x;
  const int d = blockIdx.y;
  float* out = E + ((long long)d * n_dump + m) * n_pix;
  const long long m_lo = info[2 * d], m_hi = info[2 * d + 1];
  const bool ok = m >= m_lo && m <= m_hi;
  if constexpr (VEC) {
    const int n4 = n_pix / 4;
    float4* o4 = reinterpret_cast<float4*>(out);
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      if (ok)
        for (int c = 0; c < C; c++) {
          const long long mc = m + shift[d * C + c];
          const float4 v = __ldg(reinterpret_cast<const float4*>(
                                     P.p[c] + ((long long)d * n_dump + mc) * n_pix) + i);
          acc.x += v.x;
          acc.y += v.y;
          acc.z += v.z;
          acc.w += v.w;
        }
      o4[i] = acc;
    }
  } else {
    for (int i = threadIdx.x; i < n_pix; i += blockDim.x) {
      float acc = 0.f;
      if (ok)
        for (int c = 0; c < C; c++) {
          const long long mc = m + shift[d * C + c];
          acc += __ldg(P.p[c] + ((long long)d * n_dump + mc) * n_pix + i);
        }
      out[i] = acc;
    }
  }
}

int cfail(int code, const char* msg) { return chirp_report_error(code, msg); }

}  // namespace

extern "C" int chirp_combine_channels(const float* const* P, int n_chan, int n_dm,
                                      long long n_dump, int n_pix, const long long* first,
                                      const long long* last, const double* f_c, double bw_hz,
                                      int dump_len, double k_dm, const double* dm, float* E,
                                      void* stream) {
  chirp_clear_error();
  if (!P || !first || !last || !f_c || !dm || !E)
    return cfail(CHIRP_EINVAL, "chirp_combine_channels: NULL argument");
  if (n_chan < 1 || n_chan > kMaxChan)
    return cfail(CHIRP_EINVAL, "chirp_combine_channels: n_chan must be in 1..64");
  if (n_dm < 1 || n_dm > 65535 || n_dump < 1 || n_dump >= (1LL << 31) || n_pix < 1)
    return cfail(CHIRP_EINVAL, "chirp_combine_channels: need n_dm in 1..65535, n_dump in 1..2^31-1, "
                               "n_pix >= 1");
  if (!(bw_hz > 0) || dump_len < 1)
    return cfail(CHIRP_EINVAL, "chirp_combine_channels: need bw_hz > 0 and dump_len >= 1");
  for (int c = 0; c < n_chan; c++) {
    if (!P[c]) return cfail(CHIRP_EINVAL, "chirp_combine_channels: NULL channel buffer");
    if (!(f_c[c] > 0) || !std::isfinite(f_c[c]))
      return cfail(CHIRP_EINVAL, "chirp_combine_channels: channel centres must be > 0");
  }
  for (int d = 0; d < n_dm; d++)
    if (!(dm[d] >= 0) || !std::isfinite(dm[d]))
      return cfail(CHIRP_EINVAL, "chirp_combine_channels: DMs must be finite and >= 0");
  if (!(k_dm > 0)) k_dm = chirp::kDefaultKdm;
  cudaStream_t st = (cudaStream_t)stream;

  // alignment shifts (Eq. 1 between the channel centres and the top channel)
  // and the combined valid range of every DM
  double f_ref = f_c[0];
  for (int c = 1; c < n_chan; c++) f_ref = std::max(f_ref, f_c[c]);
  std::vector<int> shift((size_t)n_dm * n_chan);
  std::vector<long long> info(2 * (size_t)n_dm);
  for (int d = 0; d < n_dm; d++) {
    long long m_lo = 0, m_hi = n_dump - 1;
    for (int c = 0; c < n_chan; c++) {
      const double s = std::rint(k_dm * dm[d] * (1.0 / (f_c[c] * f_c[c]) - 1.0 / (f_ref * f_ref)) *
                                 bw_hz / dump_len);
      if (!(std::fabs(s) < 1e9))
        return cfail(CHIRP_EINVAL, "chirp_combine_channels: alignment shift out of range");
      shift[(size_t)d * n_chan + c] = (int)s;
      const long long fc = first[(size_t)c * n_dm + d], lc = last[(size_t)c * n_dm + d];
      if (fc < 0) return cfail(CHIRP_EINVAL, "chirp_combine_channels: first dumps must be >= 0");
      m_lo = std::max(m_lo, fc - (long long)s);
      m_hi = std::min(m_hi, std::min(lc, n_dump - 1) - (long long)s);
    }
    info[2 * d] = m_lo;
    info[2 * d + 1] = m_hi;  // m_hi < m_lo: no combined dump
  }
  ChanPtrs cp{};
  bool aligned = n_pix % 4 == 0 && ((uintptr_t)E & 15) == 0;
  for (int c = 0; c < n_chan; c++) {
    cp.p[c] = P[c];
    aligned = aligned && ((uintptr_t)P[c] & 15) == 0;
  }
  // small stream-ordered workspace for the shifts and ranges
  const size_t bytes = info.size() * sizeof(long long) + shift.size() * sizeof(int);
  void* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cfail(CHIRP_ENOMEM, "chirp_combine_channels: workspace allocation failed");
  }
  long long* d_info = (long long*)ws;
  int* d_shift = (int*)(d_info + info.size());
  e = cudaMemcpyAsync(d_info, info.data(), info.size() * sizeof(long long), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_shift, shift.data(), shift.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    const dim3 grid((unsigned)n_dump, (unsigned)n_dm);
    if (aligned)
      k_combine<true><<<grid, 256, 0, st>>>(cp, n_chan, n_dump, n_pix, d_info, d_shift, E);
    else
      k_combine<false><<<grid, 256, 0, st>>>(cp, n_chan, n_dump, n_pix, d_info, d_shift, E);
    e = cudaGetLastError();
  }
  // pageable host sources are staged before cudaMemcpyAsync returns, so the
  // vectors may go; the workspace is released in stream order
  cudaFreeAsync(ws, st);
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof msg, "chirp_combine_channels: %s", cudaGetErrorString(e));
    return cfail(CHIRP_ECUDA, msg);
  }
  return CHIRP_OK;
}
