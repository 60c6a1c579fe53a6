// truedelay.cu -- true-delay (wideband) beams of the dedispersed voltages
// (Sec. 2.4.2 direct beamforming with each antenna's geometric delay of
// Eq. tau3D applied at every frequency of the overlap-save blocks).
//
// Per trial DM and chunk of (block, pixel) sequences: the beam spectra
// Y_pb(f) = sum_a W_pa(f) X_ab(f) (k_td_spectra), the inverse row pass of
// dedisperse.cu with the DM's chirp H (and 1/Nfft) multiplied in on load,
// and a column pass that detects and integrates (k_inv_cols_pow).
#include <cuda_runtime.h>

#include "fft.cuh"
#include "internal.h"

namespace chirp {

static __device__ __forceinline__ Twiddles mk_tw(TwiddlePtrs p) {
  return Twiddles{p.coarse, p.fine, p.stage};
}

// ------------------------------------------------------------------ true-delay beams
// Beam spectra of a chunk of (block, pixel) sequences: for every bin of the
// transposed spectrum order (position k1 n2 + k2 holds natural bin
// fi = k1 + n1 k2, taken as fi - Nfft from Nfft/2 up)
//   Y[(b - b0) np + p][pos] = sum_a W_pa(fi) X[b][a][pos],
//   W_pa(fi) = exp(+2 pi j (f0 + fi B / Nfft) tau_pa)      (Eq. tau3D delays).
// The phase is kept in 64-bit fixed point (cycles x 2^64, modulo 1): per
// (pixel, antenna) ph = {frac(f0 tau), frac(B tau / Nfft)} from the host in
// FP64, so the phase of bin fi is base + fi rate modulo 2^64 -- exact integer
// arithmetic -- and only the top 32 bits reach sincospif.  A thread takes
// kTdRun consecutive positions of one row (consecutive k2: fi steps by n1, and
// a run never straddles k2 = n2/2 because n2/2 is a multiple of kTdRun): the
// first weight of the run is exact, the others follow by the FP32 step
// rot_pa = exp(2 pi j n1 B tau / Nfft) (host FP64, rounded once), i.e. at most
// kTdRun - 1 rounded products (relative error ~1e-6).  kTdPix pixels per
// thread (grid.z chunks), antennas in the loop.
constexpr int kTdPix = 4;
constexpr int kTdRun = 8;

__global__ void __launch_bounds__(128) k_td_spectra(const float2* __restrict__ spec,
                                                    float2* __restrict__ Y, long long b0, int np,
                                                    int p_base, int M, int n1, int n2,
                                                    long long nfft,
                                                    const ulonglong2* __restrict__ ph,
                                                    const float2* __restrict__ rot) {
  // grid (pixel chunks, runs / 128, blocks): the pixel chunks that read the
  // same spectrum runs are the fastest grid index, so they run together and
  // find them in L2
  const long long pos0 = ((long long)blockIdx.y * blockDim.x + threadIdx.x) * kTdRun;
  if (pos0 >= nfft) return;
  const long long b = b0 + blockIdx.z;
  const int pz = blockIdx.x * kTdPix;  // first pixel of this thread's chunk (launch-local)
  const long long k1 = pos0 / n2, k2 = pos0 % n2;
  long long fi = k1 + (long long)n1 * k2;
  if (2 * fi >= nfft) fi -= nfft;
  const unsigned long long ufi = (unsigned long long)fi;  // two's complement: modular product
  float2 acc[kTdPix][kTdRun];
#pragma unroll
  for (int j = 0; j < kTdPix; j++)
#pragma unroll
    for (int r = 0; r < kTdRun; r++) acc[j][r] = make_float2(0.f, 0.f);
  for (int a = 0; a < M; a++) {
    const float4* xs = reinterpret_cast<const float4*>(spec + ((b * M) + a) * nfft + pos0);
    float2 x[kTdRun];
#pragma unroll
    for (int r = 0; r < kTdRun / 2; r++) {
      const float4 v = xs[r];
      x[2 * r] = make_float2(v.x, v.y);
      x[2 * r + 1] = make_float2(v.z, v.w);
    }
#pragma unroll
    for (int j = 0; j < kTdPix; j++) {
      const int p = pz + j;
      if (p >= np) break;
      const long long e_idx = (long long)(p_base + p) * M + a;
      const ulonglong2 e = __ldg(ph + e_idx);
      const float2 st = __ldg(rot + e_idx);
      const unsigned long long u = e.x + ufi * e.y;
      const int top = (int)(u >> 32);              // cycles x 2^32 in [-2^31, 2^31)
      float2 w;
      sincospif(ldexpf((float)top, -31), &w.y, &w.x);  // 2 pi x cycles
#pragma unroll
      for (int r = 0; r < kTdRun; r++) {
        acc[j][r].x = fmaf(w.x, x[r].x, fmaf(-w.y, x[r].y, acc[j][r].x));
        acc[j][r].y = fmaf(w.x, x[r].y, fmaf(w.y, x[r].x, acc[j][r].y));
        const float wx = w.x * st.x - w.y * st.y;  // next bin of the run: fi + n1
        w.y = w.x * st.y + w.y * st.x;
        w.x = wx;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kTdPix; j++) {
    const int p = pz + j;
    if (p >= np) break;
    float4* yo = reinterpret_cast<float4*>(Y + ((long long)blockIdx.z * np + p) * nfft + pos0);
#pragma unroll
    for (int r = 0; r < kTdRun / 2; r++)
      yo[r] = make_float4(acc[j][2 * r].x, acc[j][2 * r].y, acc[j][2 * r + 1].x,
                          acc[j][2 * r + 1].y);
  }
}

// Column pass of the inverse for beam sequences, detecting and integrating:
// sequence q of the launch is block b0 + q / np, pixel p_base + q % np; every
// owned sample t of the block inside [t_lo, t_hi) (the DM's valid dumps) adds
// |y(t)|^2 to P[t / dump_len][pixel].  The CTA's C consecutive samples of each
// of its L rows are staged as powers in the transform's shared tile (zero
// outside the owned, valid range); one thread then sums a row per dump it
// meets and adds each sum to P with one atomic add.
template <int L>
__global__ void __launch_bounds__(256, 4) k_inv_cols_pow(
    const float2* __restrict__ Z, float* __restrict__ P, long long n_samp, int n2, long long step,
    long long n_blk, long long b0, int np, int p_base, int n_pix, long long n_hi, long long n_lo,
    long long n_hi_max, int dump_len, long long t_lo, long long t_hi, TwiddlePtrs twp) {
  constexpr int C = 4096 / L;
  constexpr int T = L / 16;
  __shared__ __align__(16) float2 sm[FftTile<L, C>::SLOTS];
  const Twiddles tw = mk_tw(twp);
  const int s = threadIdx.x % C, jt = threadIdx.x / C;
  const int c = blockIdx.x * C + s;
  const bool act = c < n2;
  const long long q = blockIdx.y;
  const long long b = b0 + q / np;
  const int pix = p_base + (int)(q % np);
  const long long nfft = (long long)L * n2;
  // positions inside a block, (jt + k T) n2 + c < nfft <= 2^24, are 32-bit
  const float2* src = Z + q * nfft + c;
  float2 v[16];
#pragma unroll
  for (int k = 0; k < 16; k++) v[k] = act ? src[(jt + k * T) * n2] : make_float2(0.f, 0.f);
  fft_core<L, C, false, true>(v, sm, s, jt, tw);
  const long long base = b * step;
  const long long lo_b = (b == 0) ? n_hi : n_hi_max;
  const long long hi_b = (b == n_blk - 1) ? (n_samp - n_lo - base) : (n_hi_max + step);
  // owned and inside the DM's valid dumps: n in [nlo, nhi), clamped to [0, nfft]
  long long nlo = lo_b > t_lo - base ? lo_b : t_lo - base;
  long long nhi = hi_b < t_hi - base ? hi_b : t_hi - base;
  nlo = nlo < 0 ? 0 : (nlo > nfft ? nfft : nlo);
  nhi = nhi < 0 ? 0 : (nhi > nfft ? nfft : nhi);
  const int nlo32 = (int)nlo, nhi32 = (int)nhi;
  // powers [L rows][C columns], rows padded to C + 1 floats so that the row
  // sums below (one thread per row) read distinct banks
  float* et = reinterpret_cast<float*>(sm);
  static_assert(L * (C + 1) <= 2 * FftTile<L, C>::SLOTS, "staging fits the transform's tile");
  __syncthreads();                           // the transform is done with sm
#pragma unroll
  for (int k = 0; k < 16; k++) {
    const int row = jt + k * T;
    const int n = row * n2 + c;
    et[row * (C + 1) + s] =
        (act && n >= nlo32 && n < nhi32) ? v[k].x * v[k].x + v[k].y * v[k].y : 0.f;
  }
  __syncthreads();
  const int col0 = blockIdx.x * C;
  const int n_col = min(C, n2 - col0);
  for (int row = threadIdx.x; row < L; row += blockDim.x) {
    const int n_first = row * n2 + col0;
    if (n_first + n_col <= nlo32 || n_first >= nhi32) continue;  // nothing owned and valid
    const long long tr = base + n_first;  // the row's first sample: m dump_len + r
    long long m = tr / dump_len;
    int r = (int)(tr - m * dump_len);
    float acc = 0.f;
    for (int j = 0; j < n_col; j++) {
      acc += et[row * (C + 1) + j];
      if (++r == dump_len || j == n_col - 1) {  // end of a dump, or of the row
        if (acc != 0.f) atomicAdd(&P[m * n_pix + pix], acc);
        acc = 0.f;
        r = 0;
        m++;
      }
    }
  }
}

#define CHIRP_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

cudaError_t launch_td_spectra(const float2* spec, float2* Y, long long b0, int nb, int np,
                              int p_base, int n_ant, const GroupGeom& g, const void* ph,
                              const float2* rot, cudaStream_t st) {
  const long long runs = g.nfft / kTdRun;
  if (nb < 1 || nb > 65535 || np < 1 || (g.n2 / 2) % kTdRun != 0 || (runs + 127) / 128 > 65535)
    return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)((np + kTdPix - 1) / kTdPix), (unsigned)((runs + 127) / 128), (unsigned)nb);
  k_td_spectra<<<grid, 128, 0, st>>>(spec, Y, b0, np, p_base, n_ant, g.n1, g.n2, g.nfft,
                                     static_cast<const ulonglong2*>(ph), rot);
  return cudaGetLastError();
}

cudaError_t launch_inverse_cols_pow(const float2* Z, float* P, long long n_samp, long long b0,
                                    int nb, int np, int p_base, int n_pix, const GroupGeom& g,
                                    long long n_hi, long long n_lo, int dump_len, long long t_lo,
                                    long long t_hi, TwiddlePtrs tw, cudaStream_t st) {
  const long long nq = (long long)nb * np;
  if (nq > 65535 || nq < 1) return cudaErrorInvalidConfiguration;
  const int C = 4096 / g.n1;
  dim3 grid((g.n2 + C - 1) / C, (unsigned)nq);
  switch (g.n1) {
#define X(L)                                                                                    \
  case L:                                                                                       \
    k_inv_cols_pow<L><<<grid, 256, 0, st>>>(Z, P, n_samp, g.n2, g.step, g.n_blk, b0, np, p_base, \
                                            n_pix, n_hi, n_lo, g.n_hi_max, dump_len, t_lo, t_hi, \
                                            tw);                                                \
    break;
    CHIRP_SIZES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace chirp
