// reduced.cu -- the inverse column pass writing dedispersed voltages rounded
// once to BF16, the input of the reduced-precision visibility form of the
// Chimageator (CHIRP_BEAM_VIS_BF16): the same transform and overlap-save
// discard as the FP32 column pass of dedisperse.cu, with each owned, valid
// sample stored as a (re, im) pair of BF16 (4 bytes instead of 8), which
// halves both this pass's stores and the correlator's reads.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fft.cuh"
#include "internal.h"

namespace chirp {

static __device__ __forceinline__ Twiddles mk_tw(TwiddlePtrs p) {
  return Twiddles{p.coarse, p.fine, p.stage};
}

template <int L>
__global__ void __launch_bounds__(256, 4) k_inv_cols_y16(const float2* __restrict__ Z,
                                                      __nv_bfloat162* __restrict__ y16,
                                                      long long n_samp, int n2, long long step,
                                                      long long n_blk, int n_ant, long long n_hi,
                                                      long long n_lo, long long n_hi_max,
                                                      long long q0,
                                                      const int* __restrict__ blk_list,
                                                      TwiddlePtrs twp) {
  constexpr int C = 4096 / L;
  constexpr int T = L / 16;
  __shared__ __align__(16) float2 sm[FftTile<L, C>::SLOTS];
  const Twiddles tw = mk_tw(twp);
  const int s = threadIdx.x % C, jt = threadIdx.x / C;
  const int c = blockIdx.x * C + s;
  const bool act = c < n2;
  const long long q = blk_list ? (long long)blk_list[blockIdx.y / n_ant] * n_ant + blockIdx.y % n_ant
                               : q0 + blockIdx.y;  // block-major sequence; Z holds the launch
  const long long a = q % n_ant, b = q / n_ant;
  const long long nfft = (long long)L * n2;
  // positions inside a block, (jt + k T) n2 + c < nfft <= 2^24, are 32-bit
  const float2* src = Z + (long long)blockIdx.y * nfft + c;
  float2 v[16];
#pragma unroll
  for (int k = 0; k < 16; k++) v[k] = act ? src[(jt + k * T) * n2] : make_float2(0.f, 0.f);
  fft_core<L, C, false, true>(v, sm, s, jt, tw);
  if (!act) return;
  const long long base = b * step;
  const long long lo_b = (b == 0) ? n_hi : n_hi_max;
  const long long hi_b = (b == n_blk - 1) ? (n_samp - n_lo - base) : (n_hi_max + step);
  const int lo32 = (int)(lo_b < 0 ? 0 : (lo_b > nfft ? nfft : lo_b));
  const int hi32 = (int)(hi_b < 0 ? 0 : (hi_b > nfft ? nfft : hi_b));
  __nv_bfloat162* yb = y16 + a * n_samp + base;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    const int n = (jt + k * T) * n2 + c;
    if (n >= lo32 && n < hi32) yb[n] = __floats2bfloat162_rn(v[k].x, v[k].y);
  }
}

#define CHIRP_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

cudaError_t launch_inverse_cols_bf16(const float2* Z, void* y16, long long n_samp, int n_ant,
                                     long long q0, long long nq, const GroupGeom& g,
                                     long long n_hi, long long n_lo, TwiddlePtrs tw,
                                     cudaStream_t st, const int* blk_list) {
  if (nq > 65535 || nq < 1) return cudaErrorInvalidConfiguration;
  const int C = 4096 / g.n1;
  dim3 grid((g.n2 + C - 1) / C, (unsigned)nq);
  __nv_bfloat162* y = static_cast<__nv_bfloat162*>(y16);
  switch (g.n1) {
#define X(L)                                                                                  \
  case L:                                                                                     \
    k_inv_cols_y16<L><<<grid, 256, 0, st>>>(Z, y, n_samp, g.n2, g.step, g.n_blk, n_ant, n_hi, \
                                            n_lo, g.n_hi_max, q0, blk_list, tw);               \
    break;
    CHIRP_SIZES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace chirp
