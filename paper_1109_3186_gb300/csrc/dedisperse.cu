// dedisperse.cu -- overlap-save coherent dedispersion (Sec. 2.3.2) on sm_103a.
//
// Every block of Nfft = n1 * n2 samples is transformed with two passes over
// HBM (the "four-step" factorisation):
// Sequences (one transform each) are numbered block-major, q = b n_ant + a,
// so the sequences of a range of blocks are contiguous for all antennas.
//   forward:  column FFTs of length n1 (stride n2) on the raw voltages, times
//             the twiddle W_N^(n2 k1), then row FFTs of length n2; the
//             spectrum X[k1 + n1 k2] is left at position k1 n2 + k2;
//   inverse:  row IFFTs of length n2 on that transposed spectrum with the
//             chirp H_DM / Nfft multiplied in on load and W_N^(-n2 k1) on
//             store, then column IFFTs of length n1 that produce natural
//             time order, scattered to the owned, valid samples.
// The forward spectra do not depend on the DM and are computed once per
// FFT-length group; the inverse pair runs once per trial DM.
//
// Chirp phase (Eq. 1 integrated over frequency; FP64 only for the phase):
// the DM-independent table G = k_dm f^2/(f0^2 (f0+f)) is built in FP64, the
// per-DM phase c = DM G is formed and range-reduced (c - rint c) in FP64, and
// only the reduced fraction is converted to FP32 for sincospif.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "fft.cuh"
#include "internal.h"

namespace chirp {

static __device__ __forceinline__ Twiddles mk_tw(TwiddlePtrs p) {
  return Twiddles{p.coarse, p.fine, p.stage};
}

// ------------------------------------------------------------------ forward
// Column pass: L = n1, C = 4096 / n1 columns per CTA (interleaved tile).
// CI8: the voltages are complex int8 (re, im) times a per-antenna scale,
// converted to FP32 on load (the only read of the raw input).
template <int L, bool CI8>
__global__ void __launch_bounds__(256, 4) k_fwd_cols(const void* __restrict__ x, long long n_samp,
                                                  float2* __restrict__ spec, int n2, int log2n,
                                                  long long step, int n_ant,
                                                  const float* __restrict__ scale,
                                                  TwiddlePtrs twp, long long q0) {
  constexpr int C = 4096 / L;
  constexpr int T = L / 16;
  __shared__ float2 sm[FftTile<L, C>::SLOTS];
  const Twiddles tw = mk_tw(twp);
  const int s = threadIdx.x % C, jt = threadIdx.x / C;
  const int c = blockIdx.x * C + s;
  const bool act = c < n2;
  const long long q = q0 + blockIdx.y;  // block-major sequence: b * n_ant + a
  const long long a = q % n_ant, b = q / n_ant;
  const long long nfft = (long long)L * n2;
  const long long base = b * step;
  float2 v[16];
  if constexpr (CI8) {
    const char2* xa = (const char2*)x + a * n_samp;
    const float sc = scale ? scale[a] : 1.0f;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      long long n = base + (long long)(jt + k * T) * n2 + c;
      const char2 z = (act && n < n_samp) ? xa[n] : make_char2(0, 0);
      // rounded products, never fused into the first butterfly: the spectrum
      // equals that of the FP32 voltages scale * code
      v[k] = make_float2(__fmul_rn((float)z.x, sc), __fmul_rn((float)z.y, sc));
    }
  } else {
    const float2* xa = (const float2*)x + a * n_samp;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      long long n = base + (long long)(jt + k * T) * n2 + c;
      v[k] = (act && n < n_samp) ? xa[n] : make_float2(0.f, 0.f);
    }
  }
  fft_core<L, C, false, false>(v, sm, s, jt, tw);
  if (!act) return;
  float2* out = spec + q * nfft;
  // twiddle W_N^(c k1), k1 = jt + k T
  twiddle_run<false>(v, (unsigned)c, (unsigned)jt, (unsigned)T, log2n, tw);
#pragma unroll
  for (int k = 0; k < 16; k++) out[(long long)(jt + k * T) * n2 + c] = v[k];
}

// Row pass: L = n2, C = 4096 / L rows per CTA (row-major tile), in place.
template <int L>
__global__ void __launch_bounds__(256, 4) k_fwd_rows(float2* __restrict__ spec, int n1,
                                                  TwiddlePtrs twp) {
  constexpr int C = 4096 / L;
  constexpr int T = L / 16;
  __shared__ float2 sm[FftTile<L, C>::SLOTS];
  const Twiddles tw = mk_tw(twp);
  const int jt = threadIdx.x % T, s = threadIdx.x / T;
  const int k1 = blockIdx.x * C + s;
  const bool act = k1 < n1;
  const long long nfft = (long long)L * n1;
  float2* p = spec + (long long)blockIdx.y * nfft + (long long)k1 * L;
  float2 v[16];
#pragma unroll
  for (int k = 0; k < 16; k++) v[k] = act ? p[jt + k * T] : make_float2(0.f, 0.f);
  fft_core<L, C, true, false>(v, sm, s, jt, tw);
  if (!act) return;
#pragma unroll
  for (int k = 0; k < 16; k++) p[jt + k * T] = v[k];
}

// ------------------------------------------------------------------ table
__global__ void k_phase_table(double* __restrict__ G, long long nfft, int n1, int n2, double f0,
                              double bw, double k_dm) {
  long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= nfft) return;
  long long k1 = pos / n2, k2 = pos % n2;
  long long kf = k1 + (long long)n1 * k2;            // natural frequency index
  double fi = (double)(kf < nfft / 2 ? kf : kf - nfft);
  // f = fi B / Nfft; g = f^2 / (f0^2 (f0 + f)); G = k_dm g  (no fused ops)
  double f = __ddiv_rn(__dmul_rn(fi, bw), (double)nfft);
  double g = __ddiv_rn(__dmul_rn(f, f), __dmul_rn(__dmul_rn(f0, f0), __dadd_rn(f0, f)));
  G[pos] = __dmul_rn(k_dm, g);
}

// ------------------------------------------------------------------ chirp
// H[pos] = exp(-2 pi j frac(DM G[pos])) / Nfft for one trial DM, in the
// spectrum's order.  The product DM G and its reduction c - rint(c) are FP64
// (the phase reaches ~1e6 cycles at high DM); only the reduced fraction
// |r| <= 1/2 is rounded to FP32, and the chirp is stored as FP32 complex.
// The inverse transform's 1/Nfft rides on the chirp: Nfft is a power of two,
// so the scaling is exact and commutes with every rounding of the inverse
// FFT (the outputs equal those of scaling at the end, bit for bit).
__global__ void k_chirp_table(const double* __restrict__ G, float2* __restrict__ H, double dm,
                              long long nfft, float inv_nfft) {
  long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= nfft) return;
  double c = __dmul_rn(dm, G[pos]);
  double r = __dsub_rn(c, rint(c));  // exact
  float sn, cs;
  sincospif(-2.0f * (float)r, &sn, &cs);
  H[pos] = make_float2(cs * inv_nfft, sn * inv_nfft);
}

// The chirps of up to kMaxChirps DMs of one group in one pass over G (each
// element of G is read once); DM i's table goes to H + i h_stride.  Every
// value equals k_chirp_table's for the same DM.
struct ChirpDms {
  double dm[kMaxChirps];
};
// Grid-stride over the bins, so that a small grid can run beside other work.
__global__ void k_chirp_tables(const double* __restrict__ G, float2* __restrict__ H,
                               long long h_stride, ChirpDms dms, int n_dm, long long nfft,
                               float inv_nfft) {
  for (long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x; pos < nfft;
       pos += (long long)gridDim.x * blockDim.x) {
    const double gv = G[pos];
    for (int i = 0; i < n_dm; i++) {
      double c = __dmul_rn(dms.dm[i], gv);
      double r = __dsub_rn(c, rint(c));  // exact
      float sn, cs;
      sincospif(-2.0f * (float)r, &sn, &cs);
      H[i * h_stride + pos] = make_float2(cs * inv_nfft, sn * inv_nfft);
    }
  }
}

// ------------------------------------------------------------------ twiddles
// exp(-2 pi j e / n) from the exact fraction e / n (n a power of two), FP64
// with the argument reduced by sincospi, rounded once to FP32.
static __device__ __forceinline__ float2 unit_root(long long e, long long n) {
  double s, c;
  sincospi(-2.0 * (double)e / (double)n, &s, &c);
  return make_float2((float)c, (float)s);
}

__global__ void k_twiddles(float2* __restrict__ tw) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < 4096) {
    tw[m] = unit_root(m, 4096);
    tw[4096 + m] = unit_root(m, 1 << 24);
  }
  // stage pairs: span 16 at entries [0, 16), span 256 at [16, 272)
  if (m < kStageTwiddles) {
    const int ns = m < 16 ? 16 : 256, j = m < 16 ? m : m - 16;
    float4* st = reinterpret_cast<float4*>(tw + 8192);
    const float2 w1 = unit_root(j, 16LL * ns), w4 = unit_root(4LL * j, 16LL * ns);
    st[m] = make_float4(w1.x, w1.y, w4.x, w4.y);
  }
}

__global__ void k_row_twiddles(float2* __restrict__ rtw, int n1, int T, int log2n) {
  const long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= (long long)n1 * T) return;
  const long long k1 = pos / T, j = pos % T, n = 1LL << log2n;
  rtw[pos] = unit_root((k1 * j) & (n - 1), n);
}

// ------------------------------------------------------------------ inverse
// Row pass: X * H on load, IFFT of length L = n2, twiddle W_N^(-n2 k1) on
// store.  One CTA per (C rows, sequence); H comes from the per-DM table, the
// per-thread twiddle factor W_N^(k1 jt) from the group's row table.
// Per-DM block lists of one launch (grid dimension z = DM): DM j's
// sequences are its listed blocks' (n_seq[j] = listed blocks x antennas), or
// q0 .. q0 + n_seq[j] - 1 without a list.
struct RowLists {
  const int* blk_list[kMaxChirps];
  long long n_seq[kMaxChirps];
};

template <int L>
__global__ void __launch_bounds__(256, 4) k_inv_rows(const float2* __restrict__ spec,
                                                  float2* __restrict__ Z, long long z_stride,
                                                  const float2* __restrict__ H,
                                                  long long h_stride, int n1, int log2n,
                                                  long long q0,
                                                  const __grid_constant__ RowLists lists,
                                                  int n_ant, TwiddlePtrs twp,
                                                  const float2* __restrict__ rtw) {
  constexpr int C = 4096 / L;
  constexpr int T = L / 16;
  if (blockIdx.y >= lists.n_seq[blockIdx.z]) return;  // this DM lists fewer blocks
  const int* __restrict__ blk_list = lists.blk_list[blockIdx.z];
  Z += blockIdx.z * z_stride;
  H += blockIdx.z * h_stride;
  __shared__ float2 sm[FftTile<L, C>::SLOTS];
  const Twiddles tw = mk_tw(twp);
  const int jt = threadIdx.x % T, s = threadIdx.x / T;
  const int k1 = blockIdx.x * C + s;
  const bool act = k1 < n1;
  const long long nfft = (long long)L * n1;
  // sequence: q0 + y, or (listed block) * n_ant + antenna; Z holds the launch only
  const long long q = blk_list ? (long long)blk_list[blockIdx.y / n_ant] * n_ant + blockIdx.y % n_ant
                               : q0 + blockIdx.y;
  const float2* src = spec + q * nfft + (long long)k1 * L;
  const float2* h = H + (long long)k1 * L;
  float2 v[16];
#pragma unroll
  for (int k = 0; k < 16; k++)
    v[k] = act ? cmul(src[jt + k * T], __ldg(h + jt + k * T)) : make_float2(0.f, 0.f);
  fft_core<L, C, true, true>(v, sm, s, jt, tw);
  if (!act) return;
  float2* dst = Z + (long long)blockIdx.y * nfft + (long long)k1 * L;
  // twiddle W_N^(-k1 n2), n2 = jt + k T
  twiddle_run_base<true>(v, __ldg(rtw + (long long)k1 * T + jt), (unsigned)k1, (unsigned)T, log2n,
                         tw);
#pragma unroll
  for (int k = 0; k < 16; k++) dst[jt + k * T] = v[k];
}

// Row pass for n_dm trial DMs of one FFT-length group at once: the spectrum
// row is read from DRAM once (later DMs find it in L2) and multiplied by each
// DM's chirp in turn; DM d's rows go to Z + d * z_stride.  Saves up to half
// of the row pass's DRAM traffic (the spectrum read) for all but one DM.
// The sequence is the fast grid index, so the blocks that share the n_dm
// chirp rows of one row index run together and find them in L2 (with the
// sequence slow, n_dm whole chirp tables would have to stay in L2 beside the
// streamed spectra and outputs).
template <int L>
__global__ void __launch_bounds__(256, 4) k_inv_rows_multi(const float2* __restrict__ spec,
                                                        float2* __restrict__ Z, long long z_stride,
                                                        const float2* __restrict__ H,
                                                        long long h_stride, int n_dm, int n1,
                                                        int log2n, TwiddlePtrs twp,
                                                        const float2* __restrict__ rtw) {
  constexpr int C = 4096 / L;
  constexpr int T = L / 16;
  __shared__ float2 sm[FftTile<L, C>::SLOTS];
  const Twiddles tw = mk_tw(twp);
  const int jt = threadIdx.x % T, s = threadIdx.x / T;
  const int k1 = blockIdx.y * C + s;
  const bool act = k1 < n1;
  const long long nfft = (long long)L * n1;
  const float2* src = spec + (long long)blockIdx.x * nfft + (long long)k1 * L;
  for (int d = 0; d < n_dm; d++) {
    const float2* h = H + d * h_stride + (long long)k1 * L;
    float2 v[16];
#pragma unroll
    for (int k = 0; k < 16; k++)
      v[k] = act ? cmul(src[jt + k * T], __ldg(h + jt + k * T)) : make_float2(0.f, 0.f);
    fft_core<L, C, true, true>(v, sm, s, jt, tw);
    if (act) {
      float2* dst = Z + d * z_stride + (long long)blockIdx.x * nfft + (long long)k1 * L;
      twiddle_run_base<true>(v, __ldg(rtw + (long long)k1 * T + jt), (unsigned)k1, (unsigned)T,
                             log2n, tw);
#pragma unroll
      for (int k = 0; k < 16; k++) dst[jt + k * T] = v[k];
    }
    __syncthreads();  // sm is reused by the next DM's transform
  }
}

// Column pass of the inverse: natural-order output, overlap-save discard and
// ownership.  Block b owns block positions [lo_b, hi_b).
// IMG: instead of y, the owned samples inside [img.t0, img.t1) go to the
// beamformer's BF16 image (MN-major core matrices: a 16-byte row holds 8
// consecutive samples of one real component; head rounded to nearest BF16,
// tail the rounded remainder).  The values are staged in shared memory per
// component and written as whole rows where 8 consecutive samples are all
// owned and aligned (block starts are multiples of 8 samples), one real and
// one imaginary row together (32 bytes); elsewhere sample by sample.
template <int L, bool IMG>
__global__ void __launch_bounds__(256, 4) k_inv_cols(const float2* __restrict__ Z,
                                                  float2* __restrict__ y, long long n_samp,
                                                  int n2, long long step, long long n_blk,
                                                  int n_ant, long long n_hi, long long n_lo,
                                                  long long n_hi_max, long long q0,
                                                  const int* __restrict__ blk_list,
                                                  TwiddlePtrs twp, BeamImageOut img) {
  constexpr int C = 4096 / L;
  constexpr int T = L / 16;
  __shared__ __align__(16) float2 sm[FftTile<L, C>::SLOTS];
  const Twiddles tw = mk_tw(twp);
  int s, jt;
  col_thread<L, C>(threadIdx.x, s, jt);
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
  fft_core<L, C, false, true, kColShfl<L, C>>(v, sm, s, jt, tw);
  const long long base = b * step;
  const long long lo_b = (b == 0) ? n_hi : n_hi_max;
  const long long hi_b = (b == n_blk - 1) ? (n_samp - n_lo - base) : (n_hi_max + step);
  // (1/Nfft was applied with the chirp)
  if constexpr (IMG) {
    // staging [component][row][column] of BF16: components re_h, im_h (, re_l, im_l)
    __nv_bfloat16* stg = reinterpret_cast<__nv_bfloat16*>(sm);
    const int ncomp = img.terms == 3 ? 4 : 2;
    __syncthreads();  // every thread is done with the transform's exchanges
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const int row = jt + k * T;
      const float2 val = v[k];
      const __nv_bfloat162 h = __floats2bfloat162_rn(val.x, val.y);
      stg[(0 * L + row) * C + s] = h.x;
      stg[(1 * L + row) * C + s] = h.y;
      if (ncomp == 4) {
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(val.x - hf.x, val.y - hf.y);
        stg[(2 * L + row) * C + s] = l.x;
        stg[(3 * L + row) * C + s] = l.y;
      }
    }
    __syncthreads();
    // Owned positions inside the image's sample range: n in [nlo, nhi), at
    // image sample u = u_blk + n.  The image is [8-sample chunk][k-group]
    // [128 B] across its tiles, so chunk u >> 3 starts at (u >> 3) * grp_bytes.
    const long long nlo = lo_b > img.t0 - base ? lo_b : img.t0 - base;
    const long long nhi = hi_b < img.t1 - base ? hi_b : img.t1 - base;
    const long long u_blk = base - img.t0;
    const size_t grp_bytes = (size_t)img.GB * 128;
    // byte offset of antenna a's real row in a core-matrix column (imaginary: +16)
    const size_t a_ofs = (size_t)(a >> 2) * 128 + (size_t)(a & 3) * 32;
    const size_t tail_ofs = (size_t)img.G * 128;
    const int col_blk = blockIdx.x * C;
    if constexpr (C >= 8) {
      constexpr int CPR = C / 8;  // 8-sample chunks per row
      const int n_work = (ncomp / 2) * L * CPR;
      // Block positions n0 = row * n2 + col0 are multiples of 8, so a chunk
      // starts on an image chunk boundary when u_blk does; the owned range
      // clamped to [0, Nfft] fits 32 bits, and chunk addresses are offsets
      // from the block's first chunk.
      const bool aligned = (u_blk & 7) == 0;
      const int nlo32 = (int)(nlo < 0 ? 0 : (nlo > nfft ? nfft : nlo));
      const int nhi32 = (int)(nhi < 0 ? 0 : (nhi > nfft ? nfft : nhi));
      uint8_t* const dst_blk = img.img + a_ofs + (aligned ? (u_blk >> 3) * (long long)grp_bytes : 0);
      for (int w = threadIdx.x; w < n_work; w += 256) {
        const int j = w % CPR, rp = w / CPR;
        const int row = rp % L, pair = rp / L;  // pair 0: head, 1: tail
        const int col0 = col_blk + 8 * j;
        const int n0 = row * n2 + col0;  // < nfft <= 2^24
        const __nv_bfloat16* s_re = stg + ((2 * pair) * L + row) * C + 8 * j;
        const __nv_bfloat16* s_im = s_re + L * C;
        const size_t pofs = pair ? tail_ofs : 0;
        if (aligned && n0 >= nlo32 && n0 + 8 <= nhi32 && col0 + 8 <= n2) {
          // the real and imaginary rows are one 32-byte sector (32-byte
          // aligned: allocation base, 32-byte antenna rows, 128-byte groups):
          // one 256-bit store
          uint8_t* dst = dst_blk + pofs + (size_t)(n0 >> 3) * grp_bytes;
          const uint4 re = *reinterpret_cast<const uint4*>(s_re);
          const uint4 im = *reinterpret_cast<const uint4*>(s_im);
          asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                       :: "l"(dst), "r"(re.x), "r"(re.y), "r"(re.z), "r"(re.w), "r"(im.x),
                          "r"(im.y), "r"(im.z), "r"(im.w)
                       : "memory");
        } else if (n0 + 8 > nlo32 && n0 < nhi32) {
          uint8_t* dst0 = img.img + a_ofs + pofs;
          for (int e = 0; e < 8; e++) {
            const int n = n0 + e;
            if (col0 + e >= n2 || n < nlo32 || n >= nhi32) continue;
            const long long u = u_blk + n;
            uint8_t* dst = dst0 + (size_t)(u >> 3) * grp_bytes + (size_t)(u & 7) * 2;
            *reinterpret_cast<__nv_bfloat16*>(dst) = s_re[e];
            *reinterpret_cast<__nv_bfloat16*>(dst + 16) = s_im[e];
          }
        }
      }
    } else {
      // rows shorter than 8 samples: sample by sample from the staging
      const int n_work = (ncomp / 2) * L * C;
      for (int w = threadIdx.x; w < n_work; w += 256) {
        const int col = w % C, rp = w / C;
        const int row = rp % L, pair = rp / L;
        const int cc = col_blk + col;
        const long long n = (long long)(row * n2 + cc);
        if (cc >= n2 || n < nlo || n >= nhi) continue;
        const long long u = u_blk + n;
        uint8_t* dst = img.img + (size_t)(u >> 3) * grp_bytes + a_ofs + (pair ? tail_ofs : 0) +
                       (size_t)(u & 7) * 2;
        *reinterpret_cast<__nv_bfloat16*>(dst) = stg[((size_t)(2 * pair) * L + row) * C + col];
        *reinterpret_cast<__nv_bfloat16*>(dst + 16) = stg[((size_t)(2 * pair + 1) * L + row) * C + col];
      }
    }
  } else {
    if (!act) return;
    // the owned range clamped to [0, nfft] keeps every comparison 32-bit
    const int lo32 = (int)(lo_b < 0 ? 0 : (lo_b > nfft ? nfft : lo_b));
    const int hi32 = (int)(hi_b < 0 ? 0 : (hi_b > nfft ? nfft : hi_b));
    float2* yb = y + a * n_samp + base;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const int n = (jt + k * T) * n2 + c;
      if (n >= lo32 && n < hi32) yb[n] = v[k];
    }
  }
}

// ------------------------------------------------------------------ launchers
#define CHIRP_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

cudaError_t launch_forward(const void* x, long long n_samp, int n_ant, const GroupGeom& g,
                           float2* spec, TwiddlePtrs tw, cudaStream_t st, int in_type,
                           const float* scale, long long b0, long long b1) {
  if (b1 < 0) b1 = g.n_blk;
  if (b0 < 0 || b0 > b1 || b1 > g.n_blk) return cudaErrorInvalidValue;
  if (b0 == b1) return cudaSuccess;
  const long long q0 = b0 * n_ant;
  const long long n_seq = (long long)n_ant * (b1 - b0);
  if (n_seq > 65535) return cudaErrorInvalidConfiguration;
  {
    const int C = 4096 / g.n1;
    dim3 grid((g.n2 + C - 1) / C, (unsigned)n_seq);
    switch (g.n1) {
#define X(L)                                                                                   \
  case L:                                                                                      \
    if (in_type == 1)                                                                          \
      k_fwd_cols<L, true><<<grid, 256, 0, st>>>(x, n_samp, spec, g.n2, g.log2n, g.step, n_ant,  \
                                                scale, tw, q0);                                \
    else                                                                                       \
      k_fwd_cols<L, false><<<grid, 256, 0, st>>>(x, n_samp, spec, g.n2, g.log2n, g.step, n_ant, \
                                                 scale, tw, q0);                               \
    break;
      CHIRP_SIZES(X)
#undef X
      default: return cudaErrorInvalidValue;
    }
  }
  {
    const int C = 4096 / g.n2;
    dim3 grid((g.n1 + C - 1) / C, (unsigned)n_seq);
    float2* spec_q = spec + q0 * g.nfft;
    switch (g.n2) {
#define X(L) \
  case L: k_fwd_rows<L><<<grid, 256, 0, st>>>(spec_q, g.n1, tw); break;
      CHIRP_SIZES(X)
#undef X
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_build_phase_table(double* G, const GroupGeom& g, double f0, double bw,
                                     double k_dm, cudaStream_t st) {
  long long blocks = (g.nfft + 255) / 256;
  k_phase_table<<<(unsigned)blocks, 256, 0, st>>>(G, g.nfft, g.n1, g.n2, f0, bw, k_dm);
  return cudaGetLastError();
}

cudaError_t launch_chirp_tables(const double* G, float2* H, long long h_stride, const double* dms,
                                int n_dm, const GroupGeom& g, cudaStream_t st, int max_ctas) {
  if (n_dm < 1 || n_dm > kMaxChirps) return cudaErrorInvalidValue;
  ChirpDms d{};
  for (int i = 0; i < n_dm; i++) d.dm[i] = dms[i];
  long long blocks = (g.nfft + 255) / 256;
  if (max_ctas > 0 && blocks > max_ctas) blocks = max_ctas;
  k_chirp_tables<<<(unsigned)blocks, 256, 0, st>>>(G, H, h_stride, d, n_dm, g.nfft,
                                                   ldexpf(1.0f, -g.log2n));
  return cudaGetLastError();
}

cudaError_t launch_build_twiddles(float2* buf, cudaStream_t st) {
  k_twiddles<<<16, 256, 0, st>>>(buf);
  return cudaGetLastError();
}

cudaError_t launch_build_row_twiddles(float2* rtw, const GroupGeom& g, cudaStream_t st) {
  const long long n = (long long)g.n1 * (g.n2 / 16);
  k_row_twiddles<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rtw, g.n1, g.n2 / 16, g.log2n);
  return cudaGetLastError();
}

cudaError_t launch_chirp_table(const double* G, float2* H, double dm, const GroupGeom& g,
                               cudaStream_t st) {
  long long blocks = (g.nfft + 255) / 256;
  k_chirp_table<<<(unsigned)blocks, 256, 0, st>>>(G, H, dm, g.nfft, ldexpf(1.0f, -g.log2n));
  return cudaGetLastError();
}

static cudaError_t inverse_rows(const float2* spec, float2* Z, long long z_stride,
                                const float2* H, long long h_stride, int n_dm, long long q0,
                                const RowLists& lists, int n_ant, const GroupGeom& g,
                                TwiddlePtrs tw, const float2* rtw, cudaStream_t st) {
  if (n_dm < 1 || n_dm > kMaxChirps) return cudaErrorInvalidValue;
  long long nq = 0;
  for (int j = 0; j < n_dm; j++) nq = std::max(nq, lists.n_seq[j]);
  if (nq > 65535 || nq < 1) return cudaErrorInvalidConfiguration;
  const int C = 4096 / g.n2;
  dim3 grid((g.n1 + C - 1) / C, (unsigned)nq, (unsigned)n_dm);
  switch (g.n2) {
#define X(L) \
  case L: k_inv_rows<L><<<grid, 256, 0, st>>>(spec, Z, z_stride, H, h_stride, g.n1, g.log2n, q0, lists, n_ant, tw, rtw); break;
    CHIRP_SIZES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_inverse_rows(const float2* spec, float2* Z, const float2* H, long long q0,
                                long long nq, const GroupGeom& g, TwiddlePtrs tw,
                                const float2* rtw, cudaStream_t st, const int* blk_list,
                                int n_ant) {
  RowLists lists{};
  lists.blk_list[0] = blk_list;
  lists.n_seq[0] = nq;
  return inverse_rows(spec, Z, 0, H, 0, 1, q0, lists, n_ant, g, tw, rtw, st);
}

cudaError_t launch_inverse_rows_lists(const float2* spec, float2* Z, long long z_stride,
                                      const float2* H, long long h_stride, int n_dm,
                                      const int* const* blk_lists, const long long* n_list,
                                      int n_ant, const GroupGeom& g, TwiddlePtrs tw,
                                      const float2* rtw, cudaStream_t st) {
  if (n_dm < 1 || n_dm > kMaxChirps) return cudaErrorInvalidValue;
  RowLists lists{};
  for (int j = 0; j < n_dm; j++) {
    if (!blk_lists[j] || n_list[j] < 0) return cudaErrorInvalidValue;
    lists.blk_list[j] = blk_lists[j];
    lists.n_seq[j] = n_list[j] * n_ant;
  }
  return inverse_rows(spec, Z, z_stride, H, h_stride, n_dm, 0, lists, n_ant, g, tw, rtw, st);
}

cudaError_t launch_inverse_rows_multi(const float2* spec, float2* Z, long long z_stride,
                                      const float2* H, long long h_stride, int n_dm,
                                      long long nq, const GroupGeom& g, TwiddlePtrs tw,
                                      const float2* rtw, cudaStream_t st) {
  if (nq > 65535 || nq < 1 || n_dm < 1) return cudaErrorInvalidConfiguration;
  const int C = 4096 / g.n2;
  dim3 grid((unsigned)nq, (g.n1 + C - 1) / C);
  switch (g.n2) {
#define X(L) \
  case L: k_inv_rows_multi<L><<<grid, 256, 0, st>>>(spec, Z, z_stride, H, h_stride, n_dm, g.n1, g.log2n, tw, rtw); break;
    CHIRP_SIZES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_inverse_cols(const float2* Z, float2* y, long long n_samp, int n_ant,
                                long long q0, long long nq, const GroupGeom& g, long long n_hi,
                                long long n_lo, TwiddlePtrs tw, cudaStream_t st,
                                const int* blk_list, const BeamImageOut* img) {
  if (nq > 65535 || nq < 1) return cudaErrorInvalidConfiguration;
  const int C = 4096 / g.n1;
  dim3 grid((g.n2 + C - 1) / C, (unsigned)nq);
  const BeamImageOut io = img ? *img : BeamImageOut{nullptr, 0, 0, 0, 0, 0, 0};
  switch (g.n1) {
#define X(L)                                                                                    \
  case L:                                                                                       \
    if (img)                                                                                    \
      k_inv_cols<L, true><<<grid, 256, 0, st>>>(Z, y, n_samp, g.n2, g.step, g.n_blk, n_ant,     \
                                                n_hi, n_lo, g.n_hi_max, q0, blk_list, tw, io);  \
    else                                                                                        \
      k_inv_cols<L, false><<<grid, 256, 0, st>>>(Z, y, n_samp, g.n2, g.step, g.n_blk, n_ant,    \
                                                 n_hi, n_lo, g.n_hi_max, q0, blk_list, tw, io); \
    break;
    CHIRP_SIZES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

long long inverse_chunk_sequences(const GroupGeom& g, long long n_seq) {
  long long nq = kInverseChunkBytes / (g.nfft * (long long)sizeof(float2));
  if (nq < 1) nq = 1;
  if (nq > n_seq) nq = n_seq;
  return nq;
}

}  // namespace chirp
