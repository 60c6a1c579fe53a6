// cpi.cu -- the paper's own Chirpolator pre-integrator (Sec. 3, App. A.3) on
// the CUDA cores: pair mixing (Eq. xpq), block-based sliding DFT (Sec. A.3.2,
// Eq. block_cic) and imaging with the 2F+1-bin matched filter (Sec. 3.4,
// Eqs. pth and eth), for every trial DM.
//
// How the partial DFTs are evaluated.  V_k[m] depends on (k, N) only through
// the frequency f = k / N (cycles per sample), so every (trial DM, bin) with
// the same reduced fraction shares one V (this is the factorisation of
// Sec. A.3.3 in its block form: the DMs differ only in the length of the
// moving sum).  Each block is cut into sub-blocks of Ls samples with centre
// c; inside a sub-block exp(-2 pi j i f) = exp(-2 pi j c f) exp(-j theta u),
// u = (i - c) / (Ls / 2) in [-1, 1], theta = pi f Ls, and
//     sum_i x_i exp(-j theta u_i) = sum_j theta^j t_j,
//     t_j = (-j)^j / j! * sum_i u_i^j x_i        (Taylor series of exp),
// so one pass over the mixed samples gives J moments per (sub-block, pair)
// and every frequency is then a short polynomial in theta.  Ls is chosen so
// that theta <= 1/2 for the highest frequency and J so that the first
// dropped term is below 1e-9 of the sub-block's sum of |x| (far below FP32
// rounding).  The even and odd parts of the polynomial give f and -f
// together (the +-k sharing of Sec. A.3.4).
//
// Data layout (device):
//   T  [n_sub][J][n_pair]            float2  moments t_j
//   V  [n_vrow][n_blk][n_pair]       float2  partial DFTs; row 0: f = 0,
//                                            rows 1 + 2i / 2 + 2i: +f_i / -f_i
//   X  [n_dm][n_blk][2K+1][n_pair]   float2  window DFTs, window's own time
//   W  [n_dm][n_pair][2F+1][n_pix]   float2  matched filter, K0 its first bin
//   E  [n_dm][n_blk][n_pix]          float   |P|^2
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "../../include/chirp_gb300.h"
#include "internal.h"

using chirp::kCLight;
using chirp::kDefaultKdm;
using chirp::kPi;

namespace {

constexpr int kMaxTerms = 12;     // J
constexpr int kMaxBin = 64;       // K
constexpr int kMaxAnt = 84;
constexpr int kChunk = 64;        // samples staged per step of the moment pass
constexpr int kMaxSubPerBlk = 1024;
constexpr int kFreqPerThread = 8; // frequencies evaluated per thread (partial pass)
constexpr int kCicSeg = 256;      // blocks per thread of the moving sum
constexpr int kImgBlocks = 16;    // blocks per CTA of the imaging pass (even)
constexpr int kImgSmemBytes = 96 * 1024;

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {  // c + a b
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

// hi + lo += x with the rounding error of hi + x carried in lo (TwoSum)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float t = __fadd_rn(hi, x);
  const float bp = __fsub_rn(t, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  hi = t;
  lo = __fadd_rn(lo, e);
}

// ---------------------------------------------------------------- moments
// One CTA per sub-block s (R * n_pair threads rounded up to whole warps, at
// most 256): the antennas' samples [s Ls, (s+1) Ls) are staged kChunk at a
// time; item (pair, r) sums the samples i = r (mod R) of its pair's mixed
// series x_p x_q^* into J moments, the R partial sums of a pair are adjacent
// lanes and meet by shuffles.
__global__ void __launch_bounds__(256) k_cpi_moments(const float2* __restrict__ x, long long n_samp,
                                                     int n_ant, const short2* __restrict__ pairs,
                                                     int n_pair, int Ls, int J, int R,
                                                     float2* __restrict__ T) {
  __shared__ float2 xs[kMaxAnt * (kChunk + 1)];
  const long long s = blockIdx.x;
  const long long base = s * Ls;
  const int per = blockDim.x / R;  // pairs per pass (blockDim: a multiple of 32, <= 256)
  const float inv_ls = 1.0f / (float)Ls;  // a power of two: u below is exact
  for (int p0 = 0; p0 < n_pair; p0 += per) {
    const int item = threadIdx.x / R, r = threadIdx.x % R;
    const int pr = p0 + item;
    const bool act = item < per && pr < n_pair;
    short2 pq = act ? pairs[pr] : make_short2(0, 0);
    float2 acc[kMaxTerms];
#pragma unroll
    for (int j = 0; j < kMaxTerms; j++) acc[j] = make_float2(0.f, 0.f);
    for (int c0 = 0; c0 < Ls; c0 += kChunk) {
      const int cn = min(kChunk, Ls - c0);
      __syncthreads();
      for (int e = threadIdx.x; e < n_ant * cn; e += blockDim.x) {
        const int a = e / cn, i = e % cn;
        const long long t = base + c0 + i;
        xs[a * (kChunk + 1) + i] = t < n_samp ? x[(long long)a * n_samp + t] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      if (act) {
        // four samples per step: their power chains u^j run side by side
        int i = r;
        for (; i + 3 * R < cn; i += 4 * R) {
          float2 mx[4];
          float u[4], pw[4];
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const int ii = i + q * R;
            const float2 yp = xs[pq.x * (kChunk + 1) + ii], yq = xs[pq.y * (kChunk + 1) + ii];
            // x_pq = y_p conj(y_q) (Eq. xpq)
            mx[q] = make_float2(fmaf(yp.x, yq.x, yp.y * yq.y), fmaf(yp.y, yq.x, -yp.x * yq.y));
            u[q] = (float)(2 * (c0 + ii) - Ls + 1) * inv_ls;
            pw[q] = 1.f;
          }
#pragma unroll
          for (int j = 0; j < kMaxTerms; j++) {
            if (j < J) {
#pragma unroll
              for (int q = 0; q < 4; q++) {
                acc[j].x = fmaf(pw[q], mx[q].x, acc[j].x);
                acc[j].y = fmaf(pw[q], mx[q].y, acc[j].y);
                pw[q] *= u[q];
              }
            }
          }
        }
        for (; i < cn; i += R) {
          const float2 yp = xs[pq.x * (kChunk + 1) + i], yq = xs[pq.y * (kChunk + 1) + i];
          const float2 m = make_float2(fmaf(yp.x, yq.x, yp.y * yq.y), fmaf(yp.y, yq.x, -yp.x * yq.y));
          const float u = (float)(2 * (c0 + i) - Ls + 1) * inv_ls;
          float pw = 1.f;
#pragma unroll
          for (int j = 0; j < kMaxTerms; j++) {
            if (j < J) {
              acc[j].x = fmaf(pw, m.x, acc[j].x);
              acc[j].y = fmaf(pw, m.y, acc[j].y);
              pw *= u;
            }
          }
        }
      }
    }
    // R partial sums of one pair sit in adjacent lanes (R divides 32)
#pragma unroll
    for (int j = 0; j < kMaxTerms; j++)
      for (int o = R / 2; o > 0; o >>= 1) {
        acc[j].x += __shfl_xor_sync(0xffffffffu, acc[j].x, o);
        acc[j].y += __shfl_xor_sync(0xffffffffu, acc[j].y, o);
      }
    if (act && r == 0) {
      float fact = 1.f;
      for (int j = 0; j < J; j++) {
        if (j > 0) fact *= (float)j;
        const float inv = 1.f / fact;
        // (-j)^j: 1, -j, -1, +j
        float2 t;
        switch (j & 3) {
          case 0: t = make_float2(acc[j].x, acc[j].y); break;
          case 1: t = make_float2(acc[j].y, -acc[j].x); break;
          case 2: t = make_float2(-acc[j].x, -acc[j].y); break;
          default: t = make_float2(-acc[j].y, acc[j].x); break;
        }
        T[(s * J + j) * n_pair + pr] = make_float2(t.x * inv, t.y * inv);
      }
    }
  }
}

// ---------------------------------------------------------- partial DFTs
// Frequency descriptor: f = kp / (np L) cycles per sample (kp = 0: f = 0);
// kmin = the smallest |k| of the (DM, bin) cells that use it, so pair pq
// needs it only when kmin <= K_pq.
struct CpiFreq {
  int kp, np, kmin, pad;
};

// grid (frequency chunks, blocks).  Item (g, pair), g < G: frequencies
// chunk * G * kFreqPerThread + g * kFreqPerThread + c.  For each sub-block
// of the block the item reads its J moments once and evaluates all its
// frequencies: E = sum_{j even} t_j theta^j, O = sum_{j odd} t_j theta^j,
// V(+f) += ph (E + O), V(-f) += conj(ph) (E - O), ph = exp(-2 pi j c_s f),
// c_s = s Ls + (Ls - 1) / 2 the sub-block's centre.
__global__ void __launch_bounds__(256) k_cpi_partial(const float2* __restrict__ T,
                                                     const CpiFreq* __restrict__ freqs, int n_freq,
                                                     const int* __restrict__ kpair, int n_pair,
                                                     int L, int Ls, int J, int G, int n_blk,
                                                     int n_chunk, float2* __restrict__ V) {
  __shared__ float2 ph[kFreqPerThread * 32][17];  // [frequency of the CTA][sub-block] (chunks of 16)
  __shared__ float th[kFreqPerThread * 32];
  const int nsub = L / Ls;
  // frequency chunk fastest: the CTAs of one block run together and share its moments in L2
  const int chunk = (int)(blockIdx.x % n_chunk);
  const long long m = blockIdx.x / n_chunk;
  const int f_cta = G * kFreqPerThread;  // <= 256
  const int f0 = chunk * f_cta;
  const int g = threadIdx.x / n_pair, pr = threadIdx.x % n_pair;
  const bool act = g < G && pr < n_pair;
  // one pass per 256 pairs when n_pair > 256 (then G == 1)
  for (int p0 = 0; p0 < n_pair; p0 += 256) {
    const int pair = (n_pair > 256) ? p0 + threadIdx.x : pr;
    const bool act2 = (n_pair > 256) ? (p0 + (int)threadIdx.x < n_pair) : act;
    const int kp_lim = act2 ? kpair[pair] : -1;
    float2 vp[kFreqPerThread], vn[kFreqPerThread];
    bool need[kFreqPerThread];
#pragma unroll
    for (int c = 0; c < kFreqPerThread; c++) {
      vp[c] = vn[c] = make_float2(0.f, 0.f);
      const int fi = f0 + (n_pair > 256 ? 0 : g) * kFreqPerThread + c;
      need[c] = act2 && fi < n_freq && freqs[fi].kmin <= kp_lim;
    }
    for (int s0 = 0; s0 < nsub; s0 += 16) {
      const int sn = min(16, nsub - s0);
      __syncthreads();
      for (int e = threadIdx.x; e < f_cta * sn; e += 256) {
        const int fl = e / sn, sl = e % sn;
        const int fi = f0 + fl;
        float2 v = make_float2(1.f, 0.f);
        if (fi < n_freq && freqs[fi].kp != 0) {
          const CpiFreq fq = freqs[fi];
          const long long per2 = 2LL * fq.np * L;  // exp(-2 pi j c f) = exp(-pi j r / (np L))
          const long long s = m * nsub + s0 + sl;
          long long r = ((2 * s * Ls + Ls - 1) % per2) * fq.kp % per2;
          if (r >= per2 / 2) r -= per2;
          float sn_, cs_;
          sincospif((float)((double)r / (double)(per2 / 2)), &sn_, &cs_);
          v = make_float2(cs_, -sn_);
        }
        ph[fl][sl] = v;
        if (sl == 0)
          th[fl] = fi < n_freq ? (float)(kPi * (double)freqs[fi].kp * Ls / ((double)freqs[fi].np * L))
                               : 0.f;
      }
      __syncthreads();
      if (!act2) continue;
      for (int sl = 0; sl < sn; sl++) {
        const long long s = m * nsub + s0 + sl;
        float2 t[kMaxTerms];
#pragma unroll
        for (int j = 0; j < kMaxTerms; j++)
          t[j] = j < J ? T[(s * J + j) * n_pair + pair] : make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < kFreqPerThread; c++) {
          if (!need[c]) continue;
          const int fl = (n_pair > 256 ? 0 : g) * kFreqPerThread + c;
          const float tt = th[fl], t2 = tt * tt;
          float2 E = make_float2(0.f, 0.f), O = make_float2(0.f, 0.f);
#pragma unroll
          for (int j = kMaxTerms - 1; j >= 0; j--) {
            if ((j & 1) == 0) {
              E.x = fmaf(E.x, t2, t[j].x);
              E.y = fmaf(E.y, t2, t[j].y);
            } else {
              O.x = fmaf(O.x, t2, t[j].x);
              O.y = fmaf(O.y, t2, t[j].y);
            }
          }
          O.x *= tt;
          O.y *= tt;
          const float2 w = ph[fl][sl];
          const float2 a = make_float2(E.x + O.x, E.y + O.y);
          const float2 b = make_float2(E.x - O.x, E.y - O.y);
          vp[c] = cfma(w, a, vp[c]);
          vn[c] = cfma(make_float2(w.x, -w.y), b, vn[c]);
        }
      }
    }
    if (act2) {
#pragma unroll
      for (int c = 0; c < kFreqPerThread; c++) {
        if (!need[c]) continue;
        const int fi = f0 + (n_pair > 256 ? 0 : g) * kFreqPerThread + c;
        if (freqs[fi].kp == 0) {
          V[((long long)0 * n_blk + m) * n_pair + pair] = vp[c];
        } else {
          V[((long long)(2 * fi - 1) * n_blk + m) * n_pair + pair] = vp[c];
          V[((long long)(2 * fi) * n_blk + m) * n_pair + pair] = vn[c];
        }
      }
    }
  }
}

// ------------------------------------------------------------ moving sums
// Item (d, segment, bin, pair), pair fastest: the window DFTs of kCicSeg
// consecutive blocks.  The sum is started directly over the window that ends
// just before the segment and then advanced by Eq. block_cic, S[m] = S[m-1] + V[m] - V[m - n_win],
// in compensated FP32 (two floats per component); the result is moved to the
// window's own time,
// X[m] = exp(2 pi j (m + 1 - n_win) k / n_win) S[m] (a root of unity of order
// n_win, reduced exactly in integers).  Incomplete windows and bins beyond
// the pair's K_pq are zero.
__global__ void __launch_bounds__(256) k_cpi_cic(const float2* __restrict__ V,
                                                 const int* __restrict__ vrow,
                                                 const int* __restrict__ n_win,
                                                 const int* __restrict__ kpair, int n_pair, int K,
                                                 int n_dm, int n_blk, int n_seg,
                                                 float2* __restrict__ X) {
  const int nk = 2 * K + 1;
  const long long idx = (long long)blockIdx.x * 256 + threadIdx.x;
  const int pair = (int)(idx % n_pair);
  long long rest = idx / n_pair;
  const int kidx = (int)(rest % nk);
  rest /= nk;
  const int seg = (int)(rest % n_seg);
  const long long d = rest / n_seg;
  if (d >= n_dm) return;
  const int k = kidx - K;
  const int m0 = seg * kCicSeg, m1 = min(n_blk, m0 + kCicSeg);
  float2* out = X + ((d * n_blk) * nk + kidx) * n_pair + pair;
  const long long ostride = (long long)nk * n_pair;
  if (abs(k) > kpair[pair]) {
    for (int m = m0; m < m1; m++) out[m * ostride] = make_float2(0.f, 0.f);
    return;
  }
  const int nw = n_win[d];
  const float2* v = V + (long long)vrow[d * nk + kidx] * n_blk * n_pair + pair;
  // S[m0 - 1] = sum of V over blocks [m0 - n_win, m0 - 1], kept as an
  // unevaluated sum hi + lo of two floats per component (TwoSum, Knuth):
  // the running sum loses nothing to rounding over thousands of blocks
  // while staying on the FP32 pipes.
  float2 hi = make_float2(0.f, 0.f), lo = make_float2(0.f, 0.f);
  for (int mm = max(0, m0 - nw); mm < m0; mm++) {
    const float2 a = v[(long long)mm * n_pair];
    two_sum_acc(hi.x, lo.x, a.x);
    two_sum_acc(hi.y, lo.y, a.y);
  }
  // phase index r = ((m + 1) k) mod n_win, advanced by k each block
  const int kk = ((k % nw) + nw) % nw;
  int r = (int)(((long long)((m0 + 1) % nw) * kk) % nw);
  constexpr int U = 4;  // blocks per step: their loads are issued together
  for (int mu = m0; mu < m1; mu += U) {
    float2 add[U], sub[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int m = mu + u;
      add[u] = m < m1 ? v[(long long)m * n_pair] : make_float2(0.f, 0.f);
      sub[u] = (m < m1 && m - nw >= 0) ? v[(long long)(m - nw) * n_pair] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int m = mu + u;
      if (m >= m1) break;
      two_sum_acc(hi.x, lo.x, add[u].x);
      two_sum_acc(hi.y, lo.y, add[u].y);
      two_sum_acc(hi.x, lo.x, -sub[u].x);
      two_sum_acc(hi.y, lo.y, -sub[u].y);
      float2 o = make_float2(0.f, 0.f);
      if (m >= nw - 1) {
        const int r2 = 2 * r >= nw ? 2 * r - 2 * nw : 2 * r;  // phase pi r2 / nw in [-pi, pi)
        float sn, cs;
        sincospif((float)r2 / (float)nw, &sn, &cs);
        const float fr = hi.x + lo.x, fi = hi.y + lo.y;
        o = make_float2(fr * cs - fi * sn, fr * sn + fi * cs);
      }
      out[m * ostride] = o;
      r += kk;
      if (r >= nw) r -= nw;
    }
  }
}

// ---------------------------------------------------------------- imaging
// grid (pixel tiles of 512, block tiles of kImgBlocks, DM).  The window DFTs
// of the tile's blocks are staged pc pairs at a time as [pair][bin][block]
// rows of kImgBlocks + 2 float2 (144 bytes: lanes at different bins read
// different 16-byte bank groups).  Each thread is two adjacent pixels, whose
// filters cover nearly the same bins: per pair it walks the union of their
// 2F+1-bin ranges, reads each staged row once (128-bit loads, 8 blocks at a
// time) and adds it, times each pixel's weight for that bin (zero outside the
// pixel's range), to P of the tile's blocks (Eq. pth with the matched filter
// of Sec. 3.4); then E = |P|^2 (Eq. eth).
constexpr int kImgRow = kImgBlocks + 2;  // float2 per staged bin row
__global__ void __launch_bounds__(256) k_cpi_image(const float2* __restrict__ X,
                                                   const float2* __restrict__ W,
                                                   const short* __restrict__ K0,
                                                   const int* __restrict__ n_win, int n_pair,
                                                   int K, int F, int n_pix, int n_blk, int pc,
                                                   float* __restrict__ E) {
  extern __shared__ __align__(16) float2 xs[];  // [pair][bin][kImgRow]
  const int nk = 2 * K + 1, nj = 2 * F + 1;
  const long long d = blockIdx.z;
  const int m0 = blockIdx.y * kImgBlocks;
  const int mb = min(kImgBlocks, n_blk - m0);
  const int pa = blockIdx.x * 512 + 2 * threadIdx.x, pb = pa + 1;
  const bool va = pa < n_pix, vb = pb < n_pix;
  const int nw = n_win[d];
  float* e_out = E + (d * n_blk + m0) * n_pix;
  if (m0 + mb - 1 < nw - 1) {  // every window of the tile is incomplete
    for (int b = 0; b < mb; b++) {
      if (va) e_out[(long long)b * n_pix + pa] = 0.f;
      if (vb) e_out[(long long)b * n_pix + pb] = 0.f;
    }
    return;
  }
  float2 Pa[kImgBlocks], Pb[kImgBlocks];
#pragma unroll
  for (int b = 0; b < kImgBlocks; b++) Pa[b] = Pb[b] = make_float2(0.f, 0.f);
  for (int p0 = 0; p0 < n_pair; p0 += pc) {
    const int pn = min(pc, n_pair - p0);
    __syncthreads();
    for (int e = threadIdx.x; e < kImgBlocks * nk * pn; e += 256) {
      const int pl = e % pn, rest = e / pn;
      const int kidx = rest % nk, b = rest / nk;
      xs[(pl * nk + kidx) * kImgRow + b] =
          b < mb ? X[((d * n_blk + m0 + b) * nk + kidx) * n_pair + p0 + pl] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (va) {
      for (int pl = 0; pl < pn; pl++) {
        const long long dp = d * n_pair + p0 + pl;
        const int ka = K0[dp * n_pix + pa];
        const int kb = vb ? K0[dp * n_pix + pb] : ka;
        const int lo = min(ka, kb), hi = max(ka, kb) + nj;  // rows [lo, hi), within [0, nk)
        for (int r = lo; r < hi; r++) {
          const int ja = r - ka, jb = r - kb;
          const float2 wa = (ja >= 0 && ja < nj) ? W[(dp * nj + ja) * n_pix + pa] : make_float2(0.f, 0.f);
          const float2 wb = (vb && jb >= 0 && jb < nj) ? W[(dp * nj + jb) * n_pix + pb]
                                                       : make_float2(0.f, 0.f);
          const float4* row = reinterpret_cast<const float4*>(xs + (pl * nk + r) * kImgRow);
#pragma unroll
          for (int q = 0; q < kImgBlocks / 2; q++) {
            const float4 v = row[q];
            const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
            Pa[2 * q] = cfma(wa, v0, Pa[2 * q]);
            Pa[2 * q + 1] = cfma(wa, v1, Pa[2 * q + 1]);
            Pb[2 * q] = cfma(wb, v0, Pb[2 * q]);
            Pb[2 * q + 1] = cfma(wb, v1, Pb[2 * q + 1]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < kImgBlocks; b++) {  // static indices keep P in registers
    if (b < mb) {
      const bool ok = m0 + b >= nw - 1;
      if (va) e_out[(long long)b * n_pix + pa] = ok ? Pa[b].x * Pa[b].x + Pa[b].y * Pa[b].y : 0.f;
      if (vb) e_out[(long long)b * n_pix + pb] = ok ? Pb[b].x * Pb[b].x + Pb[b].y * Pb[b].y : 0.f;
    }
  }
}

// ---------------------------------------------------------- filter table
// Per (DM, pair, pixel), FP64: kappa = -fdot (tau_p - tau_q) N / B (Eq. f0Bt),
// k0' = rint(kappa), and for bins k = k0' - F .. k0' + F the conjugate of the
// response a unit linear chirp from the pixel's direction produces,
//   phi exp(-pi j kappa) exp(-pi j (k - kappa)(N - 1) / N) D_N(k - kappa),
//   phi = exp(pi j fdot (tau_p^2 - tau_q^2) - 2 pi j a0 (tau_p - tau_q)),
// times D_N(k - kappa) / N (Eq. dn).  A filter whose bins fall outside
// [-K, K] is zero (K0 then points at bin -K).
__global__ void k_cpi_weights(const double* __restrict__ tau, int n_ant,
                              const short2* __restrict__ pairs, int n_pair,
                              const double* __restrict__ dmc, int n_dm, int n_pix, double bw,
                              int F, int K, short* __restrict__ K0, float2* __restrict__ W) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)n_dm * n_pair * n_pix;
  if (idx >= total) return;
  const int pix = (int)(idx % n_pix);
  const long long dp = idx / n_pix;
  const int pair = (int)(dp % n_pair);
  const int d = (int)(dp / n_pair);
  const double a0 = dmc[3 * d], a1 = dmc[3 * d + 1], N = dmc[3 * d + 2];
  const short2 pq = pairs[pair];
  const double tp = tau[(long long)pix * n_ant + pq.x], tq = tau[(long long)pix * n_ant + pq.y];
  const double dt = tp - tq;
  const double kap = -a1 * dt * N / bw;
  const double kc = rint(kap);
  const int nj = 2 * F + 1;
  const long long first = (long long)kc - F + K;
  const bool ok = first >= 0 && first + 2 * F <= 2 * K;
  K0[dp * n_pix + pix] = (short)(ok ? first : 0);
  const double base = 0.5 * a1 * (tp * tp - tq * tq) - a0 * dt - 0.5 * kap;  // cycles
  for (int j = 0; j < nj; j++) {
    float2 w = make_float2(0.f, 0.f);
    if (ok) {
      const double x = kc - F + j - kap;
      double cyc = base - 0.5 * x * (N - 1.0) / N;
      cyc -= rint(cyc);
      double s, c;
      sincospi(2.0 * cyc, &s, &c);
      const double dn = fabs(x) < 1e-12 ? 1.0 : sinpi(x) / (N * sinpi(x / N));
      w = make_float2((float)(c * dn), (float)(-s * dn));
    }
    W[(dp * nj + j) * n_pix + pix] = w;
  }
}

// ------------------------------------------------------- spectra export
// Vout[d][m][k + K][pair] = V[vrow[d][k + K]][m][pair] for |k| <= K_pq, else 0.
__global__ void k_cpi_expand_v(const float2* __restrict__ V, const int* __restrict__ vrow,
                               const int* __restrict__ kpair, int n_pair, int K, int n_dm,
                               long long n_blk, float2* __restrict__ out) {
  const int nk = 2 * K + 1;
  const long long total = (long long)n_dm * n_blk * nk * n_pair;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int pair = (int)(i % n_pair);
    long long r = i / n_pair;
    const int kidx = (int)(r % nk);
    r /= nk;
    const long long m = r % n_blk, d = r / n_blk;
    out[i] = abs(kidx - K) <= kpair[pair] ? V[((long long)vrow[d * nk + kidx] * n_blk + m) * n_pair + pair]
                                          : make_float2(0.f, 0.f);
  }
}

int cfail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return chirp_report_error(code, buf);
}

#define CKC(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return cfail(CHIRP_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                   __FILE__, __LINE__);                                                    \
  } while (0)

long long gcd_ll(long long a, long long b) {
  while (b) {
    const long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace

struct chirp_cpi_plan {
  int M = 0, n_pair = 0, n_pix = 0, n_dm = 0, F = 0, K = 0, L = 0;
  int Ls = 1, J = 1, R = 1, G = 1, pc = 1, n_freq = 0, n_seg = 0, n_chunk = 0;
  long long N = 0, n_blk = 0, n_sub = 0;
  double f0 = 0, bw = 0, kdm = 0;
  std::vector<double> dm, a0, fdot;
  std::vector<int> n_win, kpq, vrow;
  std::vector<short2> pairs;
  std::vector<CpiFreq> freqs;
  cudaStream_t st = nullptr;
  float2 *d_x = nullptr, *d_T = nullptr, *d_V = nullptr, *d_X = nullptr, *d_W = nullptr;
  short* d_K0 = nullptr;
  float* d_E = nullptr;
  int image_mode = 0;              // 0: tensor-core dense image, 1: CUDA-core gathers
  uint8_t *d_aimg = nullptr, *d_bimg = nullptr;  // tensor-core operand images
  int* d_err = nullptr;            // device status word of the tensor-core pass
  CpiFreq* d_freq = nullptr;
  int *d_vrow = nullptr, *d_nwin = nullptr, *d_kpq = nullptr;
  short2* d_pairs = nullptr;
  long long work_bytes = 0;
  cudaEvent_t ev[5] = {};
  bool timed = false;
};

namespace {

void free_plan(chirp_cpi_plan* p) {
  if (!p) return;
  void* bufs[] = {p->d_x,    p->d_T,    p->d_V,    p->d_X,     p->d_W,    p->d_K0,
                  p->d_E,    p->d_freq, p->d_vrow, p->d_nwin,  p->d_kpq,  p->d_pairs,
                  p->d_aimg, p->d_bimg, p->d_err};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  delete p;
}

int alloc(chirp_cpi_plan* p, void** ptr, long long bytes, const char* what) {
  if (cudaMalloc(ptr, (size_t)std::max(bytes, 16LL)) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return cfail(CHIRP_ENOMEM, "device allocation of %lld bytes (%s) failed", bytes, what);
  }
  p->work_bytes += bytes;
  return CHIRP_OK;
}

// Host planning in FP64: pairs, per-DM chirp model and window, per-pair bins,
// the distinct frequencies and the Taylor evaluation's sub-block and terms.
int plan_host(chirp_cpi_plan* p, const chirp_cpi_config* c, std::vector<double>& tau,
              std::vector<double>& dmc) {
  if (c->n_ant < 2 || c->n_ant > kMaxAnt) return cfail(CHIRP_EINVAL, "n_ant must be in 2..84");
  if (!c->xyz_m || !c->dm || !c->pix_lm) return cfail(CHIRP_EINVAL, "xyz_m, dm and pix_lm are required");
  if (!(c->bw_hz > 0) || !(c->f0_hz > 0.5 * c->bw_hz))
    return cfail(CHIRP_EINVAL, "need bw_hz > 0 and f0_hz > bw_hz / 2");
  if (c->blk_len < 16 || c->blk_len > 65536 || (c->blk_len & (c->blk_len - 1)))
    return cfail(CHIRP_EINVAL, "blk_len must be a power of two in 16..65536");
  if (c->n_samp < c->blk_len) return cfail(CHIRP_EINVAL, "n_samp must be >= blk_len");
  if (c->n_dm < 1 || c->n_dm > 65535 || c->n_pix < 1)
    return cfail(CHIRP_EINVAL, "n_dm must be in 1..65535 and n_pix >= 1");
  if (c->half_width < 0 || c->half_width > 8) return cfail(CHIRP_EINVAL, "half_width must be in 0..8");
  if (c->max_bin < 0 || c->max_bin > kMaxBin) return cfail(CHIRP_EINVAL, "max_bin must be in 0..64");
  if (c->image_mode != 0 && c->image_mode != 1) return cfail(CHIRP_EINVAL, "image_mode must be 0 or 1");
  p->image_mode = c->image_mode;
  p->M = c->n_ant;
  p->f0 = c->f0_hz;
  p->bw = c->bw_hz;
  p->kdm = c->k_dm > 0 ? c->k_dm : kDefaultKdm;
  p->N = c->n_samp;
  p->L = c->blk_len;
  p->n_blk = c->n_samp / c->blk_len;
  if (p->n_blk > 65535LL * kImgBlocks) return cfail(CHIRP_EINVAL, "more than 1048560 blocks");
  p->n_dm = c->n_dm;
  p->n_pix = c->n_pix;
  p->F = c->half_width;
  for (int a = 0; a < p->M; a++)
    for (int b = a + 1; b < p->M; b++) p->pairs.push_back(make_short2((short)a, (short)b));
  p->n_pair = (int)p->pairs.size();
  const double nu_lo = p->f0 - 0.5 * p->bw, nu_hi = p->f0 + 0.5 * p->bw;
  for (int d = 0; d < p->n_dm; d++) {
    const double dm = c->dm[d];
    if (!(dm > 0) || !std::isfinite(dm)) return cfail(CHIRP_EINVAL, "trial DM %d must be > 0", d);
    const double T = p->kdm * dm * (1.0 / (nu_lo * nu_lo) - 1.0 / (nu_hi * nu_hi));
    const double alpha = 0.5 * (1.0 / (nu_lo * nu_lo) + 1.0 / (nu_hi * nu_hi));
    const double w = std::floor(p->bw * T / p->L + 0.5);
    if (w > (double)p->n_blk)
      return cfail(CHIRP_EINVAL, "the sweep of DM %g (%g blocks) is longer than the data", dm, w);
    p->dm.push_back(dm);
    p->a0.push_back(1.0 / std::sqrt(alpha));
    p->fdot.push_back(-0.5 / (alpha * std::sqrt(alpha)) / (p->kdm * dm));
    p->n_win.push_back(std::max(1, (int)w));
    dmc.push_back(p->a0.back());
    dmc.push_back(p->fdot.back());
    dmc.push_back((double)p->n_win.back() * p->L);
  }
  // delays (Eq. tau3D) and the bins each pair needs
  tau.resize((size_t)p->n_pix * p->M);
  for (int i = 0; i < p->n_pix; i++) {
    const double l = c->pix_lm[2 * i], m = c->pix_lm[2 * i + 1];
    if (!(l * l + m * m <= 1.0)) return cfail(CHIRP_EINVAL, "pixel %d has l^2 + m^2 > 1", i);
    const double n = std::sqrt(std::max(0.0, 1.0 - l * l - m * m));
    for (int a = 0; a < p->M; a++) {
      const double* r = c->xyz_m + 3 * a;
      tau[(size_t)i * p->M + a] = (r[0] * l + r[1] * m + r[2] * (n - 1.0)) / kCLight;
    }
  }
  p->kpq.assign(p->n_pair, 0);
  for (int d = 0; d < p->n_dm; d++) {
    const double Nd = (double)p->n_win[d] * p->L;
    for (int i = 0; i < p->n_pix; i++)
      for (int q = 0; q < p->n_pair; q++) {
        const double dt = tau[(size_t)i * p->M + p->pairs[q].x] - tau[(size_t)i * p->M + p->pairs[q].y];
        const double kc = std::fabs(std::rint(-p->fdot[d] * dt * Nd / p->bw));
        if (kc > 1e6) return cfail(CHIRP_EINVAL, "a pixel's tone is beyond any bin range");
        p->kpq[q] = std::max(p->kpq[q], (int)kc + p->F);
      }
  }
  const int need = *std::max_element(p->kpq.begin(), p->kpq.end());
  if (need > kMaxBin) return cfail(CHIRP_EINVAL, "the pixels need bins up to %d (> 64)", need);
  if (c->max_bin > 0 && c->max_bin < need)
    return cfail(CHIRP_EINVAL, "max_bin %d is below the %d the pixels need", c->max_bin, need);
  p->K = c->max_bin > 0 ? c->max_bin : need;
  // distinct frequencies k / (n_win L) as reduced fractions
  const int nk = 2 * p->K + 1;
  std::map<std::pair<long long, long long>, int> ids;
  p->freqs.push_back(CpiFreq{0, 1, 0, 0});
  p->vrow.assign((size_t)p->n_dm * nk, 0);
  double fmax = 0.0;
  for (int d = 0; d < p->n_dm; d++)
    for (int k = 1; k <= p->K; k++) {
      const long long g = gcd_ll(k, p->n_win[d]);
      const auto key = std::make_pair((long long)k / g, (long long)p->n_win[d] / g);
      auto it = ids.find(key);
      int id;
      if (it == ids.end()) {
        id = (int)p->freqs.size();
        ids.emplace(key, id);
        p->freqs.push_back(CpiFreq{(int)key.first, (int)key.second, k, 0});
        fmax = std::max(fmax, (double)key.first / ((double)key.second * p->L));
      } else {
        id = it->second;
        p->freqs[id].kmin = std::min(p->freqs[id].kmin, k);
      }
      p->vrow[(size_t)d * nk + p->K + k] = 2 * id - 1;
      p->vrow[(size_t)d * nk + p->K - k] = 2 * id;
    }
  p->n_freq = (int)p->freqs.size();
  // Taylor evaluation: theta = pi f Ls <= 1/2, first dropped term <= 1e-9
  p->Ls = std::min(p->L, 256);
  while (p->Ls > 1 && kPi * fmax * p->Ls > 0.5) p->Ls /= 2;
  if (p->L / p->Ls > kMaxSubPerBlk)
    return cfail(CHIRP_EUNSUPPORTED, "the bins need sub-blocks of %d samples (> 1024 per block)", p->Ls);
  const double th = kPi * fmax * p->Ls;
  p->J = 1;
  if (p->Ls > 1 && th > 0) {
    double t = th;  // theta^J / J!
    while (t > 1e-9 && p->J < kMaxTerms) {
      p->J++;
      t *= th / p->J;
    }
  }
  p->n_sub = p->n_blk * (p->L / p->Ls);
  while (p->R < 8 && 2 * p->R * p->n_pair <= 256) p->R *= 2;
  p->G = p->n_pair <= 256 ? std::min(32, 256 / p->n_pair) : 1;
  p->n_chunk = (p->n_freq + p->G * kFreqPerThread - 1) / (p->G * kFreqPerThread);
  p->pc = std::max(1, std::min(p->n_pair, kImgSmemBytes / ((kImgBlocks + 2) * nk * (int)sizeof(float2))));
  p->n_seg = (int)((p->n_blk + kCicSeg - 1) / kCicSeg);
  const long long cic_ctas = ((long long)p->n_dm * p->n_seg * nk * p->n_pair + 255) / 256;
  if (p->n_sub >= (1LL << 31) || (long long)p->n_chunk * p->n_blk >= (1LL << 31) ||
      cic_ctas >= (1LL << 31))
    return cfail(CHIRP_EUNSUPPORTED, "the search needs more than 2^31 CTAs in one pass");
  return CHIRP_OK;
}

}  // namespace

namespace {

// The four passes on the plan's stream; the image is skipped when E is NULL.
int cpi_enqueue(chirp_cpi_plan* p, const void* volt, int volt_loc, float* E) {
  if (!volt) return cfail(CHIRP_EINVAL, "voltages are NULL");
  if (volt_loc != CHIRP_HOST && volt_loc != CHIRP_DEVICE) return cfail(CHIRP_EINVAL, "bad volt_loc");
  const float2* x = static_cast<const float2*>(volt);
  if (volt_loc == CHIRP_HOST) {
    if (!p->d_x) {
      int rc = alloc(p, (void**)&p->d_x, (long long)p->M * p->N * 8, "voltages");
      if (rc) return rc;
    }
    CKC(cudaMemcpyAsync(p->d_x, volt, (size_t)p->M * p->N * 8, cudaMemcpyHostToDevice, p->st));
    x = p->d_x;
  }
  const int nk = 2 * p->K + 1;
  CKC(cudaEventRecord(p->ev[0], p->st));
  const int mom_threads = std::min(256, (p->R * p->n_pair + 31) / 32 * 32);
  k_cpi_moments<<<(unsigned)p->n_sub, mom_threads, 0, p->st>>>(x, p->N, p->M, p->d_pairs, p->n_pair,
                                                               p->Ls, p->J, p->R, p->d_T);
  CKC(cudaGetLastError());
  CKC(cudaEventRecord(p->ev[1], p->st));
  k_cpi_partial<<<(unsigned)((long long)p->n_chunk * p->n_blk), 256, 0, p->st>>>(
      p->d_T, p->d_freq, p->n_freq, p->d_kpq, p->n_pair, p->L, p->Ls, p->J, p->G, (int)p->n_blk,
      p->n_chunk, p->d_V);
  CKC(cudaGetLastError());
  CKC(cudaEventRecord(p->ev[2], p->st));
  const long long items = (long long)p->n_dm * p->n_seg * nk * p->n_pair;
  k_cpi_cic<<<(unsigned)((items + 255) / 256), 256, 0, p->st>>>(
      p->d_V, p->d_vrow, p->d_nwin, p->d_kpq, p->n_pair, p->K, p->n_dm, (int)p->n_blk, p->n_seg,
      p->d_X);
  CKC(cudaGetLastError());
  CKC(cudaEventRecord(p->ev[3], p->st));
  if (E && p->image_mode == 0) {
    CKC(chirp::launch_cpi_tc_image(p->d_X, p->d_bimg, p->d_aimg, p->d_nwin, p->n_dm, p->n_blk, nk,
                                   p->n_pair, p->n_pix, E, p->d_err, p->st));
  } else if (E) {
    const dim3 grid((unsigned)((p->n_pix + 511) / 512), (unsigned)((p->n_blk + kImgBlocks - 1) / kImgBlocks),
                    (unsigned)p->n_dm);
    k_cpi_image<<<grid, 256, kImgSmemBytes, p->st>>>(p->d_X, p->d_W, p->d_K0, p->d_nwin, p->n_pair,
                                                     p->K, p->F, p->n_pix, (int)p->n_blk, p->pc, E);
    CKC(cudaGetLastError());
  }
  CKC(cudaEventRecord(p->ev[4], p->st));
  p->timed = E != nullptr;
  return CHIRP_OK;
}

// After a synchronisation: CHIRP_ETIMEOUT when a bounded wait of the
// tensor-core image pass gave up (its outputs are then invalid).
int cpi_status(chirp_cpi_plan* p) {
  if (!p->d_err) return CHIRP_OK;
  int flag = 0;
  CKC(cudaMemcpy(&flag, p->d_err, 4, cudaMemcpyDeviceToHost));
  if (flag) return cfail(CHIRP_ETIMEOUT, "a bounded wait of the tensor-core image pass gave up");
  return CHIRP_OK;
}

}  // namespace

extern "C" {

int chirp_cpi_create(chirp_cpi_plan** out, const chirp_cpi_config* cfg, void* stream) {
  if (!out) return cfail(CHIRP_EINVAL, "plan pointer is NULL");
  *out = nullptr;
  if (!cfg) return cfail(CHIRP_EINVAL, "config is NULL");
  chirp_cpi_plan* p = new (std::nothrow) chirp_cpi_plan();
  if (!p) return cfail(CHIRP_ENOMEM, "host allocation failed");
  p->st = (cudaStream_t)stream;
  std::vector<double> tau, dmc;
  int rc = plan_host(p, cfg, tau, dmc);
  if (rc) {
    free_plan(p);
    return rc;
  }
  const int nk = 2 * p->K + 1, nj = 2 * p->F + 1;
  const long long n_vrow = 2LL * p->n_freq - 1;
  double* d_tau = nullptr;
  double* d_dmc = nullptr;
  struct A { void** ptr; long long bytes; const char* what; } allocs[] = {
      {(void**)&p->d_T, p->n_sub * p->J * p->n_pair * 8, "moments"},
      {(void**)&p->d_V, n_vrow * p->n_blk * p->n_pair * 8, "partial DFTs"},
      {(void**)&p->d_X, (long long)p->n_dm * p->n_blk * nk * p->n_pair * 8, "window DFTs"},
      {(void**)&p->d_W, (long long)p->n_dm * p->n_pair * nj * p->n_pix * 8, "filter"},
      {(void**)&p->d_K0, (long long)p->n_dm * p->n_pair * p->n_pix * 2, "filter bins"},
      {(void**)&p->d_freq, (long long)p->n_freq * (long long)sizeof(CpiFreq), "frequencies"},
      {(void**)&p->d_vrow, (long long)p->n_dm * nk * 4, "rows"},
      {(void**)&p->d_nwin, (long long)p->n_dm * 4, "windows"},
      {(void**)&p->d_kpq, (long long)p->n_pair * 4, "pair bins"},
      {(void**)&p->d_pairs, (long long)p->n_pair * 4, "pairs"},
  };
  for (auto& a : allocs) {
    rc = alloc(p, a.ptr, a.bytes, a.what);
    if (rc) {
      free_plan(p);
      return rc;
    }
  }
  if (cudaMalloc((void**)&d_tau, tau.size() * 8) != cudaSuccess ||
      cudaMalloc((void**)&d_dmc, dmc.size() * 8) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_tau);
    cudaFree(d_dmc);
    free_plan(p);
    return cfail(CHIRP_ENOMEM, "device allocation of the delay table failed");
  }
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t n) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, p->st);
  };
  up(p->d_freq, p->freqs.data(), p->freqs.size() * sizeof(CpiFreq));
  up(p->d_vrow, p->vrow.data(), p->vrow.size() * 4);
  up(p->d_nwin, p->n_win.data(), p->n_win.size() * 4);
  up(p->d_kpq, p->kpq.data(), p->kpq.size() * 4);
  up(p->d_pairs, p->pairs.data(), p->pairs.size() * 4);
  up(d_tau, tau.data(), tau.size() * 8);
  up(d_dmc, dmc.data(), dmc.size() * 8);
  if (e == cudaSuccess) {
    const long long total = (long long)p->n_dm * p->n_pair * p->n_pix;
    k_cpi_weights<<<(unsigned)((total + 255) / 256), 256, 0, p->st>>>(
        d_tau, p->M, p->d_pairs, p->n_pair, d_dmc, p->n_dm, p->n_pix, p->bw, p->F, p->K, p->d_K0,
        p->d_W);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cpi_image, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 kImgSmemBytes);
  if (e == cudaSuccess && p->image_mode == 0) {
    // the dense split-BF16 filter of every DM, built once from the sparse one
    const int nk = 2 * p->K + 1;
    rc = alloc(p, (void**)&p->d_aimg, chirp::cpi_tc_a_bytes(p->n_dm, p->n_pix, nk, p->n_pair),
               "tensor-core filter image");
    if (!rc) rc = alloc(p, (void**)&p->d_bimg, chirp::cpi_tc_b_bytes(p->n_dm, p->n_blk, nk, p->n_pair),
                        "tensor-core window-DFT image");
    if (!rc) rc = alloc(p, (void**)&p->d_err, 4, "status word");
    if (rc) {
      cudaStreamSynchronize(p->st);
      cudaFree(d_tau);
      cudaFree(d_dmc);
      free_plan(p);
      return rc;
    }
    e = cudaMemsetAsync(p->d_err, 0, 4, p->st);
    if (e == cudaSuccess)
      e = chirp::launch_cpi_tc_aimg(p->d_W, p->d_K0, p->n_dm, p->n_pair, 2 * p->F + 1, nk, p->n_pix,
                                    p->d_aimg, p->st);
  }
  for (auto& ev : p->ev)
    if (e == cudaSuccess) e = cudaEventCreate(&ev);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);  // the host tables above die here
  cudaFree(d_tau);
  cudaFree(d_dmc);
  if (e != cudaSuccess) {
    free_plan(p);
    return cfail(CHIRP_ECUDA, "plan setup failed: %s", cudaGetErrorString(e));
  }
  *out = p;
  return CHIRP_OK;
}

int chirp_cpi_query(const chirp_cpi_plan* p, chirp_cpi_info* info) {
  if (!p || !info) return cfail(CHIRP_EINVAL, "NULL argument");
  info->n_pair = p->n_pair;
  info->n_blk = p->n_blk;
  info->max_bin = p->K;
  info->n_freq = p->n_freq;
  info->sub_len = p->Ls;
  info->n_terms = p->J;
  info->work_bytes = p->work_bytes;
  return CHIRP_OK;
}

int chirp_cpi_layout(const chirp_cpi_plan* p, int d, int* n_win, double* fdot, int* pair_bins) {
  if (!p || d < 0 || d >= p->n_dm) return cfail(CHIRP_EINVAL, "bad plan or DM index");
  if (n_win) *n_win = p->n_win[d];
  if (fdot) *fdot = p->fdot[d];
  if (pair_bins) std::memcpy(pair_bins, p->kpq.data(), p->kpq.size() * sizeof(int));
  return CHIRP_OK;
}

int chirp_cpi_run(chirp_cpi_plan* p, const void* volt, int volt_loc, float* energy, int out_loc) {
  if (!p || !energy) return cfail(CHIRP_EINVAL, "NULL argument");
  if (out_loc != CHIRP_HOST && out_loc != CHIRP_DEVICE) return cfail(CHIRP_EINVAL, "bad out_loc");
  const long long n_out = (long long)p->n_dm * p->n_blk * p->n_pix;
  float* E = energy;
  if (out_loc == CHIRP_HOST) {
    if (!p->d_E) {
      int rc = alloc(p, (void**)&p->d_E, n_out * 4, "image");
      if (rc) return rc;
    }
    E = p->d_E;
  }
  int rc = cpi_enqueue(p, volt, volt_loc, E);
  if (rc) return rc;
  if (out_loc == CHIRP_HOST) {
    CKC(cudaMemcpyAsync(energy, E, (size_t)n_out * 4, cudaMemcpyDeviceToHost, p->st));
    CKC(cudaStreamSynchronize(p->st));
    return cpi_status(p);
  }
  return CHIRP_OK;
}

int chirp_cpi_spectra(chirp_cpi_plan* p, const void* volt, int volt_loc, void* V, void* X,
                      int out_loc) {
  if (!p) return cfail(CHIRP_EINVAL, "plan is NULL");
  if (out_loc != CHIRP_HOST && out_loc != CHIRP_DEVICE) return cfail(CHIRP_EINVAL, "bad out_loc");
  int rc = cpi_enqueue(p, volt, volt_loc, nullptr);
  if (rc) return rc;
  const int nk = 2 * p->K + 1;
  const long long n = (long long)p->n_dm * p->n_blk * nk * p->n_pair;
  const cudaMemcpyKind kind = out_loc == CHIRP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (X) CKC(cudaMemcpyAsync(X, p->d_X, (size_t)n * 8, kind, p->st));
  if (V) {
    float2* dv = static_cast<float2*>(V);
    if (out_loc == CHIRP_HOST) {
      CKC(cudaMalloc((void**)&dv, (size_t)n * 8));
    }
    k_cpi_expand_v<<<2048, 256, 0, p->st>>>(p->d_V, p->d_vrow, p->d_kpq, p->n_pair, p->K, p->n_dm,
                                            p->n_blk, dv);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && out_loc == CHIRP_HOST) {
      e = cudaMemcpyAsync(V, dv, (size_t)n * 8, cudaMemcpyDeviceToHost, p->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
      cudaFree(dv);
    }
    if (e != cudaSuccess) return cfail(CHIRP_ECUDA, "spectra export failed: %s", cudaGetErrorString(e));
  }
  if (out_loc == CHIRP_HOST) CKC(cudaStreamSynchronize(p->st));
  return CHIRP_OK;
}

int chirp_cpi_timing(chirp_cpi_plan* p, double ms[4]) {
  if (!p || !ms) return cfail(CHIRP_EINVAL, "NULL argument");
  CKC(cudaStreamSynchronize(p->st));
  for (int i = 0; i < 4; i++) {
    float t = 0.f;
    if (i < 3 || p->timed) CKC(cudaEventElapsedTime(&t, p->ev[i], p->ev[i + 1]));
    ms[i] = t;
  }
  return cpi_status(p);
}

void chirp_cpi_destroy(chirp_cpi_plan* p) {
  if (!p) return;
  cudaStreamSynchronize(p->st);
  free_plan(p);
}

}  // extern "C"
