/*
 * chirp_oracle.c -- plain, slow, FP64 CPU oracle of the coherent-dedispersion
 * pulse-search hot path (Bannister & Cornwell, "The Chirpolator & The
 * Chimageator").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library and includes none of it.
 *
 * What it computes, step by step, in the order of the method:
 *
 *  1. Dispersion sweep (Sec. 2.1, Eq. 1): a DM smears the band [f0-B/2, f0+B/2)
 *     over t = k DM (nu_lo^-2 - nu_hi^-2).  Measured from the arrival at f0,
 *     the upper half of the band came n_hi samples earlier and the lower half
 *     lasts n_lo samples longer:
 *        n_hi = ceil(k DM (f0^-2 - (f0+B/2)^-2) B),
 *        n_lo = ceil(k DM ((f0-B/2)^-2 - f0^-2) B).
 *  2. Coherent dedispersion (Sec. 2.3.2): convolve the complex baseband
 *     voltages (complex Nyquist sampling, f_s = B, Sec. 3.2) with the inverse
 *     of the ISM response.  In the frequency domain the inverse response is
 *        H_DM(f) = exp(-2 pi j k DM f^2 / (f0^2 (f0 + f)))
 *     whose group delay -(1/2pi) dPhi/df = k DM (f0^-2 - (f0+f)^-2) undoes
 *     Eq. 1 about f0.  The convolution is done by overlap-save: blocks of
 *     Nfft samples, forward DFT (e^{-2 pi j n k / N}, the paper's sign,
 *     Eq. dft), multiply by H sampled at the Nfft bins, inverse DFT with 1/Nfft,
 *     keep the n_hi..Nfft-n_lo-1 circular outputs.
 *  3. Chirpolator back-end: per DM and per dump of L samples, the zero-lag
 *     cross products V_pq = sum_t y_p(t) y_q(t)^*  (the p.q^* convention of
 *     Eq. xpq), autocorrelations included, packed upper triangle p <= q.
 *  4. Chimageator back-end: per DM, pixel and dump, the phased sum over
 *     antennas b(t) = sum_a W_pa y_a(t), W_pa = exp(+2 pi j f0 tau_a(l_p,m_p))
 *     with tau from Eq. tau3D (App. A.1) and c = 299792458 m/s, detected as
 *     |b|^2 and summed over the dump (direct beamforming, Sec. 2.4.2).
 *  5. Candidates: per (DM, pixel) series of dump powers, median and
 *     1.4826 x MAD give an S/N per cell; cells at or above a threshold that
 *     are local maxima over (DM, dump, pixel) +- 1 are the detections
 *     (thresholding of the detection metric, Sec. 3.3; best of a bank of
 *     trial filters, App. A.3).
 *
 * Readings where the paper is silent (each listed in the design notes):
 *  - FFT length per DM: Nfft(DM) = max(nfft_min, min(pow2ceil(2 n_d),
 *    pow2ceil(N))), n_d = n_hi + n_lo.  DMs with equal Nfft form a group that
 *    shares one block grid with step S = Nfft - max(n_hi) - max(n_lo) over
 *    the group, rounded down to a multiple of 8 when it is at least 8 (any
 *    step up to that difference keeps every kept output clear of the
 *    circular wrap); n_blk = 1 if N <= Nfft else ceil((N - Nfft)/S) + 1;
 *    block b reads x[b S, b S + Nfft) (zero past N).
 *  - Output time t refers to the arrival at f0.  Valid outputs of a DM are
 *    t in [n_hi, N - n_lo).  Block b owns t in [b S + max n_hi, (b+1) S +
 *    max n_hi); block 0 also owns everything below, the last block
 *    everything above.
 *  - Dumps are the absolute grid [m L, (m+1) L), m < floor(N/L); a dump is
 *    valid for a DM only if it lies inside the valid range; invalid dumps
 *    are zero in the outputs.
 *  - The phase k DM g(f_b) is formed in FP64 as DM * (k * g), reduced by
 *    subtracting rint(), and exponentiated with cos/sin of 2 pi frac.
 *
 * Every function below is written for checking by eye, not for speed: no
 * blocking, fusion or reordering beyond what the steps above state.  Loops
 * over independent antennas, blocks and dumps run under OpenMP; each output
 * is written by exactly one thread, so results do not depend on the thread
 * count.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double ORC_PI = 3.14159265358979323846264338327950288;
static const double ORC_C_LIGHT = 299792458.0;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* DFTs                                                               */
/* ------------------------------------------------------------------ */

static int orc_is_pow2(long long n) { return n > 0 && (n & (n - 1)) == 0; }

static long long orc_pow2ceil(long long n) {
  long long p = 1;
  while (p < n) p <<= 1;
  return p;
}

/* Direct DFT: X[k] = sum_n x[n] exp(sign 2 pi j n k / n_pts).  O(n^2). */
void orc_dft(const double* xin, double* Xout, long long n_pts, int sign) {
  const cplx* x = (const cplx*)xin;
  cplx* X = (cplx*)Xout;
  for (long long k = 0; k < n_pts; k++) {
    cplx acc = 0.0;
    for (long long n = 0; n < n_pts; n++) {
      long long nk = (n * k) % n_pts; /* exact phase index */
      double ang = sign * 2.0 * ORC_PI * (double)nk / (double)n_pts;
      acc += x[n] * (cos(ang) + I * sin(ang));
    }
    X[k] = acc;
  }
}

/* In-place radix-2 decimation-in-time FFT, unnormalised,
 * X[k] = sum_n x[n] exp(sign 2 pi j n k / n_pts).  Returns -1 unless n_pts is
 * a power of two. */
static int orc_fft_c(cplx* x, long long n_pts, int sign) {
  if (!orc_is_pow2(n_pts)) return -1;
  /* bit-reversal permutation */
  for (long long i = 1, j = 0; i < n_pts; i++) {
    long long bit = n_pts >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      cplx t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  if (n_pts < 2) return 0;
  /* twiddles w[k] = exp(sign 2 pi j k / n_pts), each from its own cos/sin */
  long long half_n = n_pts / 2;
  cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)half_n);
  if (!w) return -2;
  for (long long k = 0; k < half_n; k++) {
    double ang = sign * 2.0 * ORC_PI * (double)k / (double)n_pts;
    w[k] = cos(ang) + I * sin(ang);
  }
  for (long long len = 2; len <= n_pts; len <<= 1) {
    long long half = len / 2, step = n_pts / len;
    for (long long s = 0; s < n_pts; s += len) {
      for (long long k = 0; k < half; k++) {
        cplx u = x[s + k];
        cplx v = x[s + k + half] * w[k * step];
        x[s + k] = u + v;
        x[s + k + half] = u - v;
      }
    }
  }
  free(w);
  return 0;
}

int orc_fft(double* x, long long n_pts, int sign) { return orc_fft_c((cplx*)x, n_pts, sign); }

/* ------------------------------------------------------------------ */
/* Dispersion sweep, FFT length, block grid                           */
/* ------------------------------------------------------------------ */

void orc_sweep(double f0, double bw, double k_dm, double dm, long long* n_hi, long long* n_lo) {
  double fh = f0 + 0.5 * bw, fl = f0 - 0.5 * bw;
  double t_hi = k_dm * dm * (1.0 / (f0 * f0) - 1.0 / (fh * fh));
  double t_lo = k_dm * dm * (1.0 / (fl * fl) - 1.0 / (f0 * f0));
  *n_hi = (long long)ceil(t_hi * bw);
  *n_lo = (long long)ceil(t_lo * bw);
}

long long orc_nfft_for_dm(double f0, double bw, double k_dm, double dm, long long n_samp,
                          long long nfft_min) {
  long long hi, lo;
  orc_sweep(f0, bw, k_dm, dm, &hi, &lo);
  long long want = orc_pow2ceil(2 * (hi + lo) > 1 ? 2 * (hi + lo) : 1);
  long long cap = orc_pow2ceil(n_samp);
  long long n = want < cap ? want : cap;
  return n > nfft_min ? n : nfft_min;
}

typedef struct {
  long long nfft, n_hi, n_lo;         /* this DM */
  long long n_hi_max, n_lo_max;       /* over the DM's group */
  long long step, n_blk;
} orc_layout_t;

/* Block grid of DM number d of the list (see the readings in the header). */
int orc_layout(const double* dms, int n_dm, int d, double f0, double bw, double k_dm,
               long long n_samp, long long nfft_min, long long* out7) {
  if (d < 0 || d >= n_dm || !orc_is_pow2(nfft_min)) return -1;
  orc_layout_t L;
  L.nfft = orc_nfft_for_dm(f0, bw, k_dm, dms[d], n_samp, nfft_min);
  orc_sweep(f0, bw, k_dm, dms[d], &L.n_hi, &L.n_lo);
  L.n_hi_max = 0;
  L.n_lo_max = 0;
  for (int e = 0; e < n_dm; e++) {
    if (orc_nfft_for_dm(f0, bw, k_dm, dms[e], n_samp, nfft_min) != L.nfft) continue;
    long long hi, lo;
    orc_sweep(f0, bw, k_dm, dms[e], &hi, &lo);
    if (hi > L.n_hi_max) L.n_hi_max = hi;
    if (lo > L.n_lo_max) L.n_lo_max = lo;
  }
  L.step = L.nfft - L.n_hi_max - L.n_lo_max;
  if (L.step >= 8) L.step -= L.step % 8;  /* block starts on multiples of 8 samples */
  if (n_samp <= L.nfft) {
    L.n_blk = 1;
  } else {
    if (L.step <= 0) return -2;
    L.n_blk = (n_samp - L.nfft + L.step - 1) / L.step + 1;
  }
  out7[0] = L.nfft;
  out7[1] = L.n_hi;
  out7[2] = L.n_lo;
  out7[3] = L.n_hi_max;
  out7[4] = L.n_lo_max;
  out7[5] = L.step;
  out7[6] = L.n_blk;
  return 0;
}

/* Valid dump range [first, last] of one DM (last < first: none). */
void orc_dump_range(long long n_samp, long long n_hi, long long n_lo, int dump_len,
                    long long* first, long long* last) {
  *first = (n_hi + dump_len - 1) / dump_len;
  long long end = n_samp - n_lo; /* one past the last valid sample */
  *last = end >= 0 ? end / dump_len - 1 : -1;
}

/* ------------------------------------------------------------------ */
/* Chirp                                                              */
/* ------------------------------------------------------------------ */

/* H[b] = exp(-2 pi j k DM g(f_b)), g(f) = f^2/(f0^2 (f0+f)),
 * f_b = b B/Nfft for b < Nfft/2, else (b - Nfft) B/Nfft. */
void orc_chirp(double f0, double bw, double k_dm, double dm, long long nfft, double* Hout) {
  cplx* H = (cplx*)Hout;
  for (long long b = 0; b < nfft; b++) {
    double f = (double)(b < nfft / 2 ? b : b - nfft) * bw / (double)nfft;
    double g = f * f / (f0 * f0 * (f0 + f));
    double c = dm * (k_dm * g);
    double r = c - rint(c);
    H[b] = cos(2.0 * ORC_PI * r) - I * sin(2.0 * ORC_PI * r);
  }
}

/* ------------------------------------------------------------------ */
/* Overlap-save dedispersion                                          */
/* ------------------------------------------------------------------ */

/* Index of the block that owns output time t. */
static long long orc_owner(long long t, long long n_hi_max, long long step, long long n_blk) {
  if (n_blk <= 1) return 0;
  long long u = t - n_hi_max;
  long long b = u < 0 ? 0 : u / step;
  return b > n_blk - 1 ? n_blk - 1 : b;
}

/* Dedisperse the antennas of x [n_ant][n_samp] at DM number d over output
 * times [t_lo, t_hi): y [n_ant][t_hi - t_lo], zero where t is not valid. */
int orc_dedisperse_span(const double* xin, int n_ant, long long n_samp, double f0, double bw,
                        double k_dm, const double* dms, int n_dm, int d, long long nfft_min,
                        long long t_lo, long long t_hi, double* yout) {
  const cplx* x = (const cplx*)xin;
  cplx* y = (cplx*)yout;
  long long lay[7];
  int rc = orc_layout(dms, n_dm, d, f0, bw, k_dm, n_samp, nfft_min, lay);
  if (rc) return rc;
  long long nfft = lay[0], n_hi = lay[1], n_lo = lay[2], n_hi_max = lay[3];
  long long step = lay[5], n_blk = lay[6];
  long long span = t_hi - t_lo;
  if (span <= 0) return 0;
  memset(y, 0, sizeof(cplx) * (size_t)n_ant * (size_t)span);
  long long v_lo = n_hi > t_lo ? n_hi : t_lo;
  long long v_hi = (n_samp - n_lo) < t_hi ? (n_samp - n_lo) : t_hi;
  if (v_hi <= v_lo) return 0;
  long long b_first = orc_owner(v_lo, n_hi_max, step, n_blk);
  long long b_last = orc_owner(v_hi - 1, n_hi_max, step, n_blk);
  long long nb = b_last - b_first + 1;

  cplx* H = (cplx*)malloc(sizeof(cplx) * (size_t)nfft);
  if (!H) return -3;
  orc_chirp(f0, bw, k_dm, dms[d], nfft, (double*)H);

  int fail = 0;
#pragma omp parallel
  {
    cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)nfft);
    if (!buf) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for collapse(2) schedule(dynamic, 1)
    for (int a = 0; a < n_ant; a++) {
      for (long long bi = 0; bi < nb; bi++) {
        if (!buf) continue;
        long long b = b_first + bi;
        long long s0 = b * step;
        for (long long i = 0; i < nfft; i++)
          buf[i] = (s0 + i < n_samp) ? x[(size_t)a * n_samp + s0 + i] : 0.0;
        orc_fft_c(buf, nfft, -1);
        for (long long i = 0; i < nfft; i++) buf[i] *= H[i];
        orc_fft_c(buf, nfft, +1);
        for (long long t = v_lo; t < v_hi; t++) {
          if (orc_owner(t, n_hi_max, step, n_blk) != b) continue;
          long long i = t - s0; /* inside [n_hi, nfft - n_lo) by construction */
          y[(size_t)a * span + (t - t_lo)] = buf[i] / (double)nfft;
        }
      }
    }
    free(buf);
  }
  free(H);
  return fail ? -3 : 0;
}

/* ------------------------------------------------------------------ */
/* Back-ends                                                          */
/* ------------------------------------------------------------------ */

/* Zero-lag visibilities of y [n_ant][span] (span starts at dump m0) for dumps
 * m in [m0, m1): V [(m1-m0)][n_ant (n_ant+1)/2], pair order p <= q row-major.
 * Dumps outside [first, last] stay zero. */
void orc_correlate(const double* yin, int n_ant, long long span, int dump_len, long long m0,
                   long long m1, long long first, long long last, double* Vout) {
  const cplx* y = (const cplx*)yin;
  cplx* V = (cplx*)Vout;
  int n_pair = n_ant * (n_ant + 1) / 2;
  memset(V, 0, sizeof(cplx) * (size_t)(m1 - m0) * (size_t)n_pair);
#pragma omp parallel for schedule(dynamic, 1)
  for (long long m = m0; m < m1; m++) {
    if (m < first || m > last) continue;
    int k = 0;
    for (int p = 0; p < n_ant; p++) {
      for (int q = p; q < n_ant; q++, k++) {
        cplx acc = 0.0;
        for (long long t = 0; t < dump_len; t++) {
          long long i = (m - m0) * dump_len + t;
          acc += y[(size_t)p * span + i] * conj(y[(size_t)q * span + i]);
        }
        V[(size_t)(m - m0) * n_pair + k] = acc;
      }
    }
  }
}

/* Narrowband phased-sum weights W [n_pix][n_ant] = exp(+2 pi j f0 tau_a),
 * tau_a = (x l + y m + z (sqrt(1 - l^2 - m^2) - 1)) / c. */
void orc_beam_weights(const double* xyz, int n_ant, const double* pix_lm, int n_pix, double f0,
                      double* Wout) {
  cplx* W = (cplx*)Wout;
  for (int p = 0; p < n_pix; p++) {
    double l = pix_lm[2 * p], m = pix_lm[2 * p + 1];
    double n = sqrt(1.0 - l * l - m * m);
    for (int a = 0; a < n_ant; a++) {
      double tau = (xyz[3 * a] * l + xyz[3 * a + 1] * m + xyz[3 * a + 2] * (n - 1.0)) / ORC_C_LIGHT;
      double ph = 2.0 * ORC_PI * f0 * tau;
      W[(size_t)p * n_ant + a] = cos(ph) + I * sin(ph);
    }
  }
}

/* Beam powers P [(m1-m0)][n_pix] = sum over the dump of |sum_a W_pa y_a(t)|^2. */
void orc_beamform(const double* yin, int n_ant, long long span, int dump_len, long long m0,
                  long long m1, long long first, long long last, const double* Win, int n_pix,
                  double* P) {
  const cplx* y = (const cplx*)yin;
  const cplx* W = (const cplx*)Win;
  memset(P, 0, sizeof(double) * (size_t)(m1 - m0) * (size_t)n_pix);
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
  for (long long m = m0; m < m1; m++) {
    for (int p = 0; p < n_pix; p++) {
      if (m < first || m > last) continue;
      double acc = 0.0;
      for (long long t = 0; t < dump_len; t++) {
        long long i = (m - m0) * dump_len + t;
        cplx b = 0.0;
        for (int a = 0; a < n_ant; a++) b += W[(size_t)p * n_ant + a] * y[(size_t)a * span + i];
        acc += creal(b) * creal(b) + cimag(b) * cimag(b);
      }
      P[(size_t)(m - m0) * n_pix + p] = acc;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Whole searches over a selection of DMs and a range of dumps        */
/* ------------------------------------------------------------------ */

/* V [n_sel][m1-m0][n_ant(n_ant+1)/2] complex for DMs dms[d_sel[i]]. */
int orc_chirpolator(const double* x, int n_ant, long long n_samp, double f0, double bw,
                    double k_dm, const double* dms, int n_dm, long long nfft_min, int dump_len,
                    const int* d_sel, int n_sel, long long m0, long long m1, double* V) {
  long long span = (m1 - m0) * dump_len;
  int n_pair = n_ant * (n_ant + 1) / 2;
  double* y = (double*)malloc(sizeof(cplx) * (size_t)n_ant * (size_t)span);
  if (!y) return -3;
  for (int i = 0; i < n_sel; i++) {
    int d = d_sel[i];
    int rc = orc_dedisperse_span(x, n_ant, n_samp, f0, bw, k_dm, dms, n_dm, d, nfft_min,
                                 m0 * dump_len, m1 * dump_len, y);
    if (rc) {
      free(y);
      return rc;
    }
    long long lay[7], first, last;
    orc_layout(dms, n_dm, d, f0, bw, k_dm, n_samp, nfft_min, lay);
    orc_dump_range(n_samp, lay[1], lay[2], dump_len, &first, &last);
    orc_correlate(y, n_ant, span, dump_len, m0, m1, first, last,
                  V + (size_t)2 * i * (size_t)(m1 - m0) * n_pair);
  }
  free(y);
  return 0;
}

/* P [n_sel][m1-m0][n_pix] for DMs dms[d_sel[i]]. */
int orc_chimageator(const double* x, int n_ant, long long n_samp, double f0, double bw,
                    double k_dm, const double* dms, int n_dm, long long nfft_min, int dump_len,
                    const double* xyz, const double* pix_lm, int n_pix, const int* d_sel,
                    int n_sel, long long m0, long long m1, double* P) {
  long long span = (m1 - m0) * dump_len;
  double* y = (double*)malloc(sizeof(cplx) * (size_t)n_ant * (size_t)span);
  double* W = (double*)malloc(sizeof(cplx) * (size_t)n_pix * (size_t)n_ant);
  if (!y || !W) {
    free(y);
    free(W);
    return -3;
  }
  orc_beam_weights(xyz, n_ant, pix_lm, n_pix, f0, W);
  for (int i = 0; i < n_sel; i++) {
    int d = d_sel[i];
    int rc = orc_dedisperse_span(x, n_ant, n_samp, f0, bw, k_dm, dms, n_dm, d, nfft_min,
                                 m0 * dump_len, m1 * dump_len, y);
    if (rc) {
      free(y);
      free(W);
      return rc;
    }
    long long lay[7], first, last;
    orc_layout(dms, n_dm, d, f0, bw, k_dm, n_samp, nfft_min, lay);
    orc_dump_range(n_samp, lay[1], lay[2], dump_len, &first, &last);
    orc_beamform(y, n_ant, span, dump_len, m0, m1, first, last, W, n_pix,
                 P + (size_t)i * (size_t)(m1 - m0) * n_pix);
  }
  free(y);
  free(W);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Incoherent path: power-beam filterbank + shift-and-sum dedispersion */
/* ------------------------------------------------------------------ */

/* Filterbank power of the power beam (Sec. 2.3.1 with power beams, Sec. 2.4.1):
 * each antenna's series is cut into blocks of n_chan samples and transformed
 * (e^{-2 pi j n k / n_chan}); channel c holds bin k = (c + n_chan/2) mod n_chan,
 * i.e. ascending frequency f_c = f0 + (c - n_chan/2) B / n_chan.  The squared
 * magnitudes are summed over antennas and over n_int consecutive blocks:
 *   S[c][tau] = sum_a sum_{i < n_int} |X_{a, tau n_int + i}[k(c)]|^2,
 * tau < T_fb = floor(n_samp / (n_chan n_int)).  S is [n_chan][T_fb]. */
void orc_filterbank(const double* xin, int n_ant, long long n_samp, int n_chan, int n_int,
                    double* S) {
  const cplx* x = (const cplx*)xin;
  long long T_fb = n_samp / ((long long)n_chan * n_int);
  memset(S, 0, sizeof(double) * (size_t)n_chan * (size_t)T_fb);
#pragma omp parallel for schedule(static)
  for (long long tau = 0; tau < T_fb; tau++) {
    cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)n_chan);
    for (int a = 0; a < n_ant; a++) {
      for (int i = 0; i < n_int; i++) {
        const cplx* blk = x + (size_t)a * n_samp + (size_t)(tau * n_int + i) * n_chan;
        orc_dft((const double*)blk, (double*)X, n_chan, -1);
        for (int c = 0; c < n_chan; c++) {
          int k = (c + n_chan / 2) % n_chan;
          S[(size_t)c * T_fb + tau] += creal(X[k]) * creal(X[k]) + cimag(X[k]) * cimag(X[k]);
        }
      }
    }
    free(X);
  }
}

/* Channel delay of DM in filterbank samples, relative to f0 (Eq. dmdelay):
 * s_c = floor(k DM (f_c^-2 - f0^-2) / t_fb + 1/2), t_fb = n_chan n_int / B. */
long long orc_channel_shift(double f0, double bw, double k_dm, double dm, int n_chan, int n_int,
                            int c) {
  double fc = f0 + (double)(c - n_chan / 2) * bw / (double)n_chan;
  double t_fb = (double)n_chan * (double)n_int / bw;
  double tau = k_dm * dm * (1.0 / (fc * fc) - 1.0 / (f0 * f0));
  return (long long)floor(tau / t_fb + 0.5);
}

/* Incoherent dedispersion (Sec. 2.3.1): D[d][t] = sum_c S[c][t + s_c(DM_d)] for
 * t in [-min_c s_c, T_fb - max_c s_c), zero elsewhere; D is [n_dm][T_fb]. */
void orc_incoherent(const double* S, int n_chan, long long T_fb, double f0, double bw,
                    double k_dm, int n_int, const double* dms, int n_dm, double* D) {
  memset(D, 0, sizeof(double) * (size_t)n_dm * (size_t)T_fb);
#pragma omp parallel for schedule(dynamic, 1)
  for (int d = 0; d < n_dm; d++) {
    long long s_min = 0, s_max = 0;
    long long* s = (long long*)malloc(sizeof(long long) * (size_t)n_chan);
    for (int c = 0; c < n_chan; c++) {
      s[c] = orc_channel_shift(f0, bw, k_dm, dms[d], n_chan, n_int, c);
      if (c == 0 || s[c] < s_min) s_min = s[c];
      if (c == 0 || s[c] > s_max) s_max = s[c];
    }
    for (long long t = -s_min; t < T_fb - s_max; t++) {
      double acc = 0.0;
      for (int c = 0; c < n_chan; c++) acc += S[(size_t)c * T_fb + t + s[c]];
      D[(size_t)d * T_fb + t] = acc;
    }
    free(s);
  }
}

/* ---------------------------------------------------------------------------
 * Candidate detection on the beam powers (thresholding of the detection
 * metric, Sec. 3.3 after Eq. eth; the unknown DM, arrival time and direction
 * are searched by taking the best of a bank of trial filters, App. A.3).
 *
 * Per (DM d, pixel p) the series x_m = P[d][m][p] over the DM's valid dumps
 * m = first[d] .. last[d] (n values) gives
 *    med   = median(x)                (even n: mean of the two middle values)
 *    sigma = 1.4826 * median(|x - med|)
 * and every valid cell gets S/N = (x - med) / sigma (0 when sigma == 0).  A
 * candidate is a valid cell with S/N >= snr_min that no valid cell among its
 * 26 neighbours (d +- 1, m +- 1, p +- 1 in the pixel list) exceeds.
 * The statistics are computed in FP32, the precision of the powers, one
 * IEEE-rounded operation at a time:  med = (a + b) * 0.5,  |x - med|,
 * sigma = 1.4826f * mad,  S/N = (x - med) / sigma.
 * -------------------------------------------------------------------------*/
static int orc_cmp_float(const void* a, const void* b) {
  float x = *(const float*)a, y = *(const float*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* median of v[0..n) (v is sorted in place) */
static float orc_median_f(float* v, long long n) {
  qsort(v, (size_t)n, sizeof(float), orc_cmp_float);
  if (n % 2) return v[n / 2];
  volatile float s = v[n / 2 - 1] + v[n / 2];
  return s * 0.5f;
}

/* stats [n_dm][n_pix][2] = (med, sigma) */
void orc_series_stats(const float* P, int n_dm, long long n_dump, int n_pix,
                      const long long* first, const long long* last, float* stats) {
  for (int d = 0; d < n_dm; d++) {
    long long n = last[d] - first[d] + 1;
    for (int p = 0; p < n_pix; p++) {
      float med = 0.f, sigma = 0.f;
      if (n > 0) {
        float* v = (float*)malloc((size_t)n * sizeof(float));
        for (long long m = 0; m < n; m++) v[m] = P[((size_t)d * n_dump + first[d] + m) * n_pix + p];
        med = orc_median_f(v, n);
        for (long long m = 0; m < n; m++) {
          volatile float dv = v[m] - med;
          v[m] = fabsf(dv);
        }
        volatile float mad = orc_median_f(v, n);
        sigma = 1.4826f * mad;
        free(v);
      }
      stats[2 * ((size_t)d * n_pix + p)] = med;
      stats[2 * ((size_t)d * n_pix + p) + 1] = sigma;
    }
  }
}

static float orc_snr_at(const float* P, long long n_dump, int n_pix, const float* stats, int d,
                        long long m, int p) {
  const float med = stats[2 * ((size_t)d * n_pix + p)];
  const float sigma = stats[2 * ((size_t)d * n_pix + p) + 1];
  if (!(sigma > 0.f)) return 0.f;
  volatile float num = P[((size_t)d * n_dump + m) * n_pix + p] - med;
  return num / sigma;
}

/* Candidates in (d, m, p) order; returns their number (only the first
 * max_out are stored). */
long long orc_detect(const float* P, int n_dm, long long n_dump, int n_pix,
                     const long long* first, const long long* last, float snr_min,
                     const float* stats, int* cd, long long* cm, int* cp, float* csnr,
                     long long max_out) {
  long long n = 0;
  for (int d = 0; d < n_dm; d++)
    for (long long m = first[d]; m <= last[d]; m++)
      for (int p = 0; p < n_pix; p++) {
        const float s = orc_snr_at(P, n_dump, n_pix, stats, d, m, p);
        if (!(s >= snr_min)) continue;
        int peak = 1;
        for (int dd = -1; dd <= 1 && peak; dd++)
          for (long long dm = -1; dm <= 1 && peak; dm++)
            for (int dp = -1; dp <= 1 && peak; dp++) {
              if (!dd && !dm && !dp) continue;
              const int d2 = d + dd, p2 = p + dp;
              const long long m2 = m + dm;
              if (d2 < 0 || d2 >= n_dm || p2 < 0 || p2 >= n_pix) continue;
              if (m2 < first[d2] || m2 > last[d2]) continue;
              if (orc_snr_at(P, n_dump, n_pix, stats, d2, m2, p2) > s) peak = 0;
            }
        if (!peak) continue;
        if (n < max_out) {
          cd[n] = d;
          cm[n] = m;
          cp[n] = p;
          csnr[n] = s;
        }
        n++;
      }
  return n;
}
