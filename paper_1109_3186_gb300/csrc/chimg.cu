// chimg.cu -- the paper's own Chimageator pre-integrator (Sec. 4.2, App. B.2)
// on a uniform linear array: mixing (Eq. xpq_chimg), gridding of equal
// spacings, spatial DFT, integrate-and-dump and trajectory sums with the
// 2F-bin widening (Eq. chimg_pth, App. B.2.3), E = |P|^2 (Eq. eth).
//
// Gridding, the spatial DFT and integrate-and-dump are linear and commute,
// so each dump is reduced first: G_l[m] = w_l sum_p sum_{n in dump m}
// y_p[n] y_{p+l}[n]^* (the raw, DM-independent per-dump products of the
// pairs at spacing l), then Y_k[m] = sum_{l=1}^{M-1} exp(-2 pi j k l / Ns)
// G_l[m].  The trajectory image per trial DM then sums 2F+1 bins per dump
// over the DM's window of n_win dumps, with a filter that is the conjugate
// of the expected Y of a unit linear chirp from the pixel's direction (FP64
// closed form at plan creation).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <new>
#include <vector>

#include "../../include/chirp_gb300.h"
#include "internal.h"

using chirp::kCLight;
using chirp::kDefaultKdm;

namespace {

constexpr int kMaxAntUla = 32;
constexpr int kMaxNs = 1024;
constexpr int kStage = 64;  // samples staged per step of the gridding pass

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {  // c + a b
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

// One CTA per dump.  Item (spacing l, r): the samples i = r (mod R) of the
// dump, sum over p of y_p y_{p+l}^*; the R partial sums of a spacing are
// adjacent lanes and meet by shuffles.  Then thread k < Ns forms Y_k.
__global__ void __launch_bounds__(256) k_chimg_grid(const float2* __restrict__ y, long long n_samp,
                                                    int M, int L, int R, int Ns,
                                                    const float* __restrict__ wl,
                                                    float2* __restrict__ Y) {
  __shared__ float2 xs[kMaxAntUla][kStage + 1];
  __shared__ float2 G[kMaxAntUla];
  const long long m = blockIdx.x;
  const int item = threadIdx.x / R, r = threadIdx.x % R;
  const int l = item + 1;
  const bool act = l < M;
  float2 acc = make_float2(0.f, 0.f);
  for (int c0 = 0; c0 < L; c0 += kStage) {
    const int cn = min(kStage, L - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < M * cn; e += blockDim.x) {
      const int a = e / cn, i = e % cn;
      xs[a][i] = y[(long long)a * n_samp + m * L + c0 + i];
    }
    __syncthreads();
    if (act)
      for (int i = r; i < cn; i += R)
        for (int p = 0; p + l < M; p++) {
          const float2 a = xs[p][i], b = xs[p + l][i];
          acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));   // a conj(b)
          acc.y = fmaf(a.y, b.x, fmaf(-a.x, b.y, acc.y));
        }
  }
  for (int o = R / 2; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  __syncthreads();
  if (act && r == 0) G[l] = make_float2(wl[l] * acc.x, wl[l] * acc.y);
  __syncthreads();
  for (int k = threadIdx.x; k < Ns; k += blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int ll = 1; ll < M; ll++) {
      int q = (int)(((long long)k * ll) % Ns);  // exp(-2 pi j q / Ns), q in [-Ns/2, Ns/2)
      if (2 * q >= Ns) q -= Ns;
      float sn, cs;
      sincospif(2.0f * (float)q / (float)Ns, &sn, &cs);
      s = cfma(make_float2(cs, -sn), G[ll], s);
    }
    Y[m * Ns + k] = s;
  }
}

// Thread per (pixel, dump) of one DM (blockIdx.y): the window of n_win dumps
// ending at dump m, 2F+1 bins per dump: P = sum_r sum_j w[r][j] Y[m - n_win
// + 1 + r][bin[r][j]], E = |P|^2; zero while m < n_win - 1.
__global__ void __launch_bounds__(256) k_chimg_image(const float2* __restrict__ Y, int Ns,
                                                     long long n_dump, int n_pix,
                                                     const int* __restrict__ n_win,
                                                     const long long* __restrict__ tap_off, int nj,
                                                     const float2* __restrict__ w,
                                                     const short* __restrict__ bin,
                                                     float* __restrict__ E) {
  const long long d = blockIdx.y;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_pix * n_dump) return;
  const int pix = (int)(idx % n_pix);
  const long long m = idx / n_pix;
  const int nw = n_win[d];
  float e = 0.f;
  if (m >= nw - 1) {
    const long long base = tap_off[d] + (long long)pix * nw * nj;
    float2 P = make_float2(0.f, 0.f);
    for (int r = 0; r < nw; r++) {
      const float2* yr = Y + (m - nw + 1 + r) * Ns;
      for (int j = 0; j < nj; j++) {
        const long long t = base + (long long)r * nj + j;
        P = cfma(w[t], yr[bin[t]], P);
      }
    }
    e = P.x * P.x + P.y * P.y;
  }
  E[(d * n_dump + m) * n_pix + pix] = e;
}

// Filter taps of one DM, FP64: for pixel i, dump r of the window and j < 2F+1,
// bin = (rint(Ns nu_r) + j - F) mod Ns with nu_r = tau (a0 + fdot (t_r - t_c))
// at the dump's centre, and w = conj(Yhat_bin) / ((M - 1) L) with Yhat the
// expected Y of a unit chirp:
//   Yhat_k = sum_l exp(-2 pi j k l / Ns) w_l g_l exp(2 pi j l tau a0)
//            * sum_{i<L} exp(2 pi j phi (r L + i - N/2)),  phi = l tau fdot / B,
//   g_l = sum_{p<M-l} exp(-pi j fdot tau^2 l (2p + l)),  tau = D l_dir / c.
__global__ void k_chimg_taps(const double* __restrict__ ldir, int n_pix, int M, double D, int L,
                             int Ns, int F, int weights, double bw, double a0, double a1, int nw,
                             float2* __restrict__ w, short* __restrict__ bin) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nj = 2 * F + 1;
  if (idx >= (long long)n_pix * nw) return;
  const int pix = (int)(idx / nw), r = (int)(idx % nw);
  const double tau = D * ldir[pix] / kCLight;
  const double N = (double)nw * L;
  const double tr = ((double)r * L + 0.5 * (L - 1) - 0.5 * N) / bw;
  double nu = Ns * tau * (a0 + a1 * tr);
  nu -= Ns * floor(nu / Ns);
  const long long kc = (long long)rint(nu) % Ns;
  for (int j = 0; j < nj; j++) {
    const int k = (int)(((kc + j - F) % Ns + Ns) % Ns);
    double yr = 0.0, yi = 0.0;
    for (int l = 1; l < M; l++) {
      const double wl = weights == 0 ? 1.0 / (M - l) : 1.0;
      double gr = 0.0, gi = 0.0;
      for (int p = 0; p + l < M; p++) {
        double c = -0.5 * a1 * tau * tau * l * (2.0 * p + l);  // cycles
        c -= rint(c);
        double s_, c_;
        sincospi(2.0 * c, &s_, &c_);
        gr += c_;
        gi += s_;
      }
      // time sum over the dump: exp(2 pi j phi (rL - N/2)) * sum_{i<L} exp(2 pi j phi i)
      const double phi = l * tau * a1 / bw;
      double sr_, si_;
      const double den = sinpi(phi);
      double amp;
      if (fabs(den) < 1e-300) {
        amp = (double)L;
      } else {
        amp = sinpi(phi * L) / den;
      }
      double cyc = phi * ((double)r * L - 0.5 * N) + 0.5 * phi * (L - 1) + l * tau * a0 -
                   (double)((long long)k * l % Ns) / Ns;
      cyc -= rint(cyc);
      sincospi(2.0 * cyc, &si_, &sr_);
      const double tr_ = wl * amp * (gr * sr_ - gi * si_), ti_ = wl * amp * (gr * si_ + gi * sr_);
      yr += tr_;
      yi += ti_;
    }
    const double sc = 1.0 / ((double)(M - 1) * L);
    w[idx * nj + j] = make_float2((float)(yr * sc), (float)(-yi * sc));
    bin[idx * nj + j] = (short)k;
  }
}

// The partial-sum recursion of App. B.2.1 on the paper's own model of
// Sec. 4.2: natural weights, Eq. chimg_xpq without its tau^2 term, a baseband
// chirp sweeping 0..B from the window start.  A unit chirp then puts the tone
// nu(t) = rate t cycles per spacing on the grid (rate = fdot tau, t from the
// window start), so every trajectory starts at k = 0 and trials of one rate
// lie on one line.  Taps of row i (a line's rate and a dump r of its window),
// FP64: bin = (rint(Ns rate t_r) + j - F) mod Ns at the dump's centre t_r,
// w = conj(Yhat_bin) / ((M - 1) L) with
//   Yhat_k = sum_{l=1}^{M-1} exp(-2 pi j k l / Ns) sum_{i<L} exp(2 pi j l rate (rL + i) / B).
__global__ void k_chimg_line_taps(const double* __restrict__ row_rate, const int* __restrict__ row_r,
                                  long long n_rows, int M, int L, int Ns, int F, double bw,
                                  float2* __restrict__ w, short* __restrict__ bin) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows) return;
  const int nj = 2 * F + 1;
  const double rate = row_rate[i];
  const double tc = (double)row_r[i] * L + 0.5 * (L - 1);  // the dump's centre, samples
  double nu = Ns * rate * tc / bw;
  nu -= Ns * floor(nu / Ns);
  const long long kc = (long long)rint(nu) % Ns;
  for (int j = 0; j < nj; j++) {
    const int k = (int)(((kc + j - F) % Ns + Ns) % Ns);
    double yr = 0.0, yi = 0.0;
    for (int l = 1; l < M; l++) {
      const double phi = l * rate / bw;  // cycles per sample
      // sum_{i<L} exp(2 pi j phi i) = exp(pi j phi (L - 1)) sin(pi phi L) / sin(pi phi)
      const double den = sinpi(phi);
      double amp;
      if (fabs(den) < 1e-12) {
        const long long n = (long long)rint(phi);
        amp = ((n * (L - 1)) & 1) ? -(double)L : (double)L;
      } else {
        amp = sinpi(phi * L) / den;
      }
      double cyc = phi * tc - (double)((long long)k * l % Ns) / Ns;
      cyc -= rint(cyc);
      double sn, cs;
      sincospi(2.0 * cyc, &sn, &cs);
      yr += amp * cs;
      yi += amp * sn;
    }
    const double sc = 1.0 / ((double)(M - 1) * L);
    w[i * nj + j] = make_float2((float)(yr * sc), (float)(-yi * sc));
    bin[i * nj + j] = (short)k;
  }
}

// Thread per (line g = blockIdx.y, window start s): the cumulative trajectory
// sum along line g from dump s, P_r = sum_{r' <= r} sum_j w Y[s + r'][bin];
// the line's trials, sorted by length n_t, read E[t][s + n_t - 1] = |P_{n_t - 1}|^2.
__global__ void __launch_bounds__(256) k_chimg_lines(const float2* __restrict__ Y, int Ns,
                                                     long long n_dump,
                                                     const long long* __restrict__ row_off,
                                                     const int* __restrict__ n_max, int nj,
                                                     const float2* __restrict__ w,
                                                     const short* __restrict__ bin,
                                                     const int* __restrict__ trial_off,
                                                     const int* __restrict__ trial_len,
                                                     float* __restrict__ E) {
  const int g = blockIdx.y;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_dump) return;
  const long long n = min((long long)n_max[g], n_dump - s);
  int t = trial_off[g];
  const int t_end = trial_off[g + 1];
  const long long base = row_off[g] * nj;
  float2 P = make_float2(0.f, 0.f);
  for (long long r = 0; r < n && t < t_end; r++) {
    const float2* yr = Y + (s + r) * Ns;
    for (int j = 0; j < nj; j++) {
      const long long q = base + r * nj + j;
      P = cfma(w[q], yr[bin[q]], P);
    }
    for (; t < t_end && trial_len[t] == r + 1; t++)
      E[(long long)t * n_dump + s + r] = P.x * P.x + P.y * P.y;
  }
}

int gfail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return chirp_report_error(code, buf);
}

}  // namespace

struct chirp_chimg_plan {
  int M = 0, L = 0, Ns = 0, F = 0, n_pix = 0, n_dm = 0, weights = 0, R = 1;
  long long N = 0, n_dump = 0;
  double D = 0, f0 = 0, bw = 0, kdm = 0;
  std::vector<int> n_win;
  std::vector<long long> tap_off;
  cudaStream_t st = nullptr;
  float2 *d_x = nullptr, *d_Y = nullptr, *d_w = nullptr;
  short* d_bin = nullptr;
  float* d_E = nullptr;
  float* d_wl = nullptr;
  int* d_nwin = nullptr;
  long long* d_off = nullptr;
};

namespace {

void free_chimg(chirp_chimg_plan* p) {
  if (!p) return;
  void* bufs[] = {p->d_x, p->d_Y, p->d_w, p->d_bin, p->d_E, p->d_wl, p->d_nwin, p->d_off};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete p;
}

int galloc(void** ptr, long long bytes, const char* what) {
  if (cudaMalloc(ptr, (size_t)std::max(bytes, 16LL)) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return gfail(CHIRP_ENOMEM, "device allocation of %lld bytes (%s) failed", bytes, what);
  }
  return CHIRP_OK;
}

#define CKG(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return gfail(CHIRP_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                   __FILE__, __LINE__);                                                    \
  } while (0)

int chimg_grid(chirp_chimg_plan* p, const void* volt, int loc) {
  if (!volt) return gfail(CHIRP_EINVAL, "voltages are NULL");
  if (loc != CHIRP_HOST && loc != CHIRP_DEVICE) return gfail(CHIRP_EINVAL, "bad volt_loc");
  const float2* x = static_cast<const float2*>(volt);
  if (loc == CHIRP_HOST) {
    if (!p->d_x) {
      int rc = galloc((void**)&p->d_x, (long long)p->M * p->N * 8, "voltages");
      if (rc) return rc;
    }
    CKG(cudaMemcpyAsync(p->d_x, volt, (size_t)p->M * p->N * 8, cudaMemcpyHostToDevice, p->st));
    x = p->d_x;
  }
  k_chimg_grid<<<(unsigned)p->n_dump, 256, 0, p->st>>>(x, p->N, p->M, p->L, p->R, p->Ns, p->d_wl,
                                                       p->d_Y);
  CKG(cudaGetLastError());
  return CHIRP_OK;
}

}  // namespace

extern "C" {

int chirp_chimg_create(chirp_chimg_plan** out, const chirp_chimg_config* c, void* stream) {
  if (!out) return gfail(CHIRP_EINVAL, "plan pointer is NULL");
  *out = nullptr;
  if (!c || !c->dm || !c->l_dir) return gfail(CHIRP_EINVAL, "config, dm and l_dir are required");
  if (c->n_ant < 2 || c->n_ant > kMaxAntUla) return gfail(CHIRP_EINVAL, "n_ant must be in 2..32");
  if (!(c->spacing_m > 0)) return gfail(CHIRP_EINVAL, "spacing_m must be > 0");
  if (!(c->bw_hz > 0) || !(c->f0_hz > 0.5 * c->bw_hz))
    return gfail(CHIRP_EINVAL, "need bw_hz > 0 and f0_hz > bw_hz / 2");
  if (c->dump_len < 1 || c->n_samp < c->dump_len)
    return gfail(CHIRP_EINVAL, "dump_len must be in 1..n_samp");
  if (c->n_spatial < c->n_ant || c->n_spatial > kMaxNs)
    return gfail(CHIRP_EINVAL, "n_spatial must be in n_ant..1024");
  if (c->half_width < 0 || 2 * c->half_width + 1 > c->n_spatial || c->half_width > 8)
    return gfail(CHIRP_EINVAL, "half_width must be in 0..8 with 2F+1 <= n_spatial");
  if (c->n_dm < 1 || c->n_dm > 65535 || c->n_pix < 1) return gfail(CHIRP_EINVAL, "n_dm in 1..65535, n_pix >= 1");
  if (c->weights != 0 && c->weights != 1) return gfail(CHIRP_EINVAL, "weights must be 0 or 1");
  for (int i = 0; i < c->n_pix; i++)
    if (!(std::fabs(c->l_dir[i]) <= 1.0)) return gfail(CHIRP_EINVAL, "direction %d has |l_dir| > 1", i);
  if (c->n_samp / c->dump_len >= (1LL << 31) ||
      (c->n_samp / c->dump_len) * (long long)c->n_pix / 256 >= (1LL << 31))
    return gfail(CHIRP_EUNSUPPORTED, "too many dumps x directions for one launch");
  chirp_chimg_plan* p = new (std::nothrow) chirp_chimg_plan();
  if (!p) return gfail(CHIRP_ENOMEM, "host allocation failed");
  p->M = c->n_ant;
  p->D = c->spacing_m;
  p->f0 = c->f0_hz;
  p->bw = c->bw_hz;
  p->kdm = c->k_dm > 0 ? c->k_dm : kDefaultKdm;
  p->N = c->n_samp;
  p->L = c->dump_len;
  p->n_dump = c->n_samp / c->dump_len;
  p->Ns = c->n_spatial;
  p->F = c->half_width;
  p->n_pix = c->n_pix;
  p->n_dm = c->n_dm;
  p->weights = c->weights;
  p->st = (cudaStream_t)stream;
  while (p->R < 8 && 2 * p->R * (p->M - 1) <= 256) p->R *= 2;
  const double nu_lo = p->f0 - 0.5 * p->bw, nu_hi = p->f0 + 0.5 * p->bw;
  const int nj = 2 * p->F + 1;
  std::vector<double> a0(p->n_dm), a1(p->n_dm);
  long long taps = 0;
  for (int d = 0; d < p->n_dm; d++) {
    const double dm = c->dm[d];
    if (!(dm > 0) || !std::isfinite(dm)) {
      free_chimg(p);
      return gfail(CHIRP_EINVAL, "trial DM %d must be > 0", d);
    }
    const double T = p->kdm * dm * (1.0 / (nu_lo * nu_lo) - 1.0 / (nu_hi * nu_hi));
    const double alpha = 0.5 * (1.0 / (nu_lo * nu_lo) + 1.0 / (nu_hi * nu_hi));
    const double wn = std::floor(p->bw * T / p->L + 0.5);
    if (wn > (double)p->n_dump) {
      free_chimg(p);
      return gfail(CHIRP_EINVAL, "the sweep of DM %g (%g dumps) is longer than the data", dm, wn);
    }
    a0[d] = 1.0 / std::sqrt(alpha);
    a1[d] = -0.5 / (alpha * std::sqrt(alpha)) / (p->kdm * dm);
    p->n_win.push_back(std::max(1, (int)wn));
    p->tap_off.push_back(taps);
    taps += (long long)p->n_pix * p->n_win.back() * nj;
  }
  std::vector<float> wl(kMaxAntUla, 0.f);
  for (int l = 1; l < p->M; l++) wl[l] = p->weights == 0 ? 1.0f / (float)(p->M - l) : 1.0f;
  double* d_ldir = nullptr;
  int rc = galloc((void**)&p->d_Y, p->n_dump * p->Ns * 8, "gridded spectra");
  if (!rc) rc = galloc((void**)&p->d_w, taps * 8, "filter taps");
  if (!rc) rc = galloc((void**)&p->d_bin, taps * 2, "filter bins");
  if (!rc) rc = galloc((void**)&p->d_wl, kMaxAntUla * 4, "spacing weights");
  if (!rc) rc = galloc((void**)&p->d_nwin, p->n_dm * 4LL, "windows");
  if (!rc) rc = galloc((void**)&p->d_off, p->n_dm * 8LL, "tap offsets");
  if (!rc) rc = galloc((void**)&d_ldir, p->n_pix * 8LL, "directions");
  if (rc) {
    cudaFree(d_ldir);
    free_chimg(p);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(p->d_wl, wl.data(), kMaxAntUla * 4, cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_nwin, p->n_win.data(), p->n_dm * 4, cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_off, p->tap_off.data(), p->n_dm * 8, cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_ldir, c->l_dir, p->n_pix * 8, cudaMemcpyHostToDevice, p->st);
  for (int d = 0; d < p->n_dm && e == cudaSuccess; d++) {
    const long long n = (long long)p->n_pix * p->n_win[d];
    k_chimg_taps<<<(unsigned)((n + 127) / 128), 128, 0, p->st>>>(
        d_ldir, p->n_pix, p->M, p->D, p->L, p->Ns, p->F, p->weights, p->bw, a0[d], a1[d],
        p->n_win[d], p->d_w + p->tap_off[d], p->d_bin + p->tap_off[d]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  cudaFree(d_ldir);
  if (e != cudaSuccess) {
    free_chimg(p);
    return gfail(CHIRP_ECUDA, "plan setup failed: %s", cudaGetErrorString(e));
  }
  *out = p;
  return CHIRP_OK;
}

int chirp_chimg_query(const chirp_chimg_plan* p, long long* n_dump, int* n_win) {
  if (!p) return gfail(CHIRP_EINVAL, "plan is NULL");
  if (n_dump) *n_dump = p->n_dump;
  if (n_win) std::memcpy(n_win, p->n_win.data(), p->n_win.size() * sizeof(int));
  return CHIRP_OK;
}

int chirp_chimg_grid(chirp_chimg_plan* p, const void* volt, int volt_loc, void* Y, int out_loc) {
  if (!p || !Y) return gfail(CHIRP_EINVAL, "NULL argument");
  if (out_loc != CHIRP_HOST && out_loc != CHIRP_DEVICE) return gfail(CHIRP_EINVAL, "bad out_loc");
  int rc = chimg_grid(p, volt, volt_loc);
  if (rc) return rc;
  CKG(cudaMemcpyAsync(Y, p->d_Y, (size_t)p->n_dump * p->Ns * 8,
                      out_loc == CHIRP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, p->st));
  if (out_loc == CHIRP_HOST) CKG(cudaStreamSynchronize(p->st));
  return CHIRP_OK;
}

int chirp_chimg_run(chirp_chimg_plan* p, const void* volt, int volt_loc, float* energy, int out_loc) {
  if (!p || !energy) return gfail(CHIRP_EINVAL, "NULL argument");
  if (out_loc != CHIRP_HOST && out_loc != CHIRP_DEVICE) return gfail(CHIRP_EINVAL, "bad out_loc");
  const long long n_out = (long long)p->n_dm * p->n_dump * p->n_pix;
  float* E = energy;
  if (out_loc == CHIRP_HOST) {
    if (!p->d_E) {
      int rc = galloc((void**)&p->d_E, n_out * 4, "image");
      if (rc) return rc;
    }
    E = p->d_E;
  }
  int rc = chimg_grid(p, volt, volt_loc);
  if (rc) return rc;
  const long long per = (long long)p->n_pix * p->n_dump;
  const dim3 grid((unsigned)((per + 255) / 256), (unsigned)p->n_dm);
  k_chimg_image<<<grid, 256, 0, p->st>>>(p->d_Y, p->Ns, p->n_dump, p->n_pix, p->d_nwin, p->d_off,
                                         2 * p->F + 1, p->d_w, p->d_bin, E);
  CKG(cudaGetLastError());
  if (out_loc == CHIRP_HOST) {
    CKG(cudaMemcpyAsync(energy, E, (size_t)n_out * 4, cudaMemcpyDeviceToHost, p->st));
    CKG(cudaStreamSynchronize(p->st));
  }
  return CHIRP_OK;
}

void chirp_chimg_destroy(chirp_chimg_plan* p) {
  if (!p) return;
  cudaStreamSynchronize(p->st);
  free_chimg(p);
}

}  // extern "C"

// ===========================================================================
// Uniform rectangular arrays (Sec. 4.2 in two dimensions, App. B.2).
// Antenna a = iy Mx + ix sits at (ix Dx, iy Dy, 0).  The per-dump products of
// every pair p <= q, V_pq[m] = sum_{n in dump m} y_p[n] y_q[n]^*, come from the
// CUDA-core correlator on the raw voltages (DM-independent, once per search).
// Spacing s = (lx, ly) = pos(q) - pos(p) of the half plane (ly > 0, or ly = 0
// and lx > 0; every such pair has p < q) is gridded as G_s[m] = w_s sum over
// its pairs of V_pq[m], then Y[m][kx][ky] = sum_s exp(-2 pi j (kx lx / Nx +
// ky ly / Ny)) G_s[m].  The trajectory image reuses k_chimg_image over the
// flattened bins k = kx Ny + ky.
// ===========================================================================
namespace {

constexpr int kMaxAnt2d = 84;
constexpr int kMaxBins2d = 16384;  // Nx Ny, held by the image's 16-bit bin indices

// One CTA per dump: spacing sums from the dump's visibilities, then the 2-D
// DFT over the spacings with exactly reduced integer phases.
// sp[s] = {lx, ly, first pair entry, pair count}; pidx[] = packed pair indices.
__global__ void __launch_bounds__(256) k_chimg2d_grid(const float2* __restrict__ V, int n_pair,
                                                      int S, const int4* __restrict__ sp,
                                                      const int* __restrict__ pidx,
                                                      const float* __restrict__ ws, int Nx,
                                                      int Ny, float2* __restrict__ Y) {
  extern __shared__ float2 G[];  // [S]
  const long long m = blockIdx.x;
  const float2* v = V + m * n_pair;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const int4 e = sp[s];
    float2 acc = make_float2(0.f, 0.f);
    for (int i = 0; i < e.w; i++) {
      const float2 x = v[pidx[e.z + i]];
      acc.x += x.x;
      acc.y += x.y;
    }
    G[s] = make_float2(ws[s] * acc.x, ws[s] * acc.y);
  }
  __syncthreads();
  const int NN = Nx * Ny;
  for (int k = threadIdx.x; k < NN; k += blockDim.x) {
    const int kx = k / Ny, ky = k % Ny;
    float2 acc = make_float2(0.f, 0.f);
    for (int s = 0; s < S; s++) {
      const int4 e = sp[s];
      // phase (kx lx / Nx + ky ly / Ny) cycles = q / (Nx Ny), q reduced exactly
      long long q = ((long long)kx * e.x * Ny + (long long)ky * e.y * Nx) % NN;
      if (q < 0) q += NN;
      if (2 * q >= NN) q -= NN;
      float sn, cs;
      sincospif(2.0f * (float)q / (float)NN, &sn, &cs);
      acc = cfma(make_float2(cs, -sn), G[s], acc);
    }
    Y[m * NN + k] = acc;
  }
}

// Filter taps of one DM, FP64: thread per (pixel, dump r of the window).
// Yhat[kx][ky] = sum_s exp(-2 pi j (kx lx/Nx + ky ly/Ny)) w_s g_s A_s e^{2 pi j c_s}
// with, for a unit chirp from (l, m) (delays tau_a = (x_a l + y_a m) / c,
// dt = tau_p - tau_q = -(lx Dx l + ly Dy m) / c the same for every pair of s):
//   g_s = sum_{(p,q) in s} exp(pi j fdot (tau_p^2 - tau_q^2)),
//   sum_{i<L} exp(-2 pi j dt (a0 + fdot t_i)), t_i = (r L + i - N/2) / B
//       = A_s e^{2 pi j c_s},  phi = -dt fdot / B,  A_s = sin(pi phi L) / sin(pi phi),
//   c_s = -dt (a0 + fdot (r L - N/2) / B) + phi (L - 1) / 2.
// Bins (rint(Nx Dx l nu / c), rint(Ny Dy m nu / c)) mod (Nx, Ny) at the dump's
// centre, nu = a0 + fdot (t_r - t_c); w = conj(Yhat) / (S L).
__global__ void k_chimg2d_taps(const double* __restrict__ pix, int n_pix, int Mx, double Dx,
                               double Dy, int L, int Nx, int Ny, int Fx, int Fy, double bw,
                               double a0, double a1, int nw, int S, const int4* __restrict__ sp,
                               const int2* __restrict__ pairs, const float* __restrict__ ws,
                               float2* __restrict__ w, short* __restrict__ bin) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nj = (2 * Fx + 1) * (2 * Fy + 1);
  if (idx >= (long long)n_pix * nw) return;
  const int ip = (int)(idx / nw), r = (int)(idx % nw);
  const double l = pix[2 * ip], mm = pix[2 * ip + 1];
  const double N = (double)nw * L;
  const double tr = ((double)r * L + 0.5 * (L - 1) - 0.5 * N) / bw;
  const double nu = a0 + a1 * tr;
  const double vx = Nx * Dx * l * nu / kCLight, vy = Ny * Dy * mm * nu / kCLight;
  const long long cx = (((long long)rint(vx)) % Nx + Nx) % Nx;
  const long long cy = (((long long)rint(vy)) % Ny + Ny) % Ny;
  int t = 0;
  for (int jx = -Fx; jx <= Fx; jx++)
    for (int jy = -Fy; jy <= Fy; jy++, t++) {
      const long long kx = ((cx + jx) % Nx + Nx) % Nx, ky = ((cy + jy) % Ny + Ny) % Ny;
      double yr = 0.0, yi = 0.0;
      for (int s = 0; s < S; s++) {
        const int4 e = sp[s];
        const double dt = -((double)e.x * Dx * l + (double)e.y * Dy * mm) / kCLight;
        double gr = 0.0, gi = 0.0;
        for (int i = 0; i < e.w; i++) {
          const int2 pq = pairs[e.z + i];
          const double xp = (pq.x % Mx) * Dx * l + (pq.x / Mx) * Dy * mm;
          const double xq = (pq.y % Mx) * Dx * l + (pq.y / Mx) * Dy * mm;
          const double tp = xp / kCLight, tq = xq / kCLight;
          double c = 0.5 * a1 * (tp * tp - tq * tq);  // cycles
          c -= rint(c);
          double s_, c_;
          sincospi(2.0 * c, &s_, &c_);
          gr += c_;
          gi += s_;
        }
        const double phi = -dt * a1 / bw;
        const double den = sinpi(phi);
        const double amp = fabs(den) < 1e-300 ? (double)L : sinpi(phi * L) / den;
        double cyc = -dt * (a0 + a1 * ((double)r * L - 0.5 * N) / bw) + 0.5 * phi * (L - 1);
        // the DFT kernel's phase, reduced exactly: (kx lx Ny + ky ly Nx) / (Nx Ny)
        const long long NN = (long long)Nx * Ny;
        long long q = (kx * e.x * Ny + ky * e.y * Nx) % NN;
        if (q < 0) q += NN;
        cyc -= rint(cyc);
        cyc -= (double)q / (double)NN;
        double sr_, si_;
        sincospi(2.0 * cyc, &si_, &sr_);
        const double f = ws[s] * amp;
        yr += f * (gr * sr_ - gi * si_);
        yi += f * (gr * si_ + gi * sr_);
      }
      const double sc = 1.0 / ((double)S * L);
      w[idx * nj + t] = make_float2((float)(yr * sc), (float)(-yi * sc));
      bin[idx * nj + t] = (short)(kx * Ny + ky);
    }
}

}  // namespace

struct chirp_chimg2d_plan {
  int Mx = 0, My = 0, M = 0, L = 0, Nx = 0, Ny = 0, Fx = 0, Fy = 0, n_pix = 0, n_dm = 0, S = 0;
  int n_pair = 0;
  long long N = 0, n_dump = 0;
  double Dx = 0, Dy = 0, f0 = 0, bw = 0, kdm = 0;
  std::vector<int> n_win;
  std::vector<long long> tap_off;
  cudaStream_t st = nullptr;
  float2 *d_x = nullptr, *d_V = nullptr, *d_Y = nullptr, *d_w = nullptr;
  short* d_bin = nullptr;
  float *d_E = nullptr, *d_ws = nullptr;
  int4* d_sp = nullptr;
  int* d_pidx = nullptr;
  int* d_nwin = nullptr;
  long long* d_off = nullptr;
};

namespace {

void free_chimg2d(chirp_chimg2d_plan* p) {
  if (!p) return;
  void* bufs[] = {p->d_x,  p->d_V,  p->d_Y,    p->d_w,    p->d_bin, p->d_E,
                  p->d_ws, p->d_sp, p->d_pidx, p->d_nwin, p->d_off};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete p;
}

int chimg2d_grid(chirp_chimg2d_plan* p, const void* volt, int loc) {
  if (!volt) return gfail(CHIRP_EINVAL, "voltages are NULL");
  if (loc != CHIRP_HOST && loc != CHIRP_DEVICE) return gfail(CHIRP_EINVAL, "bad volt_loc");
  const float2* x = static_cast<const float2*>(volt);
  if (loc == CHIRP_HOST) {
    if (!p->d_x) {
      int rc = galloc((void**)&p->d_x, (long long)p->M * p->N * 8, "voltages");
      if (rc) return rc;
    }
    CKG(cudaMemcpyAsync(p->d_x, volt, (size_t)p->M * p->N * 8, cudaMemcpyHostToDevice, p->st));
    x = p->d_x;
  }
  CKG(chirp::launch_correlate(x, p->N, p->M, p->L, 0, p->n_dump, 0, p->n_dump - 1, p->d_V, p->st));
  k_chimg2d_grid<<<(unsigned)p->n_dump, 256, (size_t)p->S * sizeof(float2), p->st>>>(
      p->d_V, p->n_pair, p->S, p->d_sp, p->d_pidx, p->d_ws, p->Nx, p->Ny, p->d_Y);
  CKG(cudaGetLastError());
  return CHIRP_OK;
}

}  // namespace

extern "C" {

int chirp_chimg2d_create(chirp_chimg2d_plan** out, const chirp_chimg2d_config* c, void* stream) {
  chirp_clear_error();
  if (!out) return gfail(CHIRP_EINVAL, "plan pointer is NULL");
  *out = nullptr;
  if (!c || !c->dm || !c->pix_lm) return gfail(CHIRP_EINVAL, "config, dm and pix_lm are required");
  const int Mx = c->n_x, My = c->n_y;
  if (Mx < 1 || My < 1 || Mx * My < 2 || Mx * My > kMaxAnt2d)
    return gfail(CHIRP_EINVAL, "need n_x, n_y >= 1 and 2 <= n_x n_y <= 84");
  if (!(c->dx_m > 0) || !(c->dy_m > 0)) return gfail(CHIRP_EINVAL, "dx_m and dy_m must be > 0");
  if (!(c->bw_hz > 0) || !(c->f0_hz > 0.5 * c->bw_hz))
    return gfail(CHIRP_EINVAL, "need bw_hz > 0 and f0_hz > bw_hz / 2");
  if (c->dump_len < 1 || c->n_samp < c->dump_len)
    return gfail(CHIRP_EINVAL, "dump_len must be in 1..n_samp");
  const int nx_min = My == 1 ? Mx : 2 * Mx - 1;
  if (c->n_spatial_x < nx_min || c->n_spatial_y < My || c->n_spatial_y < 1 ||
      (long long)c->n_spatial_x * c->n_spatial_y > kMaxBins2d)
    return gfail(CHIRP_EINVAL,
                 "need n_spatial_x >= %d, n_spatial_y >= %d (no aliased spacings) and "
                 "n_spatial_x n_spatial_y <= 16384", nx_min, My);
  if (c->half_width_x < 0 || c->half_width_y < 0 || c->half_width_x > 8 || c->half_width_y > 8 ||
      2 * c->half_width_x + 1 > c->n_spatial_x || 2 * c->half_width_y + 1 > c->n_spatial_y)
    return gfail(CHIRP_EINVAL, "half widths must be in 0..8 with 2F+1 <= n_spatial");
  if (c->n_dm < 1 || c->n_dm > 65535 || c->n_pix < 1)
    return gfail(CHIRP_EINVAL, "n_dm in 1..65535, n_pix >= 1");
  if (c->weights != 0 && c->weights != 1) return gfail(CHIRP_EINVAL, "weights must be 0 or 1");
  for (int i = 0; i < c->n_pix; i++) {
    const double l = c->pix_lm[2 * i], m = c->pix_lm[2 * i + 1];
    if (!(l * l + m * m <= 1.0)) return gfail(CHIRP_EINVAL, "pixel %d has l^2 + m^2 > 1", i);
  }
  const long long n_dump = c->n_samp / c->dump_len;
  if (n_dump >= (1LL << 31) || n_dump * (long long)c->n_pix / 256 >= (1LL << 31))
    return gfail(CHIRP_EUNSUPPORTED, "too many dumps x pixels for one launch");
  chirp_chimg2d_plan* p = new (std::nothrow) chirp_chimg2d_plan();
  if (!p) return gfail(CHIRP_ENOMEM, "host allocation failed");
  p->Mx = Mx;
  p->My = My;
  p->M = Mx * My;
  p->Dx = c->dx_m;
  p->Dy = c->dy_m;
  p->f0 = c->f0_hz;
  p->bw = c->bw_hz;
  p->kdm = c->k_dm > 0 ? c->k_dm : kDefaultKdm;
  p->N = c->n_samp;
  p->L = c->dump_len;
  p->n_dump = n_dump;
  p->Nx = c->n_spatial_x;
  p->Ny = c->n_spatial_y;
  p->Fx = c->half_width_x;
  p->Fy = c->half_width_y;
  p->n_pix = c->n_pix;
  p->n_dm = c->n_dm;
  p->n_pair = p->M * (p->M + 1) / 2;
  p->st = (cudaStream_t)stream;

  // half-plane spacings in (ly, lx) order and their pairs (p < q)
  std::vector<int4> sp;
  std::vector<int> pidx;
  std::vector<int2> pairs;
  std::vector<float> ws;
  for (int ly = 0; ly < My; ly++)
    for (int lx = -(Mx - 1); lx <= Mx - 1; lx++) {
      if (ly == 0 && lx <= 0) continue;
      const int first = (int)pidx.size();
      for (int iy = 0; iy + ly < My; iy++)
        for (int ix = 0; ix < Mx; ix++) {
          const int jx = ix + lx;
          if (jx < 0 || jx >= Mx) continue;
          const int a = iy * Mx + ix, b = (iy + ly) * Mx + jx;  // a < b
          pidx.push_back(a * p->M - a * (a - 1) / 2 + (b - a));
          pairs.push_back(make_int2(a, b));
        }
      const int n = (int)pidx.size() - first;
      if (n == 0) continue;
      sp.push_back(make_int4(lx, ly, first, n));
      ws.push_back(c->weights == 0 ? 1.0f / (float)n : 1.0f);
    }
  p->S = (int)sp.size();

  const double nu_lo = p->f0 - 0.5 * p->bw, nu_hi = p->f0 + 0.5 * p->bw;
  const int nj = (2 * p->Fx + 1) * (2 * p->Fy + 1);
  std::vector<double> a0(p->n_dm), a1(p->n_dm);
  long long taps = 0;
  for (int d = 0; d < p->n_dm; d++) {
    const double dm = c->dm[d];
    if (!(dm > 0) || !std::isfinite(dm)) {
      free_chimg2d(p);
      return gfail(CHIRP_EINVAL, "trial DM %d must be > 0", d);
    }
    const double T = p->kdm * dm * (1.0 / (nu_lo * nu_lo) - 1.0 / (nu_hi * nu_hi));
    const double alpha = 0.5 * (1.0 / (nu_lo * nu_lo) + 1.0 / (nu_hi * nu_hi));
    const double wn = std::floor(p->bw * T / p->L + 0.5);
    if (wn > (double)p->n_dump) {
      free_chimg2d(p);
      return gfail(CHIRP_EINVAL, "the sweep of DM %g (%g dumps) is longer than the data", dm, wn);
    }
    a0[d] = 1.0 / std::sqrt(alpha);
    a1[d] = -0.5 / (alpha * std::sqrt(alpha)) / (p->kdm * dm);
    p->n_win.push_back(std::max(1, (int)wn));
    p->tap_off.push_back(taps);
    taps += (long long)p->n_pix * p->n_win.back() * nj;
  }
  double* d_pix = nullptr;
  int2* d_pairs = nullptr;
  int rc = galloc((void**)&p->d_V, p->n_dump * p->n_pair * 8LL, "visibilities");
  if (!rc) rc = galloc((void**)&p->d_Y, p->n_dump * (long long)p->Nx * p->Ny * 8, "gridded spectra");
  if (!rc) rc = galloc((void**)&p->d_w, taps * 8, "filter taps");
  if (!rc) rc = galloc((void**)&p->d_bin, taps * 2, "filter bins");
  if (!rc) rc = galloc((void**)&p->d_ws, p->S * 4LL, "spacing weights");
  if (!rc) rc = galloc((void**)&p->d_sp, p->S * 16LL, "spacings");
  if (!rc) rc = galloc((void**)&p->d_pidx, (long long)pidx.size() * 4, "pair indices");
  if (!rc) rc = galloc((void**)&d_pairs, (long long)pairs.size() * 8, "pairs");
  if (!rc) rc = galloc((void**)&p->d_nwin, p->n_dm * 4LL, "windows");
  if (!rc) rc = galloc((void**)&p->d_off, p->n_dm * 8LL, "tap offsets");
  if (!rc) rc = galloc((void**)&d_pix, p->n_pix * 16LL, "pixels");
  if (rc) {
    cudaFree(d_pix);
    cudaFree(d_pairs);
    free_chimg2d(p);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(p->d_ws, ws.data(), ws.size() * 4, cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_sp, sp.data(), sp.size() * 16, cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_pidx, pidx.data(), pidx.size() * 4, cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_pairs, pairs.data(), pairs.size() * 8, cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_nwin, p->n_win.data(), p->n_dm * 4, cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_off, p->tap_off.data(), p->n_dm * 8, cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_pix, c->pix_lm, p->n_pix * 16, cudaMemcpyHostToDevice, p->st);
  for (int d = 0; d < p->n_dm && e == cudaSuccess; d++) {
    const long long n = (long long)p->n_pix * p->n_win[d];
    k_chimg2d_taps<<<(unsigned)((n + 127) / 128), 128, 0, p->st>>>(
        d_pix, p->n_pix, p->Mx, p->Dx, p->Dy, p->L, p->Nx, p->Ny, p->Fx, p->Fy, p->bw, a0[d],
        a1[d], p->n_win[d], p->S, p->d_sp, d_pairs, p->d_ws, p->d_w + p->tap_off[d],
        p->d_bin + p->tap_off[d]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  cudaFree(d_pix);
  cudaFree(d_pairs);
  if (e != cudaSuccess) {
    free_chimg2d(p);
    return gfail(CHIRP_ECUDA, "plan setup failed: %s", cudaGetErrorString(e));
  }
  *out = p;
  return CHIRP_OK;
}

int chirp_chimg2d_query(const chirp_chimg2d_plan* p, long long* n_dump, int* n_win,
                        int* n_spacing) {
  if (!p) return gfail(CHIRP_EINVAL, "plan is NULL");
  if (n_dump) *n_dump = p->n_dump;
  if (n_win) std::memcpy(n_win, p->n_win.data(), p->n_win.size() * sizeof(int));
  if (n_spacing) *n_spacing = p->S;
  return CHIRP_OK;
}

int chirp_chimg2d_grid(chirp_chimg2d_plan* p, const void* volt, int volt_loc, void* Y,
                       int out_loc) {
  chirp_clear_error();
  if (!p || !Y) return gfail(CHIRP_EINVAL, "NULL argument");
  if (out_loc != CHIRP_HOST && out_loc != CHIRP_DEVICE) return gfail(CHIRP_EINVAL, "bad out_loc");
  int rc = chimg2d_grid(p, volt, volt_loc);
  if (rc) return rc;
  CKG(cudaMemcpyAsync(Y, p->d_Y, (size_t)p->n_dump * p->Nx * p->Ny * 8,
                      out_loc == CHIRP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                      p->st));
  if (out_loc == CHIRP_HOST) CKG(cudaStreamSynchronize(p->st));
  return CHIRP_OK;
}

int chirp_chimg2d_run(chirp_chimg2d_plan* p, const void* volt, int volt_loc, float* energy,
                      int out_loc) {
  chirp_clear_error();
  if (!p || !energy) return gfail(CHIRP_EINVAL, "NULL argument");
  if (out_loc != CHIRP_HOST && out_loc != CHIRP_DEVICE) return gfail(CHIRP_EINVAL, "bad out_loc");
  const long long n_out = (long long)p->n_dm * p->n_dump * p->n_pix;
  float* E = energy;
  if (out_loc == CHIRP_HOST) {
    if (!p->d_E) {
      int rc = galloc((void**)&p->d_E, n_out * 4, "image");
      if (rc) return rc;
    }
    E = p->d_E;
  }
  int rc = chimg2d_grid(p, volt, volt_loc);
  if (rc) return rc;
  const long long per = (long long)p->n_pix * p->n_dump;
  const dim3 grid((unsigned)((per + 255) / 256), (unsigned)p->n_dm);
  k_chimg_image<<<grid, 256, 0, p->st>>>(p->d_Y, p->Nx * p->Ny, p->n_dump, p->n_pix, p->d_nwin,
                                         p->d_off, (2 * p->Fx + 1) * (2 * p->Fy + 1), p->d_w,
                                         p->d_bin, E);
  CKG(cudaGetLastError());
  if (out_loc == CHIRP_HOST) {
    CKG(cudaMemcpyAsync(energy, E, (size_t)n_out * 4, cudaMemcpyDeviceToHost, p->st));
    CKG(cudaStreamSynchronize(p->st));
  }
  return CHIRP_OK;
}

void chirp_chimg2d_destroy(chirp_chimg2d_plan* p) {
  if (!p) return;
  cudaStreamSynchronize(p->st);
  free_chimg2d(p);
}

// ---- App. B.2.1: trials of one trajectory line from one cumulative sum
namespace {
struct DevBufs {  // device scratch of one call, freed on every exit path
  std::vector<void*> p;
  ~DevBufs() {
    for (void* q : p) cudaFree(q);
  }
  int get(void** out, long long bytes, const char* what) {
    int rc = galloc(out, bytes, what);
    if (!rc) p.push_back(*out);
    return rc;
  }
};
}  // namespace

int chirp_chimg_lines_run(const void* Y, long long n_dump, int n_ant, int n_spatial, int dump_len,
                          double bw_hz, int half_width, const double* rate, int n_line,
                          const int* trial_off, const int* trial_len, float* energy,
                          void* stream) {
  chirp_clear_error();
  if (!Y || !rate || !trial_off || !trial_len || !energy) return gfail(CHIRP_EINVAL, "NULL argument");
  if (n_ant < 2 || n_ant > kMaxAntUla || n_spatial < n_ant || n_spatial > kMaxNs ||
      half_width < 0 || 2 * half_width + 1 > n_spatial || dump_len < 1 || !(bw_hz > 0.0) ||
      n_dump < 1 || n_line < 1 || n_line > 65535)
    return gfail(CHIRP_EINVAL, "chirp_chimg_lines_run: bad shape");
  for (const void* ptr : {Y, (const void*)energy}) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return gfail(CHIRP_EINVAL, "chirp_chimg_lines_run: Y and energy must be device memory");
    }
  }
  if (trial_off[0] != 0) return gfail(CHIRP_EINVAL, "chirp_chimg_lines_run: trial_off[0] != 0");
  std::vector<int> n_max(n_line);
  std::vector<long long> row_off(n_line + 1, 0);
  for (int g = 0; g < n_line; g++) {
    if (trial_off[g + 1] <= trial_off[g])
      return gfail(CHIRP_EINVAL, "chirp_chimg_lines_run: line %d has no trial", g);
    for (int t = trial_off[g]; t < trial_off[g + 1]; t++)
      if (trial_len[t] < 1 || (t > trial_off[g] && trial_len[t] < trial_len[t - 1]))
        return gfail(CHIRP_EINVAL, "chirp_chimg_lines_run: trial lengths must be >= 1 and "
                                   "ascending within a line");
    n_max[g] = trial_len[trial_off[g + 1] - 1];
    row_off[g + 1] = row_off[g] + n_max[g];
  }
  const long long n_rows = row_off[n_line];
  const int n_trial = trial_off[n_line];
  const int nj = 2 * half_width + 1;
  if (n_rows > (1LL << 26)) return gfail(CHIRP_EUNSUPPORTED, "chirp_chimg_lines_run: too many taps");
  std::vector<double> row_rate((size_t)n_rows);
  std::vector<int> row_r((size_t)n_rows);
  for (int g = 0; g < n_line; g++)
    for (int r = 0; r < n_max[g]; r++) {
      row_rate[(size_t)(row_off[g] + r)] = rate[g];
      row_r[(size_t)(row_off[g] + r)] = r;
    }
  cudaStream_t st = (cudaStream_t)stream;
  DevBufs b;
  double* d_rate;
  int *d_r, *d_nmax, *d_toff, *d_tlen;
  long long* d_roff;
  float2* d_w;
  short* d_bin;
  int rc = b.get((void**)&d_rate, n_rows * 8, "line rates");
  if (!rc) rc = b.get((void**)&d_r, n_rows * 4, "line rows");
  if (!rc) rc = b.get((void**)&d_nmax, n_line * 4LL, "line lengths");
  if (!rc) rc = b.get((void**)&d_roff, (n_line + 1) * 8LL, "line offsets");
  if (!rc) rc = b.get((void**)&d_toff, (n_line + 1) * 4LL, "trial offsets");
  if (!rc) rc = b.get((void**)&d_tlen, n_trial * 4LL, "trial lengths");
  if (!rc) rc = b.get((void**)&d_w, n_rows * nj * 8, "line taps");
  if (!rc) rc = b.get((void**)&d_bin, n_rows * nj * 2, "line bins");
  if (rc) return rc;
  CKG(cudaMemcpyAsync(d_rate, row_rate.data(), n_rows * 8, cudaMemcpyHostToDevice, st));
  CKG(cudaMemcpyAsync(d_r, row_r.data(), n_rows * 4, cudaMemcpyHostToDevice, st));
  CKG(cudaMemcpyAsync(d_nmax, n_max.data(), n_line * 4LL, cudaMemcpyHostToDevice, st));
  CKG(cudaMemcpyAsync(d_roff, row_off.data(), (n_line + 1) * 8LL, cudaMemcpyHostToDevice, st));
  CKG(cudaMemcpyAsync(d_toff, trial_off, (n_line + 1) * 4LL, cudaMemcpyHostToDevice, st));
  CKG(cudaMemcpyAsync(d_tlen, trial_len, n_trial * 4LL, cudaMemcpyHostToDevice, st));
  k_chimg_line_taps<<<(unsigned)((n_rows + 127) / 128), 128, 0, st>>>(
      d_rate, d_r, n_rows, n_ant, dump_len, n_spatial, half_width, bw_hz, d_w, d_bin);
  CKG(cudaGetLastError());
  CKG(cudaMemsetAsync(energy, 0, (size_t)n_trial * n_dump * 4, st));
  const dim3 grid((unsigned)((n_dump + 255) / 256), (unsigned)n_line);
  k_chimg_lines<<<grid, 256, 0, st>>>((const float2*)Y, n_spatial, n_dump, d_roff, d_nmax, nj, d_w,
                                      d_bin, d_toff, d_tlen, energy);
  CKG(cudaGetLastError());
  CKG(cudaStreamSynchronize(st));  // the scratch is freed on return
  return CHIRP_OK;
}

}  // extern "C"
