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
