// noalloc.cu -- dedispersion of one trial DM that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs while another library
// holds the stream in capture (allocation calls are illegal there), real-time
// pipelines that reserve all device memory at start-up and forbid later
// allocations, and hosts where cudaMalloc/cudaFree would add implicit
// device-wide synchronisation.  For them, chirp_dedisperse_noalloc runs the
// same kernels as chirp_dedisperse_run but keeps every intermediate (twiddle
// tables, FP64 chirp-phase table, forward spectra and inverse-pass
// intermediate) in the file-scope device array below, whose size is fixed at
// CHIRP_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds that
// array until the process exits.
//
// Host code must never hand the array's name to a kernel: in host code the
// symbol is a host-side stand-in, not a device address.  The device address
// is looked up once per device with cudaGetSymbolAddress and passed down.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/chirp_gb300.h"
#include "internal.h"

using namespace chirp;

namespace {

constexpr size_t kScratchBytes = (size_t)CHIRP_NOALLOC_SCRATCH_BYTES;
constexpr size_t kTwiddleBytes = kTwiddleElems * sizeof(float2);
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceScratch {
  bool ready;
  unsigned char* base;  // device address of g_noalloc_scratch on that device
};
DeviceScratch g_dev[kMaxDevices];
std::mutex g_dev_mu;

thread_local char g_msg[256];

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

int bad(int code, const char* msg) {
  snprintf(g_msg, sizeof g_msg, "%s", msg);
  return chirp_report_error(code, g_msg);
}

// Once per device, with that device current: look up the array's device
// address and fill the constant twiddle tables.  Synchronises the stream, so
// the first call on a device must not be inside a stream capture.
int setup_device(cudaStream_t st, unsigned char** base) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return bad(CHIRP_ECUDA, "chirp_dedisperse_noalloc: no usable current device");
  std::lock_guard<std::mutex> lock(g_dev_mu);
  if (!g_dev[dev].ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      snprintf(g_msg, sizeof g_msg, "chirp_dedisperse_noalloc: cudaGetSymbolAddress failed: %s",
               cudaGetErrorString(e));
      return chirp_report_error(CHIRP_ECUDA, g_msg);
    }
    e = launch_build_twiddles((float2*)p, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      snprintf(g_msg, sizeof g_msg, "chirp_dedisperse_noalloc: set-up failed: %s",
               cudaGetErrorString(e));
      return chirp_report_error(CHIRP_ECUDA, g_msg);
    }
    g_dev[dev].base = (unsigned char*)p;
    g_dev[dev].ready = true;
  }
  *base = g_dev[dev].base;
  return CHIRP_OK;
}

// Both buffers must be memory the kernels can address: device or managed.  A
// host pointer handed to the kernels would fault the GPU, so it is refused.
bool device_reachable(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();  // an unregistered host pointer leaves no sticky error
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int chirp_dedisperse_noalloc(const void* volt, int n_ant, long long n_samp,
                                        double f0_hz, double bw_hz, double k_dm, double dm,
                                        long long nfft_min, void* y_out, void* stream) {
  chirp_clear_error();
  if (!volt || !y_out) return bad(CHIRP_EINVAL, "chirp_dedisperse_noalloc: NULL buffer");
  if (!device_reachable(volt) || !device_reachable(y_out))
    return bad(CHIRP_EINVAL,
               "chirp_dedisperse_noalloc: volt and y_out must be device (or managed) memory");
  if (n_ant < 1 || n_samp < 1) return bad(CHIRP_EINVAL, "chirp_dedisperse_noalloc: empty input");
  if (!(f0_hz > 0) || !(bw_hz > 0) || !(bw_hz < 2 * f0_hz))
    return bad(CHIRP_EINVAL, "chirp_dedisperse_noalloc: need f0 > 0 and 0 < bw < 2 f0");
  if (!(dm >= 0) || !std::isfinite(dm))
    return bad(CHIRP_EINVAL, "chirp_dedisperse_noalloc: DM must be finite and >= 0");
  if (nfft_min < 256 || nfft_min > (1LL << 24) || (nfft_min & (nfft_min - 1)))
    return bad(CHIRP_EINVAL, "chirp_dedisperse_noalloc: nfft_min must be a power of two in 256..2^24");
  if (!(k_dm > 0)) k_dm = kDefaultKdm;
  cudaStream_t st = (cudaStream_t)stream;

  // block grid of a one-DM search (same rules as a plan holding only this DM)
  const double fh = f0_hz + 0.5 * bw_hz, fl = f0_hz - 0.5 * bw_hz;
  const long long n_hi =
      (long long)std::ceil(k_dm * dm * (1.0 / (f0_hz * f0_hz) - 1.0 / (fh * fh)) * bw_hz);
  const long long n_lo =
      (long long)std::ceil(k_dm * dm * (1.0 / (fl * fl) - 1.0 / (f0_hz * f0_hz)) * bw_hz);
  long long want = 1, cap = 1;
  while (want < 2 * (n_hi + n_lo)) want <<= 1;
  while (cap < n_samp) cap <<= 1;
  long long nfft = want < cap ? want : cap;
  if (nfft < nfft_min) nfft = nfft_min;
  if (nfft > (1LL << 24))
    return bad(CHIRP_EUNSUPPORTED, "chirp_dedisperse_noalloc: the DM needs an FFT above 2^24");
  GroupGeom g;
  g.nfft = nfft;
  g.log2n = 0;
  while ((1LL << g.log2n) < nfft) g.log2n++;
  g.n1 = (int)(nfft / 4096 > 16 ? nfft / 4096 : 16);
  g.n2 = (int)(nfft / g.n1);
  g.n_hi_max = n_hi;
  g.n_lo_max = n_lo;
  g.step = nfft - n_hi - n_lo;
  if (g.step >= 8) g.step -= g.step % 8;  // blocks start on multiples of 8 samples
  if (n_samp <= nfft) {
    g.n_blk = 1;
  } else {
    if (g.step <= 0) return bad(CHIRP_EINVAL, "chirp_dedisperse_noalloc: non-positive block step");
    g.n_blk = (n_samp - nfft + g.step - 1) / g.step + 1;
  }
  if ((long long)n_ant * g.n_blk > 65535)
    return bad(CHIRP_EUNSUPPORTED, "chirp_dedisperse_noalloc: n_ant * blocks exceeds 65535");

  // scratch layout: twiddles | row twiddles | FP64 phase table | FP32 chirp | spectra |
  // inverse intermediate
  const size_t points = (size_t)n_ant * (size_t)g.n_blk * (size_t)nfft;
  const size_t off_R = align256(kTwiddleBytes);
  const size_t off_G = align256(off_R + (size_t)nfft / 16 * sizeof(float2));
  const size_t off_H = align256(off_G + (size_t)nfft * sizeof(double));
  const size_t off_spec = align256(off_H + (size_t)nfft * sizeof(float2));
  const size_t off_Z = align256(off_spec + points * sizeof(float2));
  const size_t need = align256(off_Z + points * sizeof(float2));
  if (need > kScratchBytes) {
    snprintf(g_msg, sizeof g_msg,
             "chirp_dedisperse_noalloc: this shape needs %zu bytes of scratch; the "
             "allocation-free entry point holds at most %zu (use chirp_dedisperse_run)",
             need, kScratchBytes);
    return chirp_report_error(CHIRP_EINVAL, g_msg);
  }

  unsigned char* base = nullptr;
  int rc = setup_device(st, &base);
  if (rc) return rc;
  const TwiddlePtrs tw = twiddle_ptrs((const float2*)base);
  float2* rtw = (float2*)(base + off_R);
  double* G = (double*)(base + off_G);
  float2* H = (float2*)(base + off_H);
  float2* spec = (float2*)(base + off_spec);
  float2* Z = (float2*)(base + off_Z);

  // nothing in the scratch has to start at zero: every region read below is
  // fully written first by this call; only the caller's output is cleared
  cudaError_t e = launch_build_phase_table(G, g, f0_hz, bw_hz, k_dm, st);
  if (e == cudaSuccess) e = launch_build_row_twiddles(rtw, g, st);
  if (e == cudaSuccess) e = launch_forward((const float2*)volt, n_samp, n_ant, g, spec, tw, st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(y_out, 0, (size_t)n_ant * (size_t)n_samp * sizeof(float2), st);
  if (e == cudaSuccess) e = launch_chirp_table(G, H, dm, g, st);
  const long long n_seq = (long long)n_ant * g.n_blk;
  if (e == cudaSuccess) e = launch_inverse_rows(spec, Z, H, 0, n_seq, g, tw, rtw, st);
  if (e == cudaSuccess)
    e = launch_inverse_cols(Z, (float2*)y_out, n_samp, n_ant, 0, n_seq, g, n_hi, n_lo, tw, st);
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof g_msg, "chirp_dedisperse_noalloc: launch failed: %s",
             cudaGetErrorString(e));
    return chirp_report_error(CHIRP_ECUDA, g_msg);
  }
  return CHIRP_OK;
}
