// plan.cu -- the C ABI of include/chirp_gb300.h: plan creation (block grids,
// device workspace, FP64 tables, beam weights) and the run entry points that
// sequence the kernels on the plan's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <vector>

#include "../../include/chirp_gb300.h"
#include "internal.h"

using namespace chirp;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(CHIRP_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                  __FILE__, __LINE__);                                                    \
  } while (0)


long long pow2ceil(long long n) {
  long long p = 1;
  while (p < n) p <<= 1;
  return p;
}
int ilog2ll(long long n) {
  int l = 0;
  while ((1LL << l) < n) l++;
  return l;
}
bool is_pow2(long long n) { return n > 0 && (n & (n - 1)) == 0; }

// Eq. 1 sweep about f0 in samples (above, below the band centre)
void sweep(double f0, double bw, double k_dm, double dm, long long* n_hi, long long* n_lo) {
  double fh = f0 + 0.5 * bw, fl = f0 - 0.5 * bw;
  double t_hi = k_dm * dm * (1.0 / (f0 * f0) - 1.0 / (fh * fh));
  double t_lo = k_dm * dm * (1.0 / (fl * fl) - 1.0 / (f0 * f0));
  *n_hi = (long long)std::ceil(t_hi * bw);
  *n_lo = (long long)std::ceil(t_lo * bw);
}

struct Group {
  GroupGeom geom;
  std::vector<int> dms;
  double* d_G = nullptr;     // FP64 phase table, spectrum order
  float2* d_spec = nullptr;  // [n_blk][n_ant][nfft] (block-major sequences)
  float2* d_rtw = nullptr;   // row-pass twiddles [n1][n2/16]
  void* d_tdph = nullptr;    // true-delay beams: [n_pix][n_ant] 64-bit phase pairs (lazy)
  float2* d_tdrot = nullptr; // true-delay beams: [n_pix][n_ant] weight step along a row
};

struct DmInfo {
  int group;
  long long n_hi, n_lo, first, last;
};

}  // namespace

// Cost model of the two exact Chimageator forms, seconds per DM-sample (both
// read the dedispersed voltages once; the column pass writes the same bytes
// for either).  Phased-sum GEMM: 8 n_pix M flops, executed ~3.3x over in the
// split-BF16 form, at the tensor pipe's measured ~1.85 PFLOP/s, or its read of
// the 8 M-byte BF16 image at ~5 TB/s when that is slower.  Visibility
// identity sum_t |w.y|^2 = w^H V w: the correlator's 8 M(M+1)/2 flops, bound
// by its ~1.5e13 flop/s or by reading 8 M bytes at ~2.5 TB/s (both measured on
// GB300 at 12 antennas), plus the quadratic form's 4 M(M+1)/2 n_pix flops per
// dump of L samples at ~2e13 flop/s.
bool vis_beats_gemm(int M, int n_pix, int L) {
  const double pairs = 0.5 * M * (M + 1.0);
  const double t_gemm = std::max(8.0 * n_pix * M * 3.33 / 1.85e15, 8.0 * M / 5e12);
  const double t_corr = std::max(8.0 * pairs / 1.5e13, 8.0 * M / 2.5e12);
  const double t_vis = t_corr + 4.0 * pairs * n_pix / L / 2e13;
  return t_vis < t_gemm;
}

int chirp_report_error(int code, const char* msg) { return fail(code, "%s", msg); }
void chirp_clear_error() { g_err[0] = 0; }

struct chirp_plan {
  int M = 0;
  std::vector<double> xyz;
  double f0 = 0, bw = 0, kdm = 0;
  long long N = 0;
  std::vector<double> dm;
  int L = 0;
  long long nfft_min = 0;
  std::vector<double> pix;
  int n_pix = 0;
  int beam_mode = 0;
  int beam_terms = 3;         // tensor-core modes: 3 (split BF16) or 1 (BF16)
  int beam_shape = 0;         // tensor-core kernel shape (beam_tc_pick)
  int corr_mode = CHIRP_CORR_FP32_SIMT;  // resolved CHIRP_CORR_*
  bool corr_forced = false;              // set explicitly (else AUTO)
  int in_type = CHIRP_IN_C64;
  float* d_scale = nullptr;   // [M] CHIRP_IN_CI8 scales
  cudaStream_t stream = nullptr;
  std::vector<Group> groups;
  std::vector<DmInfo> dmi;
  long long n_dump = 0;
  int n_pair = 0;
  // device workspace
  float2* d_tw = nullptr;    // [kTwiddleElems]: coarse, fine, stage pairs
  float2* d_x = nullptr;     // staging copy of host voltages [M][N]
  float2* d_Z = nullptr;     // inverse-row intermediate, largest group
  float2* d_H = nullptr;     // FP32 chirps of the current DMs [dm_chunk][h_stride]
  int dm_chunk = 1;          // DMs of one group whose row passes run together
  long long h_stride = 0;    // elements between chirp tables
  size_t z_stride = 0;       // elements between the DMs' inverse workspaces
  float2* d_y = nullptr;     // dedispersed voltages [y_slots][M][N] (allocated on first use)
  int y_slots = 1;           // DMs of a chunk whose voltages are held at once
  // CHIRP_FLAG_LEAN: one spectra buffer shared by the groups, each group's
  // spectra formed right before its DMs (spec_group: the group it holds)
  bool lean = false;
  float2* d_spec_shared = nullptr;
  int spec_group = -1;
  const void* spec_src = nullptr;
  float2* d_W = nullptr;     // beam weights [n_pix][M]
  uint8_t* d_aimg = nullptr; // tensor-core A image (split-BF16 weights)
  uint8_t* d_bimg = nullptr; // tensor-core B image of one DM (split-BF16 voltages)
  size_t bimg_bytes = 0;
  int* d_err = nullptr;      // device status word (bounded waits that timed out)
  float2* d_V = nullptr;     // visibilities [dm_chunk][n_dump][n_pair] (beam mode VIS)
  size_t v_stride = 0;       // elements between the DMs' visibilities
  float* d_wpair = nullptr;  // real pair weights, beam_vis_rows x beam_vis_ld (beam mode VIS)
  // true-delay beams (chirp_truedelay_run), allocated on first use
  float2* d_tdY = nullptr;   // beam spectra of a chunk of (block, pixel) sequences
  float2* d_tdZ = nullptr;   // their inverse-row intermediate
  long long td_cap = 0;      // sequences per chunk
  // incoherent filterbank search
  int fb_chan = 0, fb_int = 0, fb_n_dm = 0;
  long long T_fb = 0;
  int* d_fb_shift = nullptr;   // [fb_n_dm][fb_chan]
  float* d_fb_S = nullptr;     // [fb_chan][T_fb]
  float* d_fb_D = nullptr;     // staging for host outputs
  // candidate detection (chirp_detect), allocated on first use
  long long* d_first_last = nullptr;  // [2][n_dm] valid dump range (set up at creation)
  float* d_det_P = nullptr;           // staging of host powers
  float2* d_det_stats = nullptr;      // [n_dm][n_pix] (med, sigma)
  int* d_det_counts = nullptr;        // per chunk
  long long* d_det_offsets = nullptr; // per chunk + 1 (total)
  chirp_candidate* d_det_cand = nullptr;  // staging of host candidate lists
  long long det_cand_cap = 0;
  int* d_lists = nullptr;      // selective searches: block and dump index lists
  size_t lists_cap = 0;
  // CUDA-graph replay of full device-buffer searches (chirp_config.flags)
  bool use_graphs = false;
  struct GraphEntry {
    const void* in;
    void* out;
    int be;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  void* d_out = nullptr;     // staging for host outputs
  size_t out_bytes = 0;
  // Host buffers in page-locked memory: the input is copied in time chunks on
  // copy_stream and the forward transforms follow chunk by chunk; outputs go
  // back one DM slab at a time while later DMs are searched.
  cudaStream_t copy_stream = nullptr;
  // Full searches form the next chunk's chirp tables on side_stream while the
  // current chunk's column passes and back-ends run (d_H holds two sets of
  // dm_chunk tables): side_ev[0] orders side after main, side_ev[1 + set]
  // marks a table set complete.
  cudaStream_t side_stream = nullptr;
  cudaEvent_t side_ev[3] = {nullptr, nullptr, nullptr};
  int n_sm = 0;                        // SMs of the plan's device
  // and (device outputs) the chunk's beams from visibilities beside the next
  // chunk's passes: beam_ev[0] orders side after the correlator, beam_ev[1]
  // marks the beams done (the next correlator overwrites d_V after it)
  bool beam_side = false, beam_pending = false;
  cudaEvent_t beam_ev[2] = {nullptr, nullptr};
  // the beams of the last batched chunk, launched on the side stream after
  // the next chunk's row pass (so that they run beside its column passes)
  std::vector<VisJob> beam_jobs;
  cudaEvent_t io_ev = nullptr;         // search stream -> copy stream ordering
  std::vector<cudaEvent_t> in_ev;      // chunk k of the input has landed
  std::vector<long long> in_t1;        // samples [0, in_t1[k]) of every antenna
  int in_pending = 0;                  // chunks the forward pass has not consumed
  char* drain_host = nullptr;          // page-locked host output filled per DM
  const char* drain_dev = nullptr;
  size_t drain_per_dm = 0;
  std::vector<char> drained;
  size_t ws_bytes = 0;
  long long ifft_points = 0, valid_samples = 0;
  // optional per-stage event timing (chirp_stage_timing)
  bool timing = false;
  unsigned timing_mask = 0;  // stages timed: bit CHIRP_STAGE_*
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<int, int>>> ev_marks;  // stage, (start ev, stop ev)
  size_t ev_next = 0;
  double stage_ms[CHIRP_N_STAGES] = {0};
  long long stage_launches[CHIRP_N_STAGES] = {0};

  TwiddlePtrs tw() const { return twiddle_ptrs(d_tw); }
};

namespace {

bool tc_beams(const chirp_plan* p) {
  return p->beam_mode == CHIRP_BEAM_TC_3XBF16 || p->beam_mode == CHIRP_BEAM_TC_BF16;
}
// Beams from per-dump visibilities (exact FP32, or from BF16-rounded voltages).
bool vis_beams(const chirp_plan* p) {
  return p->beam_mode == CHIRP_BEAM_VIS || p->beam_mode == CHIRP_BEAM_VIS_BF16;
}

int dev_alloc(chirp_plan* p, void** ptr, size_t bytes, const char* what) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? CHIRP_ENOMEM : CHIRP_ECUDA,
                "cudaMalloc(%zu bytes) for %s failed: %s", bytes, what, cudaGetErrorString(e));
  }
  p->ws_bytes += bytes;
  return CHIRP_OK;
}

// The dedispersed-voltage buffer, allocated on the first call that needs it
// (the tensor-core beam path writes its own image and never does).
// Full searches keep one slot per DM of a row-pass chunk (unless the plan is
// lean or the slots would pass 4 GB), so that the chunk's back-ends run as
// one batched launch.
int ensure_y(chirp_plan* p) {
  if (p->d_y) return CHIRP_OK;
  const size_t slot = (size_t)p->M * p->N * sizeof(float2);
  p->y_slots = !p->lean && p->dm_chunk > 1 && p->dm_chunk * slot <= (4ull << 30) ? p->dm_chunk : 1;
  return dev_alloc(p, (void**)&p->d_y, p->y_slots * slot, "voltages");
}

void release(chirp_plan* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  for (auto& g : p->groups) {
    cudaFree(g.d_G);
    cudaFree(g.d_rtw);
    if (!p->lean) cudaFree(g.d_spec);
    cudaFree(g.d_tdph);
    cudaFree(g.d_tdrot);
  }
  cudaFree(p->d_tdY);
  cudaFree(p->d_tdZ);
  cudaFree(p->d_spec_shared);
  cudaFree(p->d_tw);
  cudaFree(p->d_x);
  cudaFree(p->d_Z);
  cudaFree(p->d_H);
  cudaFree(p->d_y);
  cudaFree(p->d_W);
  cudaFree(p->d_aimg);
  cudaFree(p->d_bimg);
  cudaFree(p->d_err);
  cudaFree(p->d_V);
  cudaFree(p->d_wpair);
  cudaFree(p->d_fb_shift);
  cudaFree(p->d_fb_S);
  cudaFree(p->d_fb_D);
  cudaFree(p->d_lists);
  cudaFree(p->d_scale);
  cudaFree(p->d_first_last);
  cudaFree(p->d_det_P);
  cudaFree(p->d_det_stats);
  cudaFree(p->d_det_counts);
  cudaFree(p->d_det_offsets);
  cudaFree(p->d_det_cand);
  for (auto& g : p->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  cudaFree(p->d_out);
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  if (p->copy_stream) {
    cudaStreamSynchronize(p->copy_stream);
    cudaStreamDestroy(p->copy_stream);
  }
  if (p->io_ev) cudaEventDestroy(p->io_ev);
  for (cudaEvent_t e : p->in_ev) cudaEventDestroy(e);
  if (p->side_stream) {
    cudaStreamSynchronize(p->side_stream);
    cudaStreamDestroy(p->side_stream);
  }
  for (cudaEvent_t e : p->side_ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : p->beam_ev)
    if (e) cudaEventDestroy(e);
}

// Two-pass FFT split autotuner.  Every split Nfft = n1 * n2 with the row
// length n2 in 256..4096 and the column length n1 in 16..4096 gives the same
// transform up to rounding; the kernels' memory behaviour differs (row tiles
// of 4096 points hold 4096 / n2 rows, column tiles 4096 / n1 columns).  The
// forward pass and one DM's inverse passes over the group's blocks are timed
// with CUDA events for each candidate (one warm-up, best of three) on the
// plan's own workspace, and the fastest split is kept for the (device, Nfft,
// antennas, blocks) key for the rest of the process.
cudaError_t autotune_split(chirp_plan* p, Group& g) {
  static std::mutex mu;
  static std::map<std::tuple<int, long long, int, long long>, int> cache;
  GroupGeom& G = g.geom;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_tuple(dev, G.nfft, p->M, G.n_blk);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      G.n2 = it->second;
      G.n1 = (int)(G.nfft / G.n2);
      return cudaSuccess;
    }
  }
  std::vector<int> cand;
  for (int n2 = 256; n2 <= 4096; n2 *= 2)
    if (G.nfft / n2 >= 16 && G.nfft / n2 <= 4096) cand.push_back(n2);
  const int n2_default = G.n2;
  if (cand.size() > 1) {
    const size_t ybytes = (size_t)p->M * p->N * sizeof(float2);
    e = cudaMemsetAsync(p->d_y, 0, ybytes, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_H, 0, (size_t)G.nfft * sizeof(float2), p->stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const long long n_seq = (long long)p->M * G.n_blk;
    const long long nq = inverse_chunk_sequences(G, n_seq);
    float best = 1e30f;
    int best_n2 = n2_default;
    for (int n2 : cand) {
      if (e != cudaSuccess) break;
      G.n2 = n2;
      G.n1 = (int)(G.nfft / n2);
      e = launch_build_row_twiddles(g.d_rtw, G, p->stream);
      if (e != cudaSuccess) break;
      auto pass = [&]() -> cudaError_t {
        cudaError_t r = launch_forward(p->d_y, p->N, p->M, G, g.d_spec, p->tw(), p->stream);
        for (long long q0 = 0; r == cudaSuccess && q0 < n_seq; q0 += nq) {
          const long long n = std::min(nq, n_seq - q0);
          r = launch_inverse_rows(g.d_spec, p->d_Z, p->d_H, q0, n, G, p->tw(), g.d_rtw,
                                  p->stream);
          if (r == cudaSuccess)
            r = launch_inverse_cols(p->d_Z, p->d_y, p->N, p->M, q0, n, G, G.n_hi_max, G.n_lo_max,
                                    p->tw(), p->stream);
        }
        return r;
      };
      e = pass();
      for (int rep = 0; e == cudaSuccess && rep < 3; rep++) {
        e = cudaEventRecord(e0, p->stream);
        if (e == cudaSuccess) e = pass();
        if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) {
          best = ms;
          best_n2 = n2;
        }
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    G.n2 = best_n2;
    G.n1 = (int)(G.nfft / G.n2);
  }
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = G.n2;
  return cudaSuccess;
}

// events bracketing one kernel launch of a stage (no-op unless timing is on
// for that stage)
int mark_begin(chirp_plan* p, int stage) {
  if (!p->timing || !((p->timing_mask >> stage) & 1u)) return -1;
  if (p->ev_next + 2 > p->ev_pool.size()) {
    for (int i = 0; i < 256; i++) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      p->ev_pool.push_back(e);
    }
  }
  int i = (int)p->ev_next;
  p->ev_next += 2;
  cudaEventRecord(p->ev_pool[i], p->stream);
  return i;
}
void mark_end(chirp_plan* p, int stage, int i) {
  if (i < 0) return;
  cudaEventRecord(p->ev_pool[i + 1], p->stream);
  p->ev_marks.push_back({stage, {i, i + 1}});
}
// fold recorded events into the per-stage totals (synchronises the stream)
void collect_marks(chirp_plan* p) {
  if (p->ev_marks.empty()) return;
  cudaStreamSynchronize(p->stream);
  for (auto& m : p->ev_marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev_pool[m.second.first], p->ev_pool[m.second.second]) ==
        cudaSuccess) {
      p->stage_ms[m.first] += ms;
      p->stage_launches[m.first] += 1;
    }
  }
  p->ev_marks.clear();
  p->ev_next = 0;
}

int validate(const chirp_config* c) {
  if (!c) return fail(CHIRP_EINVAL, "config is NULL");
  if (c->n_ant < 1 || c->n_ant > 84) return fail(CHIRP_EINVAL, "n_ant must be in 1..84");
  if (!(c->f0_hz > 0) || !(c->bw_hz > 0) || !(c->bw_hz < 2 * c->f0_hz))
    return fail(CHIRP_EINVAL, "need f0 > 0 and 0 < bw < 2 f0");
  if (c->n_samp < 1) return fail(CHIRP_EINVAL, "n_samp must be >= 1");
  if (!c->dm || c->n_dm < 1) return fail(CHIRP_EINVAL, "need at least one DM");
  for (int d = 0; d < c->n_dm; d++)
    if (!(c->dm[d] >= 0) || !std::isfinite(c->dm[d]))
      return fail(CHIRP_EINVAL, "DM %d is negative or not finite", d);
  if (c->dump_len < 1 || c->dump_len > c->n_samp)
    return fail(CHIRP_EINVAL, "dump_len must be in 1..n_samp");
  if (!is_pow2(c->nfft_min) || c->nfft_min < 256 || c->nfft_min > (1LL << 24))
    return fail(CHIRP_EINVAL, "nfft_min must be a power of two in 256..2^24");
  if (c->fft_row != 0 && (!is_pow2(c->fft_row) || c->fft_row < 256 || c->fft_row > 4096))
    return fail(CHIRP_EINVAL, "fft_row must be 0 or a power of two in 256..4096");
  if (c->beam_shape < 0 || c->beam_shape > 3)
    return fail(CHIRP_EINVAL, "beam_shape must be 0..3");
  if (c->corr_mode < 0 || c->corr_mode > CHIRP_CORR_TC_BF16)
    return fail(CHIRP_EINVAL, "unknown corr_mode");
  if (c->flags & ~(CHIRP_FLAG_GRAPHS | CHIRP_FLAG_AUTOTUNE | CHIRP_FLAG_LEAN))
    return fail(CHIRP_EINVAL, "unknown flag bits 0x%x", c->flags);
  if (c->n_pix < 0) return fail(CHIRP_EINVAL, "n_pix must be >= 0");
  if (c->n_pix > 0 && (!c->pix_lm || !c->xyz_m))
    return fail(CHIRP_EINVAL, "beams need pix_lm and xyz_m");
  if (c->n_pix > 0)
    for (int p = 0; p < c->n_pix; p++) {
      double l = c->pix_lm[2 * p], m = c->pix_lm[2 * p + 1];
      if (!(l * l + m * m <= 1.0)) return fail(CHIRP_EINVAL, "pixel %d has l^2 + m^2 > 1", p);
    }
  if (c->beam_mode < 0 || c->beam_mode > CHIRP_BEAM_VIS_BF16)
    return fail(CHIRP_EINVAL, "unknown beam_mode");
  if (c->in_type != CHIRP_IN_C64 && c->in_type != CHIRP_IN_CI8)
    return fail(CHIRP_EINVAL, "unknown in_type");
  if (c->in_type == CHIRP_IN_CI8 && c->in_scale)
    for (int a = 0; a < c->n_ant; a++)
      if (!std::isfinite(c->in_scale[a])) return fail(CHIRP_EINVAL, "in_scale must be finite");
  if (c->fb_chan != 0) {
    if (!is_pow2(c->fb_chan) || c->fb_chan < 16 || c->fb_chan > 4096)
      return fail(CHIRP_EINVAL, "fb_chan must be 0 or a power of two in 16..4096");
    if (c->fb_int < 1) return fail(CHIRP_EINVAL, "fb_int must be >= 1");
    if (!c->fb_dm || c->fb_n_dm < 1) return fail(CHIRP_EINVAL, "fb_dm needs at least one DM");
    for (int d = 0; d < c->fb_n_dm; d++)
      if (!(c->fb_dm[d] >= 0) || !std::isfinite(c->fb_dm[d]))
        return fail(CHIRP_EINVAL, "fb_dm %d is negative or not finite", d);
  }
  return CHIRP_OK;
}

}  // namespace

extern "C" {

const char* chirp_last_error(void) { return g_err; }

int chirp_stage_timing(chirp_plan* p, int enable, double* ms, long long* launches) {
  if (!p) return fail(CHIRP_EINVAL, "plan is NULL");
  collect_marks(p);
  if (ms)
    for (int i = 0; i < CHIRP_N_STAGES; i++) ms[i] = p->stage_ms[i];
  if (launches)
    for (int i = 0; i < CHIRP_N_STAGES; i++) launches[i] = p->stage_launches[i];
  for (int i = 0; i < CHIRP_N_STAGES; i++) {
    p->stage_ms[i] = 0;
    p->stage_launches[i] = 0;
  }
  p->timing = enable != 0;
  p->timing_mask = (enable & CHIRP_TIMING_SELECT) ? (unsigned)enable & ((1u << CHIRP_N_STAGES) - 1u)
                                                  : (1u << CHIRP_N_STAGES) - 1u;
  return CHIRP_OK;
}

int chirp_plan_create(chirp_plan** out, const chirp_config* cfg, void* stream) {
  g_err[0] = 0;
  if (!out) return fail(CHIRP_EINVAL, "plan pointer is NULL");
  *out = nullptr;
  int rc = validate(cfg);
  if (rc) return rc;
  chirp_plan* p = new (std::nothrow) chirp_plan();
  if (!p) return fail(CHIRP_ENOMEM, "host allocation failed");
  p->M = cfg->n_ant;
  if (cfg->xyz_m) p->xyz.assign(cfg->xyz_m, cfg->xyz_m + 3 * cfg->n_ant);
  p->f0 = cfg->f0_hz;
  p->bw = cfg->bw_hz;
  p->kdm = cfg->k_dm > 0 ? cfg->k_dm : kDefaultKdm;
  p->N = cfg->n_samp;
  p->dm.assign(cfg->dm, cfg->dm + cfg->n_dm);
  p->L = cfg->dump_len;
  p->nfft_min = cfg->nfft_min;
  if (cfg->n_pix > 0) p->pix.assign(cfg->pix_lm, cfg->pix_lm + 2 * cfg->n_pix);
  p->n_pix = cfg->n_pix;
  // AUTO: the faster of the two exact (FP32-accurate) forms, by the cost model
  // of vis_beats_gemm; the visibility identity also where no tensor-core
  // shape fits
  p->beam_mode = cfg->beam_mode;
  if (p->beam_mode == CHIRP_BEAM_AUTO)
    p->beam_mode = cfg->n_pix > 0 && (beam_tc_pick(cfg->n_ant, cfg->n_pix, cfg->dump_len, 3, 0) == 0 ||
                                      vis_beats_gemm(cfg->n_ant, cfg->n_pix, cfg->dump_len))
                       ? CHIRP_BEAM_VIS
                       : CHIRP_BEAM_TC_3XBF16;
  p->beam_terms = p->beam_mode == CHIRP_BEAM_TC_BF16 ? 1 : 3;
  p->corr_mode = cfg->corr_mode;
  p->corr_forced = cfg->corr_mode != CHIRP_CORR_AUTO;
  // AUTO: up to 16 antennas the staged FP32 correlator (12 antennas, 2^22
  // samples, 64 DMs: 6.0 ms against 9.5 ms per search for the tensor cores,
  // whose 128-row MMA tiles carry 24 useful rows there); above, the tensor
  // cores (36 antennas: 1.6x faster than the CUDA cores)
  if (p->corr_mode == CHIRP_CORR_AUTO)
    p->corr_mode = cfg->n_ant > 16 && corr_tc_supported(cfg->n_ant, cfg->dump_len, 3)
                       ? CHIRP_CORR_TC_3XBF16
                       : CHIRP_CORR_FP32_SIMT;
  if (p->corr_mode != CHIRP_CORR_FP32_SIMT &&
      !corr_tc_supported(cfg->n_ant, cfg->dump_len, p->corr_mode == CHIRP_CORR_TC_BF16 ? 1 : 3)) {
    delete p;
    return fail(CHIRP_EUNSUPPORTED,
                "tensor-core correlation needs a dump length that lines up with its 128- or "
                "256-sample chunks and an antenna count whose operands fit (48 for split-BF16, "
                "84 for BF16)");
  }
  if (cfg->n_pix > 0 && tc_beams(p)) {
    p->beam_shape = beam_tc_pick(p->M, cfg->n_pix, cfg->dump_len, p->beam_terms, cfg->beam_shape);
    if (p->beam_shape == 0) {
      delete p;
      return fail(CHIRP_EUNSUPPORTED,
                  cfg->beam_shape ? "the requested tensor-core beam kernel shape does not fit this "
                                    "search"
                                  : "tensor-core beam tiles for these antennas do not fit in "
                                    "shared memory; use CHIRP_BEAM_VIS or CHIRP_BEAM_FP32_SIMT");
    }
  }
  p->in_type = cfg->in_type;
  p->stream = (cudaStream_t)stream;
  p->use_graphs = (cfg->flags & CHIRP_FLAG_GRAPHS) != 0;
  p->lean = (cfg->flags & CHIRP_FLAG_LEAN) != 0;
  if (p->use_graphs && p->stream == nullptr) {
    delete p;
    return fail(CHIRP_EINVAL, "CUDA graphs need a plan stream other than the legacy default stream");
  }
  p->n_dump = p->N / p->L;
  p->n_pair = p->M * (p->M + 1) / 2;

  // ---- per-DM FFT length and groups
  const int n_dm = (int)p->dm.size();
  std::vector<long long> nfft(n_dm), hi(n_dm), lo(n_dm);
  for (int d = 0; d < n_dm; d++) {
    sweep(p->f0, p->bw, p->kdm, p->dm[d], &hi[d], &lo[d]);
    long long nd = hi[d] + lo[d];
    long long want = pow2ceil(2 * nd > 1 ? 2 * nd : 1);
    long long cap = pow2ceil(p->N);
    long long n = std::min(want, cap);
    nfft[d] = std::max(n, p->nfft_min);
    if (nfft[d] > (1LL << 24)) {
      delete p;
      return fail(CHIRP_EUNSUPPORTED, "DM %g needs an FFT of %lld points (> 2^24)", p->dm[d],
                  nfft[d]);
    }
  }
  p->dmi.resize(n_dm);
  for (int d = 0; d < n_dm; d++) {
    int gi = -1;
    for (size_t g = 0; g < p->groups.size(); g++)
      if (p->groups[g].geom.nfft == nfft[d]) gi = (int)g;
    if (gi < 0) {
      Group g;
      std::memset(&g.geom, 0, sizeof g.geom);
      g.geom.nfft = nfft[d];
      p->groups.push_back(g);
      gi = (int)p->groups.size() - 1;
    }
    p->groups[gi].dms.push_back(d);
    p->dmi[d].group = gi;
  }
  for (auto& g : p->groups) {
    GroupGeom& G = g.geom;
    G.log2n = ilog2ll(G.nfft);
    G.n1 = (int)std::max<long long>(16, G.nfft / 4096);
    G.n2 = (int)(G.nfft / G.n1);
    if (cfg->fft_row > 0 && G.nfft / cfg->fft_row >= 16 && G.nfft / cfg->fft_row <= 4096) {
      G.n2 = cfg->fft_row;
      G.n1 = (int)(G.nfft / G.n2);
    }
    G.n_hi_max = 0;
    G.n_lo_max = 0;
    for (int d : g.dms) {
      G.n_hi_max = std::max(G.n_hi_max, hi[d]);
      G.n_lo_max = std::max(G.n_lo_max, lo[d]);
    }
    G.step = G.nfft - G.n_hi_max - G.n_lo_max;
    if (G.step >= 8) G.step -= G.step % 8;  // blocks start on multiples of 8 samples
    if (p->N <= G.nfft) {
      G.n_blk = 1;
    } else {
      if (G.step <= 0) {
        delete p;
        return fail(CHIRP_EINVAL, "internal: non-positive block step");
      }
      G.n_blk = (p->N - G.nfft + G.step - 1) / G.step + 1;
    }
    if ((long long)p->M * G.n_blk > 65535) {
      delete p;
      return fail(CHIRP_EUNSUPPORTED, "n_ant * blocks = %lld exceeds 65535",
                  (long long)p->M * G.n_blk);
    }
  }
  for (int d = 0; d < n_dm; d++) {
    DmInfo& I = p->dmi[d];
    I.n_hi = hi[d];
    I.n_lo = lo[d];
    I.first = (I.n_hi + p->L - 1) / p->L;
    long long end = p->N - I.n_lo;
    I.last = end >= 0 ? end / p->L - 1 : -1;
    const GroupGeom& G = p->groups[I.group].geom;
    p->ifft_points += (long long)p->M * G.n_blk * G.nfft;
    long long v = p->N - I.n_hi - I.n_lo;
    p->valid_samples += (long long)p->M * (v > 0 ? v : 0);
  }

  // ---- device workspace
  rc = dev_alloc(p, (void**)&p->d_tw, kTwiddleElems * sizeof(float2), "twiddles");
  size_t z_elems = 0, max_spec = 0;
  for (auto& g : p->groups)
    max_spec = std::max(max_spec, (size_t)p->M * (size_t)g.geom.n_blk * (size_t)g.geom.nfft);
  if (!rc && p->lean)
    rc = dev_alloc(p, (void**)&p->d_spec_shared, max_spec * sizeof(float2), "spectra (shared)");
  for (auto& g : p->groups) {
    size_t elems = (size_t)p->M * g.geom.n_blk * g.geom.nfft;
    z_elems = std::max(z_elems, (size_t)inverse_chunk_sequences(g.geom, (long long)p->M * g.geom.n_blk) *
                                    (size_t)g.geom.nfft);
    if (p->lean)
      g.d_spec = p->d_spec_shared;
    else if (!rc)
      rc = dev_alloc(p, (void**)&g.d_spec, elems * sizeof(float2), "spectra");
    if (!rc) rc = dev_alloc(p, (void**)&g.d_G, g.geom.nfft * sizeof(double), "phase table");
    if (!rc)
      rc = dev_alloc(p, (void**)&g.d_rtw, g.geom.nfft / 16 * sizeof(float2), "row twiddles");
  }
  // Full searches run the row pass of up to 4 DMs of a group together (the
  // spectrum is read once for them), each with its own workspace, as long
  // as those workspaces stay within 4 GB and no group is chunked.
  bool chunked = false;
  for (auto& g : p->groups)
    chunked |= inverse_chunk_sequences(g.geom, (long long)p->M * g.geom.n_blk) <
               (long long)p->M * g.geom.n_blk;
  p->dm_chunk = 1;
  if (!chunked)
    while (p->dm_chunk < kMaxChirps && (size_t)(p->dm_chunk + 1) * z_elems * sizeof(float2) <= (4ull << 30))
      p->dm_chunk++;
  p->z_stride = z_elems;
  if (!rc)
    rc = dev_alloc(p, (void**)&p->d_Z, (size_t)p->dm_chunk * z_elems * sizeof(float2),
                   "inverse workspace");
  long long max_nfft = 0;
  for (auto& g : p->groups) max_nfft = std::max(max_nfft, g.geom.nfft);
  p->h_stride = max_nfft;
  if (!rc)
    rc = dev_alloc(p, (void**)&p->d_H, (size_t)2 * p->dm_chunk * max_nfft * sizeof(float2),
                   "chirp tables (two sets)");
  // (the dedispersed-voltage buffer d_y is allocated on first use: ensure_y)
  if (!rc && p->n_pix > 0)
    rc = dev_alloc(p, (void**)&p->d_W, (size_t)p->n_pix * p->M * sizeof(float2), "weights");
  if (!rc) rc = dev_alloc(p, (void**)&p->d_err, sizeof(int), "status word");
  std::vector<long long> first_last(2 * p->dmi.size());
  for (size_t d = 0; d < p->dmi.size(); d++) {
    first_last[d] = p->dmi[d].first;
    first_last[p->dmi.size() + d] = p->dmi[d].last;
  }
  if (!rc) rc = dev_alloc(p, (void**)&p->d_first_last, first_last.size() * sizeof(long long),
                          "dump ranges");
  std::vector<float> scale;
  if (!rc && p->in_type == CHIRP_IN_CI8) {
    scale.assign((size_t)p->M, 1.0f);
    if (cfg->in_scale) std::copy(cfg->in_scale, cfg->in_scale + p->M, scale.begin());
    rc = dev_alloc(p, (void**)&p->d_scale, scale.size() * sizeof(float), "input scales");
  }
  std::vector<int> fb_shift;
  if (!rc && cfg->fb_chan > 0) {
    p->fb_chan = cfg->fb_chan;
    p->fb_int = cfg->fb_int;
    p->fb_n_dm = cfg->fb_n_dm;
    p->T_fb = p->N / ((long long)p->fb_chan * p->fb_int);
    const double t_fb = (double)p->fb_chan * (double)p->fb_int / p->bw;
    fb_shift.resize((size_t)p->fb_n_dm * p->fb_chan);
    for (int d = 0; d < p->fb_n_dm; d++)
      for (int c = 0; c < p->fb_chan; c++) {
        // Eq. dmdelay lag of channel c relative to f0, in filterbank samples
        const double fc = p->f0 + (double)(c - p->fb_chan / 2) * p->bw / (double)p->fb_chan;
        const double tau = p->kdm * cfg->fb_dm[d] * (1.0 / (fc * fc) - 1.0 / (p->f0 * p->f0));
        fb_shift[(size_t)d * p->fb_chan + c] = (int)std::floor(tau / t_fb + 0.5);
      }
    rc = dev_alloc(p, (void**)&p->d_fb_shift, fb_shift.size() * sizeof(int), "fb shifts");
    if (!rc)
      rc = dev_alloc(p, (void**)&p->d_fb_S,
                     (size_t)std::max(1LL, p->T_fb) * p->fb_chan * sizeof(float), "filterbank");
  }
  std::vector<uint8_t> aimg;
  std::vector<float> wpair;
  if (!rc && p->n_pix > 0 && vis_beams(p)) {
    p->v_stride = (size_t)std::max(1LL, p->n_dump) * p->n_pair;
    rc = dev_alloc(p, (void**)&p->d_V, (size_t)p->dm_chunk * p->v_stride * sizeof(float2),
                   "visibilities");
    const size_t wrows = (size_t)beam_vis_rows(p->M), wld = (size_t)beam_vis_ld(p->n_pix);
    if (!rc) rc = dev_alloc(p, (void**)&p->d_wpair, wrows * wld * sizeof(float), "pair weights");
    if (!rc) {
      wpair.assign(wrows * wld, 0.0f);
      std::vector<double> wr(p->M), wi(p->M);
      for (int q = 0; q < p->n_pix; q++) {
        double l = p->pix[2 * q], m = p->pix[2 * q + 1];
        double n = std::sqrt(1.0 - l * l - m * m);
        for (int a = 0; a < p->M; a++) {
          double tau = (p->xyz[3 * a] * l + p->xyz[3 * a + 1] * m + p->xyz[3 * a + 2] * (n - 1.0)) /
                       kCLight;
          double ph = 2.0 * kPi * p->f0 * tau;
          wr[a] = std::cos(ph);
          wi[a] = std::sin(ph);
        }
        int k = 0;
        for (int a = 0; a < p->M; a++)
          for (int b = a; b < p->M; b++, k++) {
            const double c = a == b ? 1.0 : 2.0;  // W_a conj(W_b), doubled above the diagonal
            // Re P gets Re w Re V - Im w Im V: rows 2k (Re w) and 2k+1 (-Im w)
            wpair[(2 * (size_t)k) * wld + q] = (float)(c * (wr[a] * wr[b] + wi[a] * wi[b]));
            wpair[(2 * (size_t)k + 1) * wld + q] = (float)(-c * (wi[a] * wr[b] - wr[a] * wi[b]));
          }
      }
    }
  }
  if (!rc && p->n_pix > 0 && tc_beams(p)) {
    long long max_tiles = 0;
    for (const DmInfo& I : p->dmi)
      if (I.last >= I.first) {
        long long span = (I.last - I.first + 1) * p->L;
        const int ts = beam_tc_tile_samples(p->beam_shape);
        long long nt = (span + ts - 1) / ts;
        max_tiles = std::max(max_tiles, nt);
      }
    p->bimg_bytes = (size_t)std::max(1LL, max_tiles) *
                    (size_t)beam_tc_tile_bytes(p->M, p->beam_shape, p->beam_terms);
    rc = dev_alloc(p, (void**)&p->d_bimg, p->bimg_bytes, "beam B image");
    if (!rc) {
      std::vector<double> Wd((size_t)p->n_pix * p->M * 2);
      for (int q = 0; q < p->n_pix; q++) {
        double l = p->pix[2 * q], m = p->pix[2 * q + 1];
        double n = std::sqrt(1.0 - l * l - m * m);
        for (int a = 0; a < p->M; a++) {
          double tau = (p->xyz[3 * a] * l + p->xyz[3 * a + 1] * m + p->xyz[3 * a + 2] * (n - 1.0)) /
                       kCLight;
          double ph = 2.0 * kPi * p->f0 * tau;
          Wd[2 * ((size_t)q * p->M + a)] = std::cos(ph);
          Wd[2 * ((size_t)q * p->M + a) + 1] = std::sin(ph);
        }
      }
      aimg = build_beam_a_image(Wd.data(), p->M, p->n_pix, p->beam_terms);
      rc = dev_alloc(p, (void**)&p->d_aimg, aimg.size(), "beam A image");
    }
  }
  if (rc) {
    release(p);
    delete p;
    return rc;
  }

  // ---- beam weights W_pa = exp(+2 pi j f0 tau_a(l_p, m_p)), Eq. tau3D
  std::vector<float2> W((size_t)p->n_pix * p->M);
  for (int q = 0; q < p->n_pix; q++) {
    double l = p->pix[2 * q], m = p->pix[2 * q + 1];
    double n = std::sqrt(1.0 - l * l - m * m);
    for (int a = 0; a < p->M; a++) {
      double tau = (p->xyz[3 * a] * l + p->xyz[3 * a + 1] * m + p->xyz[3 * a + 2] * (n - 1.0)) /
                   kCLight;
      double ph = 2.0 * kPi * p->f0 * tau;
      W[(size_t)q * p->M + a] = make_float2((float)std::cos(ph), (float)std::sin(ph));
    }
  }
  cudaError_t e = launch_build_twiddles(p->d_tw, p->stream);
  if (e == cudaSuccess && p->n_pix > 0)
    e = cudaMemcpyAsync(p->d_W, W.data(), W.size() * sizeof(float2), cudaMemcpyHostToDevice,
                        p->stream);
  if (e == cudaSuccess && !wpair.empty())
    e = cudaMemcpyAsync(p->d_wpair, wpair.data(), wpair.size() * sizeof(float),
                        cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess && !aimg.empty())
    e = cudaMemcpyAsync(p->d_aimg, aimg.data(), aimg.size(), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_err, 0, sizeof(int), p->stream);
  // the B image slots of absent antennas (n_ant % 4) and of the padding
  // k-group are never written and must read as zeros
  if (e == cudaSuccess && p->d_bimg) e = cudaMemsetAsync(p->d_bimg, 0, p->bimg_bytes, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_first_last, first_last.data(), first_last.size() * sizeof(long long),
                        cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess && !scale.empty())
    e = cudaMemcpyAsync(p->d_scale, scale.data(), scale.size() * sizeof(float),
                        cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess && !fb_shift.empty())
    e = cudaMemcpyAsync(p->d_fb_shift, fb_shift.data(), fb_shift.size() * sizeof(int),
                        cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess && (cfg->flags & CHIRP_FLAG_AUTOTUNE) && cfg->fft_row == 0) {
    if (ensure_y(p)) {
      release(p);
      delete p;
      return CHIRP_ENOMEM;
    }
    for (auto& g : p->groups)
      if (e == cudaSuccess) e = autotune_split(p, g);
  }
  for (auto& g : p->groups) {
    if (e == cudaSuccess)
      e = launch_build_phase_table(g.d_G, g.geom, p->f0, p->bw, p->kdm, p->stream);
    if (e == cudaSuccess) e = launch_build_row_twiddles(g.d_rtw, g.geom, p->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    release(p);
    delete p;
    return fail(CHIRP_ECUDA, "plan set-up failed: %s", cudaGetErrorString(e));
  }
  *out = p;
  return CHIRP_OK;
}

void chirp_plan_destroy(chirp_plan* p) {
  release(p);
  delete p;
}

int chirp_plan_query(const chirp_plan* p, chirp_plan_info* info) {
  if (!p || !info) return fail(CHIRP_EINVAL, "NULL argument");
  info->n_dump = p->n_dump;
  info->n_pair = p->n_pair;
  info->n_group = (int)p->groups.size();
  info->workspace_bytes = (long long)p->ws_bytes;
  info->ifft_points = p->ifft_points;
  info->valid_samples = p->valid_samples;
  info->beam_mode = p->beam_mode;
  info->beam_shape = p->beam_shape;
  info->corr_mode = p->corr_mode;
  info->dm_chunk = p->dm_chunk;
  info->fb_samples = p->T_fb;
  return CHIRP_OK;
}

int chirp_dm_layout(const chirp_plan* p, int d, long long* out7) {
  if (!p || !out7 || d < 0 || d >= (int)p->dm.size()) return fail(CHIRP_EINVAL, "bad argument");
  const DmInfo& I = p->dmi[d];
  const GroupGeom& G = p->groups[I.group].geom;
  out7[0] = G.nfft;
  out7[1] = I.n_hi;
  out7[2] = I.n_lo;
  out7[3] = G.n_hi_max;
  out7[4] = G.n_lo_max;
  out7[5] = G.step;
  out7[6] = G.n_blk;
  return CHIRP_OK;
}

int chirp_dump_range(const chirp_plan* p, long long* first, long long* last) {
  if (!p || !first || !last) return fail(CHIRP_EINVAL, "NULL argument");
  for (size_t d = 0; d < p->dmi.size(); d++) {
    first[d] = p->dmi[d].first;
    last[d] = p->dmi[d].last;
  }
  return CHIRP_OK;
}

}  // extern "C"

namespace {

// voltages on the device, copying host input into the plan's staging buffer
size_t in_elem_bytes(const chirp_plan* p) {
  return p->in_type == CHIRP_IN_CI8 ? 2 : sizeof(float2);
}

bool host_pinned(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

constexpr int kInputChunks = 8;

// The copy stream and its events, created on first use.
int ensure_copy_stream(chirp_plan* p) {
  if (p->copy_stream) return CHIRP_OK;
  CK(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&p->io_ev, cudaEventDisableTiming));
  p->in_ev.assign(kInputChunks, nullptr);
  for (auto& e : p->in_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return CHIRP_OK;
}

// Host voltages go to the staging buffer.  chunked: page-locked input is
// copied in kInputChunks time chunks (all antennas) on the copy stream, and
// the forward pass (forward_all) waits for each chunk before transforming the
// blocks it completes; otherwise the search stream waits for the whole input.
int stage_input(chirp_plan* p, const void* volt, int loc, const void** dx, bool chunked = false) {
  p->in_pending = 0;
  if (!volt) return fail(CHIRP_EINVAL, "voltage pointer is NULL");
  if (loc == CHIRP_DEVICE) {
    *dx = volt;
    return CHIRP_OK;
  }
  if (loc != CHIRP_HOST) return fail(CHIRP_EINVAL, "bad buffer location");
  const size_t eb = in_elem_bytes(p);
  const size_t bytes = (size_t)p->M * p->N * eb;
  if (!p->d_x) {
    int rc = dev_alloc(p, (void**)&p->d_x, bytes, "input staging");
    if (rc) return rc;
  }
  *dx = p->d_x;
  if (!chunked || p->lean || !host_pinned(volt)) {
    CK(cudaMemcpyAsync(p->d_x, volt, bytes, cudaMemcpyHostToDevice, p->stream));
    return CHIRP_OK;
  }
  int rc = ensure_copy_stream(p);
  if (rc) return rc;
  // the staging buffer is free once the search stream's earlier work is done
  CK(cudaEventRecord(p->io_ev, p->stream));
  CK(cudaStreamWaitEvent(p->copy_stream, p->io_ev, 0));
  const long long per = (p->N + kInputChunks - 1) / kInputChunks;
  p->in_t1.assign(kInputChunks, p->N);
  for (int k = 0; k < kInputChunks; k++) {
    const long long t0 = std::min(p->N, k * per), t1 = std::min(p->N, t0 + per);
    if (t1 > t0)
      CK(cudaMemcpy2DAsync((char*)p->d_x + t0 * eb, p->N * eb, (const char*)volt + t0 * eb,
                           p->N * eb, (t1 - t0) * eb, p->M, cudaMemcpyHostToDevice,
                           p->copy_stream));
    CK(cudaEventRecord(p->in_ev[k], p->copy_stream));
    p->in_t1[k] = t1;
  }
  p->in_pending = kInputChunks;
  return CHIRP_OK;
}

// The search stream waits for whatever input chunks are still in flight.
int input_wait_all(chirp_plan* p) {
  if (p->in_pending > 0) CK(cudaStreamWaitEvent(p->stream, p->in_ev[kInputChunks - 1], 0));
  p->in_pending = 0;
  return CHIRP_OK;
}

// Page-locked host output: slabs of whole DMs are copied back on the copy
// stream as their back-end finishes (drain_dm), the rest at the end.
int drain_begin(chirp_plan* p, void* user, const void* dev, size_t bytes) {
  p->drain_host = nullptr;
  if (!host_pinned(user) || p->dm.empty()) return CHIRP_OK;
  int rc = ensure_copy_stream(p);
  if (rc) return rc;
  p->drain_host = (char*)user;
  p->drain_dev = (const char*)dev;
  p->drain_per_dm = bytes / p->dm.size();
  p->drained.assign(p->dm.size(), 0);
  return CHIRP_OK;
}

int drain_dm(chirp_plan* p, int d) {
  if (!p->drain_host || p->drained[(size_t)d]) return CHIRP_OK;
  CK(cudaEventRecord(p->io_ev, p->stream));
  CK(cudaStreamWaitEvent(p->copy_stream, p->io_ev, 0));
  const size_t off = (size_t)d * p->drain_per_dm;
  CK(cudaMemcpyAsync(p->drain_host + off, p->drain_dev + off, p->drain_per_dm,
                     cudaMemcpyDeviceToHost, p->copy_stream));
  p->drained[(size_t)d] = 1;
  return CHIRP_OK;
}

int out_buffer(chirp_plan* p, void* user, int loc, size_t bytes, void** dev) {
  if (!user) return fail(CHIRP_EINVAL, "output pointer is NULL");
  if (loc == CHIRP_DEVICE) {
    *dev = user;
    return CHIRP_OK;
  }
  if (loc != CHIRP_HOST) return fail(CHIRP_EINVAL, "bad buffer location");
  if (p->out_bytes < bytes) {
    cudaFree(p->d_out);
    p->d_out = nullptr;
    p->out_bytes = 0;
    int rc = dev_alloc(p, &p->d_out, bytes, "output staging");
    if (rc) return rc;
    p->out_bytes = bytes;
  }
  *dev = p->d_out;
  return CHIRP_OK;
}

int finish_out(chirp_plan* p, void* user, int loc, const void* dev, size_t bytes) {
  if (loc != CHIRP_HOST) return CHIRP_OK;
  if (p->drain_host) {
    for (int d = 0; d < (int)p->dm.size(); d++) {
      int rc = drain_dm(p, d);
      if (rc) return rc;
    }
    p->drain_host = nullptr;
    CK(cudaStreamSynchronize(p->copy_stream));
  } else {
    CK(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, p->stream));
  }
  CK(cudaStreamSynchronize(p->stream));
  return CHIRP_OK;
}

int forward_all(chirp_plan* p, const void* dx) {
  if (p->lean) {  // spectra are formed per group, right before its DMs
    int rc = input_wait_all(p);
    if (rc) return rc;
    p->spec_group = -1;
    p->spec_src = dx;
    return CHIRP_OK;
  }
  if (p->in_pending > 0) {
    // chunk by chunk: every group transforms the blocks the chunk completes
    // (block b reads samples [b step, b step + nfft))
    std::vector<long long> done(p->groups.size(), 0);
    for (int k = 0; k < kInputChunks; k++) {
      CK(cudaStreamWaitEvent(p->stream, p->in_ev[k], 0));
      const long long t1 = p->in_t1[k];
      for (size_t gi = 0; gi < p->groups.size(); gi++) {
        Group& g = p->groups[gi];
        const GroupGeom& G = g.geom;
        long long ready = G.n_blk;
        if (t1 < p->N) ready = t1 >= G.nfft ? std::min(G.n_blk, (t1 - G.nfft) / G.step + 1) : 0;
        if (ready <= done[gi]) continue;
        int mk = mark_begin(p, CHIRP_STAGE_FORWARD);
        CK(launch_forward(dx, p->N, p->M, G, g.d_spec, p->tw(), p->stream, p->in_type, p->d_scale,
                          done[gi], ready));
        mark_end(p, CHIRP_STAGE_FORWARD, mk);
        done[gi] = ready;
      }
    }
    p->in_pending = 0;
    return CHIRP_OK;
  }
  for (auto& g : p->groups) {
    int mk = mark_begin(p, CHIRP_STAGE_FORWARD);
    CK(launch_forward(dx, p->N, p->M, g.geom, g.d_spec, p->tw(), p->stream, p->in_type,
                      p->d_scale));
    mark_end(p, CHIRP_STAGE_FORWARD, mk);
  }
  return CHIRP_OK;
}

// Lean plans: the shared spectra buffer holds group gi's spectra of the
// current input afterwards (formed now unless it already does).
int ensure_spec(chirp_plan* p, int gi) {
  if (!p->lean || p->spec_group == gi) return CHIRP_OK;
  Group& g = p->groups[gi];
  int mk = mark_begin(p, CHIRP_STAGE_FORWARD);
  CK(launch_forward(p->spec_src, p->N, p->M, g.geom, g.d_spec, p->tw(), p->stream, p->in_type,
                    p->d_scale));
  mark_end(p, CHIRP_STAGE_FORWARD, mk);
  p->spec_group = gi;
  return CHIRP_OK;
}

// Dedisperse DM d over the blocks [b0, b1) of its group (all antennas).
int dedisperse_blocks(chirp_plan* p, int d, float2* y, long long b0, long long b1,
                      const BeamImageOut* img = nullptr, bool y16 = false) {
  const DmInfo& I = p->dmi[d];
  Group& g = p->groups[I.group];
  const long long q_end = b1 * p->M;
  const long long nq = inverse_chunk_sequences(g.geom, (long long)p->M * g.geom.n_blk);
  for (long long q0 = b0 * p->M; q0 < q_end; q0 += nq) {
    const long long n = std::min(nq, q_end - q0);
    int mk = mark_begin(p, CHIRP_STAGE_INV_ROWS);
    CK(launch_inverse_rows(g.d_spec, p->d_Z, p->d_H, q0, n, g.geom, p->tw(), g.d_rtw,
                           p->stream));
    mark_end(p, CHIRP_STAGE_INV_ROWS, mk);
    mk = mark_begin(p, CHIRP_STAGE_INV_COLS);
    if (y16)
      CK(launch_inverse_cols_bf16(p->d_Z, y, p->N, p->M, q0, n, g.geom, I.n_hi, I.n_lo, p->tw(),
                                  p->stream));
    else
      CK(launch_inverse_cols(p->d_Z, y, p->N, p->M, q0, n, g.geom, I.n_hi, I.n_lo, p->tw(),
                             p->stream, nullptr, img));
    mark_end(p, CHIRP_STAGE_INV_COLS, mk);
  }
  return CHIRP_OK;
}

int chirp_for(chirp_plan* p, int d, int slot = 0) {
  const DmInfo& I = p->dmi[d];
  int mk = mark_begin(p, CHIRP_STAGE_CHIRP);
  CK(launch_chirp_table(p->groups[I.group].d_G, p->d_H + (size_t)slot * p->h_stride, p->dm[d],
                        p->groups[I.group].geom, p->stream));
  mark_end(p, CHIRP_STAGE_CHIRP, mk);
  return CHIRP_OK;
}

int dedisperse_one(chirp_plan* p, int d, float2* y) {
  int rc = chirp_for(p, d);
  if (rc) return rc;
  return dedisperse_blocks(p, d, y, 0, p->groups[p->dmi[d].group].geom.n_blk);
}

// Block of DM d's group that owns output sample t (the overlap-save rule).
long long owner_block(const GroupGeom& G, long long t) {
  if (G.n_blk <= 1) return 0;
  long long u = t - G.n_hi_max;
  long long b = u < 0 ? 0 : u / G.step;
  return b > G.n_blk - 1 ? G.n_blk - 1 : b;
}

enum Backend { kCorrelate, kBeams };

// A Chimageator search in a tensor-core mode has the inverse column pass
// write the beamformer's BF16 image of DM d's valid dumps directly.
bool fused_image(const chirp_plan* p, Backend be) { return be == kBeams && tc_beams(p); }
BeamImageOut beam_image_for(const chirp_plan* p, int d);
// A Chimageator search in the reduced-precision visibility form has the
// inverse column pass write the voltages as BF16 pairs (into d_y's memory).
bool bf16_y(const chirp_plan* p, Backend be) {
  return be == kBeams && p->beam_mode == CHIRP_BEAM_VIS_BF16;
}

// Inverse column pass of DM d over sequences [q0, q0 + nq) (or the listed
// blocks) with the output the back-end reads: FP32 voltages, BF16 voltages,
// or the tensor-core beamformer's image.
cudaError_t column_pass(chirp_plan* p, int d, Backend be, const float2* Z, long long q0,
                        long long nq, const int* blist, float2* y = nullptr) {
  const DmInfo& I = p->dmi[d];
  const GroupGeom& G = p->groups[I.group].geom;
  if (!y) y = p->d_y;
  if (bf16_y(p, be))
    return launch_inverse_cols_bf16(Z, y, p->N, p->M, q0, nq, G, I.n_hi, I.n_lo, p->tw(),
                                    p->stream, blist);
  const BeamImageOut img = fused_image(p, be) ? beam_image_for(p, d) : BeamImageOut{};
  return launch_inverse_cols(Z, y, p->N, p->M, q0, nq, G, I.n_hi, I.n_lo, p->tw(), p->stream,
                             blist, fused_image(p, be) ? &img : nullptr);
}

BeamImageOut beam_image_for(const chirp_plan* p, int d) {
  const DmInfo& I = p->dmi[d];
  const int nt = beam_tc_tile_samples(p->beam_shape);
  int log2_nt = 0;
  while ((1 << log2_nt) < nt) log2_nt++;
  BeamImageOut o;
  o.img = p->d_bimg;
  o.t0 = I.first * p->L;
  o.t1 = (I.last + 1) * p->L;
  o.log2_nt = log2_nt;
  o.G = beam_tc_groups(p->M);
  o.GB = beam_tc_bgroups(p->M, p->beam_terms);
  o.terms = p->beam_terms;
  return o;
}

// Back-end of DM d over its valid dumps [m0, m1) (inside [first, last]).
// The tensor-core modes read the image the inverse column pass wrote, whose
// tiles count from the DM's first valid dump.
int backend_dumps(chirp_plan* p, int d, Backend be, long long m0, long long m1, void* dout) {
  if (m1 <= m0) return CHIRP_OK;
  const long long last = m1 - 1;
  // visibilities of dumps [m0, m1) into vis[m][pair] (absolute dump index m).
  // The visibility beam identity sums M^2 pair terms per pixel, which
  // multiplies a visibility's relative error by up to M, so unless a
  // tensor-core correlation was asked for explicitly it uses FP32 products.
  auto correlate = [&](float2* vis, bool for_beams) -> int {
    int mk = mark_begin(p, CHIRP_STAGE_CORRELATE);
    if (for_beams && p->beam_mode == CHIRP_BEAM_VIS_BF16)
      CK(launch_correlate_bf16(p->d_y, p->N, p->M, p->L, m0, m1 - m0, m0, last, vis, p->stream));
    else if (p->corr_mode == CHIRP_CORR_FP32_SIMT || (for_beams && !p->corr_forced))
      CK(launch_correlate(p->d_y, p->N, p->M, p->L, m0, m1 - m0, m0, last, vis, p->stream));
    else
      CK(launch_correlate_tc(p->d_y, p->N, p->M, p->L, m0, last, vis, p->d_err,
                             p->corr_mode == CHIRP_CORR_TC_BF16 ? 1 : 3, p->stream));
    mark_end(p, CHIRP_STAGE_CORRELATE, mk);
    return CHIRP_OK;
  };
  if (be == kCorrelate)
    return correlate((float2*)dout + d * (size_t)p->n_dump * p->n_pair, false);
  float* out = (float*)dout + (size_t)d * p->n_dump * p->n_pix;
  if (vis_beams(p)) {
    int rc = correlate(p->d_V, true);
    if (rc) return rc;
    int mk;
    mk = mark_begin(p, CHIRP_STAGE_BEAMFORM);
    CK(launch_beam_from_vis(p->d_V, p->d_wpair, p->M, p->n_pix, m0, last, out, p->stream));
    mark_end(p, CHIRP_STAGE_BEAMFORM, mk);
  } else if (tc_beams(p)) {
    const long long origin = p->dmi[d].first * p->L;
    int mk = mark_begin(p, CHIRP_STAGE_BEAMFORM);
    CK(launch_beam_tc(p->d_bimg, p->d_aimg, p->M, p->n_pix, p->L, m0, last, origin, out,
                      p->d_err, p->beam_terms, p->beam_shape, p->stream));
    mark_end(p, CHIRP_STAGE_BEAMFORM, mk);
  } else {
    int mk = mark_begin(p, CHIRP_STAGE_BEAMFORM);
    CK(launch_beamform_simt(p->d_y, p->N, p->M, p->L, m0, m1 - m0, m0, last, p->d_W, p->n_pix,
                            out, p->stream));
    mark_end(p, CHIRP_STAGE_BEAMFORM, mk);
  }
  return CHIRP_OK;
}

// A selection of (DM, dump) cells: per DM the device list of its selected
// valid dumps (dlist + off[d], n[d] entries) and its mask row.
struct Selection {
  const unsigned char* mask = nullptr;
  const int* d_lists = nullptr;
  const long long* off = nullptr;
  const long long* n = nullptr;
  const char* dense_group = nullptr;  // groups searched with the multi-DM inverse
};

// The back-end of DM d over its selected dumps only: the visibility paths take
// the dump list, the other beam modes run over runs of consecutive dumps.
int selected_backend(chirp_plan* p, int d, Backend be, void* dout, const Selection& sel) {
  const DmInfo& I = p->dmi[d];
  const int* dlist = sel.d_lists + sel.off[d];
  const long long n_sel = sel.n[d];
  if (be == kCorrelate || vis_beams(p)) {
    float2* vout = be == kCorrelate ? (float2*)dout + (size_t)d * p->n_dump * p->n_pair : p->d_V;
    int mk = mark_begin(p, CHIRP_STAGE_CORRELATE);
    if (bf16_y(p, be))
      CK(launch_correlate_bf16(p->d_y, p->N, p->M, p->L, 0, n_sel, I.first, I.last, vout,
                               p->stream, dlist));
    else
      CK(launch_correlate(p->d_y, p->N, p->M, p->L, 0, n_sel, I.first, I.last, vout, p->stream,
                          dlist));
    mark_end(p, CHIRP_STAGE_CORRELATE, mk);
    if (be == kBeams) {
      mk = mark_begin(p, CHIRP_STAGE_BEAMFORM);
      CK(launch_beam_from_vis(p->d_V, p->d_wpair, p->M, p->n_pix, I.first, I.last,
                              (float*)dout + (size_t)d * p->n_dump * p->n_pix, p->stream, dlist,
                              n_sel));
      mark_end(p, CHIRP_STAGE_BEAMFORM, mk);
    }
    return CHIRP_OK;
  }
  const unsigned char* row = sel.mask + (size_t)d * p->n_dump;
  for (long long m = I.first; m <= I.last;) {
    if (!row[m]) {
      m++;
      continue;
    }
    long long e = m;
    while (e <= I.last && row[e]) e++;
    int rc = backend_dumps(p, d, be, m, e, dout);
    if (rc) return rc;
    m = e;
  }
  return CHIRP_OK;
}

// The back-ends of a chunk batch into one correlator launch (and one launch
// of beams from visibilities) when they run on the staged CUDA-core
// correlator -- the choice backend_dumps makes -- and every DM of the chunk
// has its own voltage slot.
bool batched_backend(const chirp_plan* p, Backend be) {
  if (p->y_slots < p->dm_chunk || p->dm_chunk < 2) return false;
  if (be == kCorrelate) return p->corr_mode == CHIRP_CORR_FP32_SIMT;
  return vis_beams(p) && (p->beam_mode == CHIRP_BEAM_VIS_BF16 ||
                          p->corr_mode == CHIRP_CORR_FP32_SIMT || !p->corr_forced);
}

// Back-ends of the chunk's DMs ds[0 .. n), DM ds[j]'s voltages in slot j:
// over their valid dumps, or over their selected dumps.
int batched_backends(chirp_plan* p, Backend be, void* dout, const int* ds, int n,
                     const Selection* sel) {
  CorrJob cj[kCorrBatchMax];
  VisJob vj[kCorrBatchMax];
  const size_t slot = (size_t)p->M * p->N;
  for (int j = 0; j < n; j++) {
    const int d = ds[j];
    const DmInfo& I = p->dmi[d];
    const int* dl = sel ? sel->d_lists + sel->off[d] : nullptr;
    const long long n_m = sel ? sel->n[d] : I.last - I.first + 1;
    float2* vis = be == kCorrelate ? (float2*)dout + (size_t)d * p->n_dump * p->n_pair
                                   : p->d_V + (size_t)j * p->v_stride;
    cj[j] = CorrJob{p->d_y + (size_t)j * slot, vis, I.first, n_m, I.first, I.last, dl};
    vj[j] = VisJob{vis, (float*)dout + (size_t)d * p->n_dump * p->n_pix, I.first, n_m, dl};
  }
  if (p->beam_pending) {  // the previous chunk's beams still read d_V
    CK(cudaStreamWaitEvent(p->stream, p->beam_ev[1], 0));
    p->beam_pending = false;
  }
  int mk = mark_begin(p, CHIRP_STAGE_CORRELATE);
  CK(launch_correlate_batch(cj, n, bf16_y(p, be), p->N, p->M, p->L, p->stream));
  mark_end(p, CHIRP_STAGE_CORRELATE, mk);
  if (be == kBeams && p->beam_side) {  // launched by side_beams after the next row pass
    p->beam_jobs.assign(vj, vj + n);
  } else if (be == kBeams) {
    mk = mark_begin(p, CHIRP_STAGE_BEAMFORM);
    CK(launch_beam_from_vis_batch(vj, n, p->d_wpair, p->M, p->n_pix, p->stream));
    mark_end(p, CHIRP_STAGE_BEAMFORM, mk);
  }
  return CHIRP_OK;
}

// The beams deferred by batched_backends: on the side stream, one CTA per
// SM, ordered after everything the plan's stream has queued so far.
int side_beams(chirp_plan* p) {
  if (p->beam_jobs.empty()) return CHIRP_OK;
  CK(cudaEventRecord(p->beam_ev[0], p->stream));
  CK(cudaStreamWaitEvent(p->side_stream, p->beam_ev[0], 0));
  CK(launch_beam_from_vis_batch(p->beam_jobs.data(), (int)p->beam_jobs.size(), p->d_wpair, p->M,
                                p->n_pix, p->side_stream, p->n_sm));
  CK(cudaEventRecord(p->beam_ev[1], p->side_stream));
  p->beam_jobs.clear();
  p->beam_pending = true;
  return CHIRP_OK;
}

// The whole search with the row passes of up to dm_chunk DMs of a group in
// one launch: per chunk the chirp tables, one multi-DM row pass, then per
// DM the column pass (voltages or the beam image) and the back-end, or, when
// the back-ends batch, the column passes into the DMs' slots and then one
// batched back-end.  With a selection: only the groups it marks dense, only
// their DMs with a selected dump, and the back-end over the selected dumps.
int full_search_chunked(chirp_plan* p, Backend be, void* dout, const Selection* sel = nullptr) {
  struct Chunk {
    int group;
    std::vector<int> dms;
  };
  std::vector<Chunk> chunks;
  for (size_t gi = 0; gi < p->groups.size(); gi++) {
    if (sel && !sel->dense_group[gi]) continue;
    std::vector<int> dms;
    for (int d : p->groups[gi].dms)
      if (p->dmi[d].last >= p->dmi[d].first && (!sel || sel->n[d] > 0)) dms.push_back(d);
    for (size_t c0 = 0; c0 < dms.size(); c0 += (size_t)p->dm_chunk)
      chunks.push_back({(int)gi, std::vector<int>(dms.begin() + c0,
                                                   dms.begin() + std::min(dms.size(),
                                                                          c0 + (size_t)p->dm_chunk))});
  }
  // The chirp tables of chunk c + 1 are formed on the side stream while
  // chunk c's column passes and back-ends run (FP64 pipe beside FP32 and
  // load/store work), into the table set chunk c - 1 used; in stream order
  // instead while stage timing records the chirp stage (its events are on
  // the plan's stream).
  const bool overlap = chunks.size() > 1 &&
                       !(p->timing && ((p->timing_mask >> CHIRP_STAGE_CHIRP) & 1u));
  if (overlap && !p->side_stream) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaStreamCreateWithFlags(&p->side_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : p->side_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (cudaEvent_t& e : p->beam_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  // device outputs of visibility beams: each chunk's quadratic form on the
  // side stream too, one CTA per SM, launched after the next chunk's row pass
  // so that it runs beside that chunk's column passes (side_beams)
  p->beam_side = overlap && be == kBeams && vis_beams(p) && !sel && !p->drain_host &&
                 !(p->timing && ((p->timing_mask >> CHIRP_STAGE_BEAMFORM) & 1u));
  // (on the side stream one CTA per SM, striding over the bins, so that the
  // column passes beside it keep their CTA slots)
  auto tables = [&](size_t c, cudaStream_t st) -> cudaError_t {
    const Chunk& k = chunks[c];
    double dmv[kMaxChirps];
    for (size_t j = 0; j < k.dms.size(); j++) dmv[j] = p->dm[k.dms[j]];
    Group& grp = p->groups[(size_t)k.group];
    return launch_chirp_tables(grp.d_G, p->d_H + (c & 1) * (size_t)p->dm_chunk * p->h_stride,
                               p->h_stride, dmv, (int)k.dms.size(), grp.geom, st,
                               st == p->side_stream ? p->n_sm : 0);
  };
  for (size_t c = 0; c < chunks.size(); c++) {
    const Chunk& k = chunks[c];
    Group& grp = p->groups[(size_t)k.group];
    int rc0 = ensure_spec(p, k.group);
    if (rc0) return rc0;
    const GroupGeom& G = grp.geom;
    const long long nq = (long long)p->M * G.n_blk;
    const int n = (int)k.dms.size();
    int mk;
    if (!overlap || c == 0) {
      mk = mark_begin(p, CHIRP_STAGE_CHIRP);
      CK(tables(c, p->stream));
      mark_end(p, CHIRP_STAGE_CHIRP, mk);
    } else {
      CK(cudaStreamWaitEvent(p->stream, p->side_ev[1 + (c & 1)], 0));
    }
    mk = mark_begin(p, CHIRP_STAGE_INV_ROWS);
    CK(launch_inverse_rows_multi(grp.d_spec, p->d_Z, (long long)p->z_stride,
                                 p->d_H + (c & 1) * (size_t)p->dm_chunk * p->h_stride,
                                 p->h_stride, n, nq, G, p->tw(), grp.d_rtw, p->stream));
    mark_end(p, CHIRP_STAGE_INV_ROWS, mk);
    {  // the previous chunk's beams, beside this chunk's column passes
      int rc = side_beams(p);
      if (rc) return rc;
    }
    if (overlap && c + 1 < chunks.size()) {
      CK(cudaEventRecord(p->side_ev[0], p->stream));
      CK(cudaStreamWaitEvent(p->side_stream, p->side_ev[0], 0));
      CK(tables(c + 1, p->side_stream));
      CK(cudaEventRecord(p->side_ev[1 + ((c + 1) & 1)], p->side_stream));
    }
    const bool batch = n > 1 && batched_backend(p, be);
    for (int j = 0; j < n; j++) {
      const int d = k.dms[(size_t)j];
      const DmInfo& I = p->dmi[d];
      mk = mark_begin(p, CHIRP_STAGE_INV_COLS);
      CK(column_pass(p, d, be, p->d_Z + (size_t)j * p->z_stride, 0, nq, nullptr,
                     batch ? p->d_y + (size_t)j * p->M * p->N : nullptr));
      mark_end(p, CHIRP_STAGE_INV_COLS, mk);
      if (batch) continue;
      if (p->beam_pending) {  // the previous chunk's side-stream beams still read d_V
        CK(cudaStreamWaitEvent(p->stream, p->beam_ev[1], 0));
        p->beam_pending = false;
      }
      int rc = sel ? selected_backend(p, d, be, dout, *sel)
                   : backend_dumps(p, d, be, I.first, I.last + 1, dout);
      if (!rc) rc = drain_dm(p, d);
      if (rc) return rc;
    }
    if (batch) {
      int rc = batched_backends(p, be, dout, k.dms.data(), n, sel);
      for (int j = 0; j < n && !rc; j++) rc = drain_dm(p, k.dms[(size_t)j]);
      if (rc) return rc;
    }
  }
  {  // the last batched chunk's beams
    int rc = side_beams(p);
    if (rc) return rc;
  }
  p->beam_side = false;
  if (p->beam_pending) {  // join the last chunk's beams
    CK(cudaStreamWaitEvent(p->stream, p->beam_ev[1], 0));
    p->beam_pending = false;
  }
  return CHIRP_OK;
}

// The selected DMs of the groups a selection does not mark dense, per chunk
// of up to dm_chunk DMs of a group: one chirp-table launch, one row pass over
// each DM's listed blocks (blk_off/blk_n into the device lists), the column
// passes over the same blocks, then the back-ends over the selected dumps
// (one batched launch where they batch).  A DM whose listed blocks do not fit
// a workspace slot runs alone, its list in pieces.
int sparse_search(chirp_plan* p, Backend be, void* dout, const Selection& sel,
                  const std::vector<char>& dense, const std::vector<long long>& blk_off,
                  const std::vector<long long>& blk_n) {
  std::vector<int> dms;
  for (size_t gi = 0; gi < p->groups.size(); gi++) {
    if (dense[gi]) continue;
    Group& g = p->groups[gi];
    const GroupGeom& G = g.geom;
    dms.clear();
    for (int d : g.dms)
      if (p->dmi[d].last >= p->dmi[d].first && sel.n[d] > 0) dms.push_back(d);
    if (dms.empty()) continue;
    int rc = ensure_spec(p, (int)gi);
    if (rc) return rc;
    const long long cap = (long long)(p->z_stride / (size_t)G.nfft) / p->M;  // blocks per slot
    for (size_t c0 = 0; c0 < dms.size();) {
      int n = (int)std::min((size_t)std::max(1, p->dm_chunk), dms.size() - c0);
      for (int j = 0; j < n; j++)
        if (blk_n[dms[c0 + j]] > cap) n = j == 0 ? 1 : std::min(n, j);
      const int* bl[kMaxChirps];
      long long nb[kMaxChirps];
      double dmv[kMaxChirps];
      for (int j = 0; j < n; j++) {
        dmv[j] = p->dm[dms[c0 + j]];
        bl[j] = p->d_lists + blk_off[dms[c0 + j]];
        nb[j] = blk_n[dms[c0 + j]];
      }
      int mk = mark_begin(p, CHIRP_STAGE_CHIRP);
      CK(launch_chirp_tables(g.d_G, p->d_H, p->h_stride, dmv, n, G, p->stream));
      mark_end(p, CHIRP_STAGE_CHIRP, mk);
      if (n == 1) {  // a lone DM: its list in pieces of at most a slot's blocks
        const int d = dms[c0];
        const long long piece = std::max(1LL, cap);
        for (long long k0 = 0; k0 < nb[0]; k0 += piece) {
          const int* blp = bl[0] + k0;
          const long long nbp = std::min(piece, nb[0] - k0);
          mk = mark_begin(p, CHIRP_STAGE_INV_ROWS);
          CK(launch_inverse_rows_lists(g.d_spec, p->d_Z, 0, p->d_H, 0, 1, &blp, &nbp, p->M, G,
                                       p->tw(), g.d_rtw, p->stream));
          mark_end(p, CHIRP_STAGE_INV_ROWS, mk);
          mk = mark_begin(p, CHIRP_STAGE_INV_COLS);
          CK(column_pass(p, d, be, p->d_Z, 0, nbp * p->M, blp));
          mark_end(p, CHIRP_STAGE_INV_COLS, mk);
        }
        rc = selected_backend(p, d, be, dout, sel);
      } else {
        mk = mark_begin(p, CHIRP_STAGE_INV_ROWS);
        CK(launch_inverse_rows_lists(g.d_spec, p->d_Z, (long long)p->z_stride, p->d_H,
                                     p->h_stride, n, bl, nb, p->M, G, p->tw(), g.d_rtw,
                                     p->stream));
        mark_end(p, CHIRP_STAGE_INV_ROWS, mk);
        // batched: every DM's voltages into its slot, then one back-end launch;
        // otherwise each DM's column pass right before its own back-end
        const bool batch = batched_backend(p, be);
        for (int j = 0; j < n && !rc; j++) {
          mk = mark_begin(p, CHIRP_STAGE_INV_COLS);
          CK(column_pass(p, dms[c0 + j], be, p->d_Z + (size_t)j * p->z_stride, 0, nb[j] * p->M,
                         bl[j], batch ? p->d_y + (size_t)j * p->M * p->N : nullptr));
          mark_end(p, CHIRP_STAGE_INV_COLS, mk);
          if (!batch) rc = selected_backend(p, dms[c0 + j], be, dout, sel);
        }
        if (batch && !rc) rc = batched_backends(p, be, dout, dms.data() + c0, n, &sel);
      }
      if (rc) return rc;
      c0 += (size_t)n;
    }
  }
  return CHIRP_OK;
}

// The whole search, or (mask != NULL) only the (DM, dump) cells whose mask
// byte is nonzero; outputs are zero elsewhere.  A selective search lists, per
// DM, its selected valid dumps and the blocks that own them.  An FFT-length
// group whose DMs need at least kDenseBlocks of their (DM, block) pairs runs
// the full multi-DM inverse and restricts only the back-end to the listed
// dumps; the other groups inverse-transform, per DM, just the listed blocks
// (up to dm_chunk DMs per launch, sparse_search).  Per block the per-DM form costs ~1.2x
// in the row pass and ~2x in the chirp tables (the multi-DM forms read each
// spectrum and phase table once for up to 4 DMs), so it wins below ~85 %.
constexpr double kDenseBlocks = 0.85;

int enqueue_search(chirp_plan* p, const void* dx, const unsigned char* mask, Backend be,
                   void* dout, size_t bytes) {
  p->beam_side = false;
  p->beam_jobs.clear();
  int rc = forward_all(p, dx);
  if (rc) return rc;
  CK(cudaMemsetAsync(dout, 0, bytes, p->stream));  // invalid / unselected cells stay zero
  if (!mask && p->dm_chunk > 1) return full_search_chunked(p, be, dout);
  std::vector<int> lists;
  std::vector<long long> blk_off(p->dm.size(), 0), blk_n(p->dm.size(), 0);
  std::vector<long long> dmp_off(p->dm.size(), 0), dmp_n(p->dm.size(), 0);
  std::vector<char> dense(p->groups.size(), 0);
  if (mask) {
    std::vector<unsigned char> need;
    std::vector<long long> g_need(p->groups.size(), 0), g_all(p->groups.size(), 0);
    for (int d = 0; d < (int)p->dm.size(); d++) {
      const DmInfo& I = p->dmi[d];
      const GroupGeom& G = p->groups[I.group].geom;
      const unsigned char* row = mask + (size_t)d * p->n_dump;
      need.assign((size_t)G.n_blk, 0);
      dmp_off[d] = (long long)lists.size();
      for (long long m = I.first; m <= I.last; m++)
        if (row[m]) {
          lists.push_back((int)m);
          for (long long b = owner_block(G, m * p->L); b <= owner_block(G, (m + 1) * p->L - 1); b++)
            need[(size_t)b] = 1;
        }
      dmp_n[d] = (long long)lists.size() - dmp_off[d];
      blk_off[d] = (long long)lists.size();
      for (long long b = 0; b < G.n_blk; b++)
        if (need[(size_t)b]) lists.push_back((int)b);
      blk_n[d] = (long long)lists.size() - blk_off[d];
      if (dmp_n[d] > 0) {
        g_need[I.group] += blk_n[d];
        g_all[I.group] += G.n_blk;
      }
    }
    if (p->dm_chunk > 1)
      for (size_t gi = 0; gi < p->groups.size(); gi++)
        dense[gi] = g_all[gi] > 0 && (double)g_need[gi] >= kDenseBlocks * (double)g_all[gi];
    if (!lists.empty()) {
      if (p->lists_cap < lists.size()) {
        cudaFree(p->d_lists);
        p->d_lists = nullptr;
        p->lists_cap = 0;
        rc = dev_alloc(p, (void**)&p->d_lists, lists.size() * sizeof(int), "index lists");
        if (rc) return rc;
        p->lists_cap = lists.size();
      }
      CK(cudaMemcpyAsync(p->d_lists, lists.data(), lists.size() * sizeof(int),
                         cudaMemcpyHostToDevice, p->stream));
    }
    Selection sel;
    sel.mask = mask;
    sel.d_lists = p->d_lists;
    sel.off = dmp_off.data();
    sel.n = dmp_n.data();
    sel.dense_group = dense.data();
    rc = full_search_chunked(p, be, dout, &sel);
    if (rc) return rc;
    return sparse_search(p, be, dout, sel, dense, blk_off, blk_n);
  }
  for (int d = 0; d < (int)p->dm.size(); d++) {
    const DmInfo& I = p->dmi[d];
    if (I.last < I.first) continue;
    const GroupGeom& G = p->groups[I.group].geom;
    rc = ensure_spec(p, I.group);
    if (!rc) rc = chirp_for(p, d);
    if (rc) return rc;
    const BeamImageOut img = fused_image(p, be) ? beam_image_for(p, d) : BeamImageOut{};
    rc = dedisperse_blocks(p, d, p->d_y, 0, G.n_blk, fused_image(p, be) ? &img : nullptr,
                           bf16_y(p, be));
    if (!rc) rc = backend_dumps(p, d, be, I.first, I.last + 1, dout);
    if (!rc) rc = drain_dm(p, d);
    if (rc) return rc;
  }
  return CHIRP_OK;
}

// ---- true-delay (wideband) beams
// x mod 1 as cycles x 2^64 (exact: f * 2^32 splits without rounding).
unsigned long long frac_u64(double x) {
  const double f = x - std::floor(x);
  const double hi = std::floor(f * 4294967296.0);
  const double lo = std::floor((f * 4294967296.0 - hi) * 4294967296.0);
  return ((unsigned long long)hi << 32) + (unsigned long long)lo;
}

constexpr size_t kTdChunkBytes = 1ull << 30;  // per chunk buffer (beam spectra, intermediate)

// The beam spectra of a group do not depend on the DM: they are formed once
// per group and chunk of pixels, for every block, and every DM of the group
// is searched over them.  Pixels per chunk so that the chunk's spectra stay
// within kTdBeamBytes (at least one pixel).
constexpr size_t kTdBeamBytes = 8ull << 30;
int td_pixel_chunk(const chirp_plan* p, const GroupGeom& G) {
  const long long per_pix = G.n_blk * G.nfft * (long long)sizeof(float2);
  return (int)std::max(1LL, std::min((long long)p->n_pix, (long long)kTdBeamBytes / per_pix));
}

// First use: per group the phase pairs {frac(f0 tau), frac(B tau / Nfft)} of
// every (pixel, antenna) in FP64, the beam-spectra buffer and the chunk buffer
// of the inverse.
int truedelay_setup(chirp_plan* p) {
  if (p->d_tdY) return CHIRP_OK;
  long long max_nfft = 0, max_seq = 0;
  for (auto& g : p->groups) {
    max_nfft = std::max(max_nfft, g.geom.nfft);
    max_seq = std::max(max_seq, g.geom.n_blk * (long long)p->n_pix);
  }
  p->td_cap = std::max(1LL, std::min({(long long)(kTdChunkBytes / (max_nfft * sizeof(float2))),
                                      max_seq, 65535LL}));
  std::vector<unsigned long long> ph(2 * (size_t)p->n_pix * p->M);
  std::vector<float2> rot((size_t)p->n_pix * p->M);
  for (auto& g : p->groups) {
    for (int q = 0; q < p->n_pix; q++) {
      const double l = p->pix[2 * q], m = p->pix[2 * q + 1];
      const double n = std::sqrt(std::max(0.0, 1.0 - l * l - m * m));
      for (int a = 0; a < p->M; a++) {
        const double tau = (p->xyz[3 * a] * l + p->xyz[3 * a + 1] * m + p->xyz[3 * a + 2] * (n - 1.0)) /
                           kCLight;
        const size_t i = 2 * ((size_t)q * p->M + a);
        ph[i] = frac_u64(p->f0 * tau);
        ph[i + 1] = frac_u64(p->bw * tau / (double)g.geom.nfft);
        // step along a row of the transposed spectrum: n1 bins
        double c = (double)g.geom.n1 * p->bw * tau / (double)g.geom.nfft;
        c -= std::rint(c);
        rot[(size_t)q * p->M + a] = make_float2((float)std::cos(2.0 * kPi * c),
                                                (float)std::sin(2.0 * kPi * c));
      }
    }
    int rc = dev_alloc(p, &g.d_tdph, ph.size() * sizeof(unsigned long long), "true-delay phases");
    if (!rc) rc = dev_alloc(p, (void**)&g.d_tdrot, rot.size() * sizeof(float2), "true-delay steps");
    if (rc) return rc;
    CK(cudaMemcpyAsync(g.d_tdph, ph.data(), ph.size() * sizeof(unsigned long long),
                       cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(g.d_tdrot, rot.data(), rot.size() * sizeof(float2), cudaMemcpyHostToDevice,
                       p->stream));
    CK(cudaStreamSynchronize(p->stream));  // ph is reused for the next group
  }
  size_t ybytes = 0;
  for (auto& g : p->groups)
    ybytes = std::max(ybytes, (size_t)g.geom.n_blk * (size_t)td_pixel_chunk(p, g.geom) *
                                  (size_t)g.geom.nfft * sizeof(float2));
  int rc = dev_alloc(p, (void**)&p->d_tdY, ybytes, "true-delay beam spectra");
  if (!rc)  // one chunk buffer per DM of a multi-DM row pass
    rc = dev_alloc(p, (void**)&p->d_tdZ,
                   (size_t)p->dm_chunk * p->td_cap * (size_t)max_nfft * sizeof(float2),
                   "true-delay intermediate");
  return rc;
}

// Per group and chunk of pixels: the beam spectra of every block once; then
// per chunk of up to dm_chunk DMs of the group their chirps, and per chunk of
// (block, pixel) sequences (whole blocks of the chunk's pixels when they fit
// the inverse's buffer, else pixel ranges of one block) one multi-DM inverse
// row pass with the chirps and, per DM, the column pass that detects and
// integrates into dout (cleared first).
int truedelay_search(chirp_plan* p, const void* dx, float* dout, size_t bytes) {
  int rc = truedelay_setup(p);
  if (rc) return rc;
  rc = forward_all(p, dx);
  if (rc) return rc;
  CK(cudaMemsetAsync(dout, 0, bytes, p->stream));
  for (size_t gi = 0; gi < p->groups.size(); gi++) {
    Group& g = p->groups[gi];
    const GroupGeom& G = g.geom;
    std::vector<int> dms;
    for (int d : g.dms)
      if (p->dmi[d].last >= p->dmi[d].first) dms.push_back(d);
    if (dms.empty()) continue;
    rc = ensure_spec(p, (int)gi);
    if (rc) return rc;
    const int np_max = td_pixel_chunk(p, G);
    for (int p0 = 0; p0 < p->n_pix; p0 += np_max) {
      const int np = std::min(np_max, p->n_pix - p0);
      int mk = mark_begin(p, CHIRP_STAGE_TD_SPECTRA);
      CK(launch_td_spectra(g.d_spec, p->d_tdY, 0, (int)G.n_blk, np, p0, p->M, G, g.d_tdph,
                           g.d_tdrot, p->stream));
      mark_end(p, CHIRP_STAGE_TD_SPECTRA, mk);
      // up to dm_chunk DMs per row pass (the beam spectra read once for all of
      // them), then each DM's column pass
      const size_t z_stride = (size_t)p->td_cap * (size_t)G.nfft;
      for (size_t c0 = 0; c0 < dms.size(); c0 += (size_t)p->dm_chunk) {
        const int n = (int)std::min((size_t)p->dm_chunk, dms.size() - c0);
        double dmv[kMaxChirps];
        for (int j = 0; j < n; j++) dmv[j] = p->dm[dms[c0 + j]];
        mk = mark_begin(p, CHIRP_STAGE_CHIRP);
        CK(launch_chirp_tables(g.d_G, p->d_H, p->h_stride, dmv, n, G, p->stream));
        mark_end(p, CHIRP_STAGE_CHIRP, mk);
        // (b0, nb blocks) x (pp, npp pixels of the chunk) per inverse launch
        const long long nb_max = np <= p->td_cap ? std::max(1LL, p->td_cap / np) : 1;
        const int npp_max = (int)std::min<long long>(np, p->td_cap);
        for (long long b0 = 0; b0 < G.n_blk; b0 += nb_max) {
          const int nb = (int)std::min(nb_max, G.n_blk - b0);
          for (int pp = 0; pp < np; pp += npp_max) {
            const int npp = std::min(npp_max, np - pp);
            mk = mark_begin(p, CHIRP_STAGE_INV_ROWS);
            CK(launch_inverse_rows_multi(p->d_tdY + (size_t)(b0 * np + pp) * G.nfft, p->d_tdZ,
                                         (long long)z_stride, p->d_H, p->h_stride, n,
                                         (long long)nb * npp, G, p->tw(), g.d_rtw, p->stream));
            mark_end(p, CHIRP_STAGE_INV_ROWS, mk);
            for (int j = 0; j < n; j++) {
              const DmInfo& I = p->dmi[dms[c0 + j]];
              float* out = dout + (size_t)dms[c0 + j] * p->n_dump * p->n_pix;
              mk = mark_begin(p, CHIRP_STAGE_INV_COLS);
              CK(launch_inverse_cols_pow(p->d_tdZ + (size_t)j * z_stride, out, p->N, b0, nb, npp,
                                         p0 + pp, p->n_pix, G, I.n_hi, I.n_lo, p->L,
                                         I.first * p->L, (I.last + 1) * p->L, p->tw(),
                                         p->stream));
              mark_end(p, CHIRP_STAGE_INV_COLS, mk);
            }
          }
        }
      }
    }
  }
  return CHIRP_OK;
}

// Full searches on device buffers replay a CUDA graph: the first call with a
// given (input, output, back-end) runs eagerly (lazy allocations and kernel
// attributes happen there), the second captures and instantiates the launch
// sequence, later calls launch the graph.
int graph_search(chirp_plan* p, const void* dx, Backend be, void* dout, size_t bytes) {
  for (auto& g : p->graphs) {
    if (g.in != dx || g.out != dout || g.be != (int)be) continue;
    if (g.exec) {
      CK(cudaGraphLaunch(g.exec, p->stream));
      return CHIRP_OK;
    }
    const bool timing = p->timing;
    p->timing = false;  // no event marks inside a capture
    CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_search(p, dx, nullptr, be, dout, bytes);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->stream, &graph);
    p->timing = timing;
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return fail(CHIRP_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      return fail(CHIRP_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    CK(cudaGraphLaunch(g.exec, p->stream));
    return CHIRP_OK;
  }
  if (p->graphs.size() >= 8) {
    if (p->graphs.front().exec) cudaGraphExecDestroy(p->graphs.front().exec);
    p->graphs.erase(p->graphs.begin());
  }
  p->graphs.push_back({dx, dout, (int)be, nullptr});
  return enqueue_search(p, dx, nullptr, be, dout, bytes);
}

int run_search(chirp_plan* p, const void* volt, int volt_loc, const unsigned char* mask,
               Backend be, void* out_user, int out_loc) {
  g_err[0] = 0;
  if (!p) return fail(CHIRP_EINVAL, "plan is NULL");
  if (be == kBeams && p->n_pix <= 0) return fail(CHIRP_EUNSUPPORTED, "plan was created without pixels");
  p->drain_host = nullptr;
  if (be == kCorrelate || !tc_beams(p)) {
    int rc = ensure_y(p);
    if (rc) return rc;
  }
  const size_t per_dm = be == kCorrelate ? (size_t)p->n_dump * p->n_pair : (size_t)p->n_dump * p->n_pix;
  const size_t bytes = per_dm * p->dm.size() * (be == kCorrelate ? sizeof(float2) : sizeof(float));
  void* dout;
  int rc = out_buffer(p, out_user, out_loc, bytes, &dout);
  if (rc) return rc;
  const void* dx;
  rc = stage_input(p, volt, volt_loc, &dx, true);
  if (rc) return rc;
  if (out_loc == CHIRP_HOST && !mask) {
    rc = drain_begin(p, out_user, dout, bytes);
    if (rc) return rc;
  }
  if (p->use_graphs && !mask && volt_loc == CHIRP_DEVICE && out_loc == CHIRP_DEVICE)
    rc = graph_search(p, dx, be, dout, bytes);
  else
    rc = enqueue_search(p, dx, mask, be, dout, bytes);
  if (!rc) rc = input_wait_all(p);
  if (rc) return rc;
  rc = finish_out(p, out_user, out_loc, dout, bytes);
  if (rc) return rc;
  if (be == kBeams && out_loc == CHIRP_HOST) return chirp_plan_status(p);
  return CHIRP_OK;
}

}  // namespace

extern "C" {

int chirp_dedisperse_run(chirp_plan* p, const void* volt, int volt_loc, int d, void* y_out,
                         int y_loc) {
  g_err[0] = 0;
  if (!p) return fail(CHIRP_EINVAL, "plan is NULL");
  if (d < 0 || d >= (int)p->dm.size()) return fail(CHIRP_EINVAL, "DM index out of range");
  const void* dx;
  int rc = stage_input(p, volt, volt_loc, &dx);
  if (rc) return rc;
  size_t bytes = (size_t)p->M * p->N * sizeof(float2);
  void* dy;
  rc = out_buffer(p, y_out, y_loc, bytes, &dy);
  if (rc) return rc;
  const DmInfo& I = p->dmi[d];
  Group& g = p->groups[I.group];
  CK(launch_forward(dx, p->N, p->M, g.geom, g.d_spec, p->tw(), p->stream, p->in_type,
                    p->d_scale));
  p->spec_group = p->lean ? I.group : -1;  // the shared buffer now holds this group
  p->spec_src = dx;
  CK(cudaMemsetAsync(dy, 0, bytes, p->stream));
  rc = dedisperse_one(p, d, (float2*)dy);
  if (rc) return rc;
  return finish_out(p, y_out, y_loc, dy, bytes);
}

int chirpolator_run(chirp_plan* p, const void* volt, int volt_loc, void* vis_out, int vis_loc) {
  return run_search(p, volt, volt_loc, nullptr, kCorrelate, vis_out, vis_loc);
}

int chimageator_run(chirp_plan* p, const void* volt, int volt_loc, float* pow_out, int pow_loc) {
  return run_search(p, volt, volt_loc, nullptr, kBeams, pow_out, pow_loc);
}

int chirp_truedelay_run(chirp_plan* p, const void* volt, int volt_loc, float* pow_out,
                        int pow_loc) {
  g_err[0] = 0;
  if (!p) return fail(CHIRP_EINVAL, "plan is NULL");
  if (p->n_pix <= 0) return fail(CHIRP_EUNSUPPORTED, "plan was created without pixels");
  if (p->xyz.empty()) return fail(CHIRP_EINVAL, "plan was created without antenna positions");
  const void* dx;
  int rc = stage_input(p, volt, volt_loc, &dx);
  if (rc) return rc;
  const size_t bytes = (size_t)p->n_dump * p->n_pix * p->dm.size() * sizeof(float);
  void* dout;
  rc = out_buffer(p, pow_out, pow_loc, bytes, &dout);
  if (rc) return rc;
  rc = truedelay_search(p, dx, (float*)dout, bytes);
  if (rc) return rc;
  return finish_out(p, pow_out, pow_loc, dout, bytes);
}

int chirpolator_run_selective(chirp_plan* p, const void* volt, int volt_loc,
                              const unsigned char* cell_mask, void* vis_out, int vis_loc) {
  if (!cell_mask) return fail(CHIRP_EINVAL, "cell_mask is NULL");
  return run_search(p, volt, volt_loc, cell_mask, kCorrelate, vis_out, vis_loc);
}

int chimageator_run_selective(chirp_plan* p, const void* volt, int volt_loc,
                              const unsigned char* cell_mask, float* pow_out, int pow_loc) {
  if (!cell_mask) return fail(CHIRP_EINVAL, "cell_mask is NULL");
  return run_search(p, volt, volt_loc, cell_mask, kBeams, pow_out, pow_loc);
}

int chirp_incoherent_run(chirp_plan* p, const void* volt, int volt_loc, float* S_out,
                         float* D_out, int out_loc) {
  g_err[0] = 0;
  if (!p) return fail(CHIRP_EINVAL, "plan is NULL");
  if (p->fb_chan <= 0) return fail(CHIRP_EUNSUPPORTED, "plan was created without a filterbank");
  if (!D_out) return fail(CHIRP_EINVAL, "D_out is NULL");
  if (out_loc != CHIRP_HOST && out_loc != CHIRP_DEVICE)
    return fail(CHIRP_EINVAL, "bad buffer location");
  const void* dx;
  int rc = stage_input(p, volt, volt_loc, &dx);
  if (!rc) rc = ensure_y(p);  // the filterbank's scratch
  if (rc) return rc;
  const size_t vbytes = (size_t)p->M * p->N * sizeof(float2);
  const size_t sbytes = (size_t)p->fb_chan * p->T_fb * sizeof(float);
  const size_t dbytes = (size_t)p->fb_n_dm * p->T_fb * sizeof(float);
  float* dD = D_out;
  if (out_loc == CHIRP_HOST) {
    if (!p->d_fb_D) {
      rc = dev_alloc(p, (void**)&p->d_fb_D, std::max<size_t>(dbytes, 16), "incoherent output");
      if (rc) return rc;
    }
    dD = p->d_fb_D;
  }
  float* dS = (out_loc == CHIRP_DEVICE && S_out) ? S_out : p->d_fb_S;
  int mk = mark_begin(p, CHIRP_STAGE_INCOHERENT);
  // the filterbank transforms a copy of the voltages in the dedispersion scratch
  if (p->in_type == CHIRP_IN_CI8)
    CK(launch_unpack_ci8(dx, p->d_scale, p->M, p->N, p->d_y, p->stream));
  else
    CK(cudaMemcpyAsync(p->d_y, dx, vbytes, cudaMemcpyDeviceToDevice, p->stream));
  CK(launch_incoherent(p->d_y, p->N, p->M, p->fb_chan, p->fb_int, p->T_fb, p->d_fb_shift,
                       p->fb_n_dm, dS, dD, p->tw(), p->stream));
  mark_end(p, CHIRP_STAGE_INCOHERENT, mk);
  if (out_loc == CHIRP_HOST) {
    CK(cudaMemcpyAsync(D_out, dD, dbytes, cudaMemcpyDeviceToHost, p->stream));
    if (S_out) CK(cudaMemcpyAsync(S_out, dS, sbytes, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
  }
  return CHIRP_OK;
}

int chirp_plan_fft_split(const chirp_plan* p, long long* nfft, int* n_col, int* n_row) {
  g_err[0] = 0;
  if (!p || !nfft || !n_col || !n_row) return fail(CHIRP_EINVAL, "NULL argument");
  for (size_t g = 0; g < p->groups.size(); g++) {
    nfft[g] = p->groups[g].geom.nfft;
    n_col[g] = p->groups[g].geom.n1;
    n_row[g] = p->groups[g].geom.n2;
  }
  return CHIRP_OK;
}

int chirp_batch_run(chirp_plan* const* plans, const void* const* volts, const int* volt_locs,
                    void* const* outs, const int* out_locs, const int* backends, int n) {
  g_err[0] = 0;
  if (n < 0 || (n > 0 && (!plans || !volts || !volt_locs || !outs || !out_locs || !backends)))
    return fail(CHIRP_EINVAL, "bad batch arguments");
  for (int i = 0; i < n; i++) {
    if (backends[i] != 0 && backends[i] != 1) return fail(CHIRP_EINVAL, "backend %d must be 0 or 1", i);
    int rc = run_search(plans[i], volts[i], volt_locs[i], nullptr,
                        backends[i] == 0 ? kCorrelate : kBeams, outs[i], out_locs[i]);
    if (rc) return rc;
  }
  return CHIRP_OK;
}

int chirp_detect(chirp_plan* p, const float* pow, int pow_loc, float snr_min,
                 chirp_candidate* cand, long long max_cand, int cand_loc, long long* n_cand,
                 float* stats_out) {
  g_err[0] = 0;
  if (!p || !pow || !n_cand || max_cand < 0 || (max_cand > 0 && !cand))
    return fail(CHIRP_EINVAL, "NULL argument or negative max_cand");
  if (p->n_pix <= 0) return fail(CHIRP_EUNSUPPORTED, "plan was created without pixels");
  if (std::isnan(snr_min)) return fail(CHIRP_EINVAL, "snr_min is NaN");
  if ((pow_loc != CHIRP_HOST && pow_loc != CHIRP_DEVICE) ||
      (cand_loc != CHIRP_HOST && cand_loc != CHIRP_DEVICE))
    return fail(CHIRP_EINVAL, "bad buffer location");
  const int n_dm = (int)p->dm.size();
  const size_t pbytes = (size_t)n_dm * p->n_dump * p->n_pix * sizeof(float);
  const long long nc = detect_chunks(n_dm, p->n_dump, p->n_pix);
  int rc = CHIRP_OK;
  if (!p->d_det_stats) {
    rc = dev_alloc(p, (void**)&p->d_det_stats, (size_t)n_dm * p->n_pix * sizeof(float2),
                   "detection statistics");
    if (!rc) rc = dev_alloc(p, (void**)&p->d_det_counts, (size_t)std::max(1LL, nc) * sizeof(int),
                            "detection counts");
    if (!rc) rc = dev_alloc(p, (void**)&p->d_det_offsets,
                            (size_t)(std::max(1LL, nc) + 1) * sizeof(long long), "detection offsets");
    if (rc) return rc;
  }
  const float* dP = pow;
  if (pow_loc == CHIRP_HOST) {
    if (!p->d_det_P) {
      rc = dev_alloc(p, (void**)&p->d_det_P, pbytes, "power staging");
      if (rc) return rc;
    }
    CK(cudaMemcpyAsync(p->d_det_P, pow, pbytes, cudaMemcpyHostToDevice, p->stream));
    dP = p->d_det_P;
  }
  chirp_candidate* dc = cand;
  if (cand_loc == CHIRP_HOST && max_cand > 0) {
    if (p->det_cand_cap < max_cand) {
      cudaFree(p->d_det_cand);
      p->d_det_cand = nullptr;
      p->det_cand_cap = 0;
      rc = dev_alloc(p, (void**)&p->d_det_cand, (size_t)max_cand * sizeof(chirp_candidate),
                     "candidate staging");
      if (rc) return rc;
      p->det_cand_cap = max_cand;
    }
    dc = p->d_det_cand;
  }
  const long long* dfirst = p->d_first_last;
  const long long* dlast = p->d_first_last + n_dm;
  long long* d_total = p->d_det_offsets + std::max(1LL, nc);
  int mk = mark_begin(p, CHIRP_STAGE_DETECT);
  CK(launch_detect(dP, n_dm, p->n_dump, p->n_pix, dfirst, dlast, snr_min, p->d_det_stats,
                   p->d_det_counts, p->d_det_offsets, d_total, dc, max_cand, p->stream));
  mark_end(p, CHIRP_STAGE_DETECT, mk);
  long long total = 0;
  CK(cudaMemcpyAsync(&total, d_total, sizeof(long long), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  const long long n_copy = std::min(total, max_cand);
  const cudaMemcpyKind sk = cand_loc == CHIRP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (cand_loc == CHIRP_HOST && n_copy > 0)
    CK(cudaMemcpyAsync(cand, dc, (size_t)n_copy * sizeof(chirp_candidate), cudaMemcpyDeviceToHost,
                       p->stream));
  if (stats_out)
    CK(cudaMemcpyAsync(stats_out, p->d_det_stats, (size_t)n_dm * p->n_pix * sizeof(float2), sk,
                       p->stream));
  CK(cudaStreamSynchronize(p->stream));
  *n_cand = total;
  return CHIRP_OK;
}

int chirp_plan_status(chirp_plan* p) {
  if (!p) return fail(CHIRP_EINVAL, "plan is NULL");
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  if (flag) return fail(CHIRP_ETIMEOUT, "a device wait timed out; outputs of the affected runs are invalid");
  return CHIRP_OK;
}

}  // extern "C"
