// internal.h -- host-side declarations shared by the library's translation
// units (plan orchestration <-> kernel launchers).  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/chirp_gb300.h"

// Records msg as the calling thread's chirp_last_error() and returns code.
int chirp_report_error(int code, const char* msg);
// Clears the calling thread's chirp_last_error() text (entry of every ABI call).
void chirp_clear_error();

namespace chirp {

// Physical constants shared by every plan type.
constexpr double kDefaultKdm = 4.148808e15;  // dispersion constant k, s Hz^2 / (pc cm^-3), Eq. 1
constexpr double kCLight = 299792458.0;      // m/s, the delays of Eq. tau3D
constexpr double kPi = 3.14159265358979323846264338327950288;

// One FFT-length group: DMs that share Nfft and therefore one block grid.
struct GroupGeom {
  long long nfft;   // transform length
  int log2n;
  int n1, n2;       // nfft = n1 * n2; column pass of length n1, row pass of length n2
  long long step;   // block step S
  long long n_blk;  // blocks per antenna
  long long n_hi_max, n_lo_max;
};

struct TwiddlePtrs {
  const float2* coarse;  // exp(-2 pi j m / 4096), m < 4096
  const float2* fine;    // exp(-2 pi j m / 2^24), m < 4096
  const float4* stage;   // radix-16 stage pairs (w, w^4), spans 16 and 256
};
// One buffer of kTwiddleElems float2 holds coarse | fine | stage.
constexpr int kTwiddleElems = 8192 + 2 * (16 + 256);
inline TwiddlePtrs twiddle_ptrs(const float2* buf) {
  return TwiddlePtrs{buf, buf + 4096, reinterpret_cast<const float4*>(buf + 8192)};
}
// Fills such a buffer (FP64, rounded once).
cudaError_t launch_build_twiddles(float2* buf, cudaStream_t st);
// Row-pass twiddles of one group: rtw[k1 * (n2/16) + j] = exp(-2 pi j' (k1 j mod
// nfft) / nfft) for k1 < n1, j < n2/16 (FP64, rounded once); nfft/16 entries.
cudaError_t launch_build_row_twiddles(float2* rtw, const GroupGeom& g, cudaStream_t st);

// ---- dedispersion kernels (dedisperse.cu) ----
// spectra of every (antenna, block) of one group; spec [n_blk][n_ant][nfft]
// holds X[k1 + n1 k2] at position k1 * n2 + k2.
// x: complex64 [n_ant][n_samp] (in_type 0) or complex int8 pairs times
// scale[a] (in_type 1, scale NULL = 1)
// Blocks [b0, b1) only (b1 < 0: through the last block): the sequences
// [b0 n_ant, b1 n_ant), which read samples [b0 step, (b1 - 1) step + nfft).
cudaError_t launch_forward(const void* x, long long n_samp, int n_ant, const GroupGeom& g,
                           float2* spec, TwiddlePtrs tw, cudaStream_t st, int in_type = 0,
                           const float* scale = nullptr, long long b0 = 0, long long b1 = -1);
// G[pos] = k_dm f^2/(f0^2 (f0 + f)) in the spectrum's (transposed) order, FP64
cudaError_t launch_build_phase_table(double* G, const GroupGeom& g, double f0, double bw,
                                     double k_dm, cudaStream_t st);
// H[pos] = exp(-2 pi j frac(dm G[pos])) / nfft, FP64 phase, FP32 complex result
// (the inverse FFT's normalisation, exact: nfft is a power of two)
// The same for n_dm <= kMaxChirps DMs at once: DM i's table at H + i h_stride.
constexpr int kMaxChirps = 4;
// max_ctas > 0 caps the grid (the kernel strides over the bins), e.g. to run
// it beside other kernels without taking their CTA slots.
cudaError_t launch_chirp_tables(const double* G, float2* H, long long h_stride, const double* dms,
                                int n_dm, const GroupGeom& g, cudaStream_t st, int max_ctas = 0);
cudaError_t launch_chirp_table(const double* G, float2* H, double dm, const GroupGeom& g,
                               cudaStream_t st);
// The inverse can run over chunks of (antenna, block) sequences [q0, q0 + nq)
// (measured: separate launches per L2-sized chunk lose more to kernel ramp-up
// than they save, so the default chunk is the whole group):
// Z holds one chunk (nq x nfft) so that the row pass's output is still in L2
// when the column pass reads it.
#ifndef CHIRP_INVERSE_CHUNK_BYTES
#define CHIRP_INVERSE_CHUNK_BYTES (1LL << 40)
#endif
constexpr long long kInverseChunkBytes = CHIRP_INVERSE_CHUNK_BYTES;
long long inverse_chunk_sequences(const GroupGeom& g, long long n_seq);
// Z[0 .. nq) = rows of IFFT of sequences q0.. after the chirp multiply and twiddle
// With blk_list (device int array), the launch covers nq = n_listed * n_ant
// sequences: listed block b, antenna a -> sequence b * n_ant + a.
// rtw: the group's row-pass twiddles (launch_build_row_twiddles).
cudaError_t launch_inverse_rows(const float2* spec, float2* Z, const float2* H, long long q0,
                                long long nq, const GroupGeom& g, TwiddlePtrs tw,
                                const float2* rtw, cudaStream_t st,
                                const int* blk_list = nullptr, int n_ant = 1);
// The row pass of n_dm <= kMaxChirps DMs, each over its own listed blocks, in
// one launch (grid dimension z = DM): DM d multiplies by H + d h_stride, takes
// the n_list[d] blocks of blk_lists[d] (device) and writes Z + d z_stride.
cudaError_t launch_inverse_rows_lists(const float2* spec, float2* Z, long long z_stride,
                                      const float2* H, long long h_stride, int n_dm,
                                      const int* const* blk_lists, const long long* n_list,
                                      int n_ant, const GroupGeom& g, TwiddlePtrs tw,
                                      const float2* rtw, cudaStream_t st);
// The row pass of all (antenna, block) sequences of a group for n_dm DMs at
// once: DM d multiplies by H + d h_stride and writes Z + d z_stride.
cudaError_t launch_inverse_rows_multi(const float2* spec, float2* Z, long long z_stride,
                                      const float2* H, long long h_stride, int n_dm,
                                      long long nq, const GroupGeom& g, TwiddlePtrs tw,
                                      const float2* rtw, cudaStream_t st);
// The tensor-core beamformer's B image, written directly by the inverse
// column pass (instead of y) when a Chimageator search runs in a tensor-core
// mode: sample t in [t0, t1) of antenna a goes to tile (t - t0) >> log2_nt,
// as BF16 head (and, for three terms, tail) in the layout of beamform_tc.cu.
struct BeamImageOut {
  uint8_t* img;
  long long t0, t1;
  int log2_nt;
  int G, GB, terms;
};
// y[a][t] = dedispersed voltage for every owned, valid t of sequences q0.. (other t untouched)
cudaError_t launch_inverse_cols(const float2* Z, float2* y, long long n_samp, int n_ant,
                                long long q0, long long nq, const GroupGeom& g, long long n_hi,
                                long long n_lo, TwiddlePtrs tw, cudaStream_t st,
                                const int* blk_list = nullptr, const BeamImageOut* img = nullptr);

// The same column pass writing the owned, valid samples as BF16 (re, im)
// pairs: y16 is [n_ant][n_samp] __nv_bfloat162 (reduced.cu).
cudaError_t launch_inverse_cols_bf16(const float2* Z, void* y16, long long n_samp, int n_ant,
                                     long long q0, long long nq, const GroupGeom& g,
                                     long long n_hi, long long n_lo, TwiddlePtrs tw,
                                     cudaStream_t st, const int* blk_list = nullptr);

// ---- true-delay beams (truedelay.cu) ----
// Y[(b - b0) np + p] = sum_a W_pa(f) X[b][a] for blocks b0 .. b0+nb-1 and
// pixels p_base .. p_base+np-1 of the group's spectra; ph: [n_pix][n_ant]
// {frac(f0 tau), frac(B tau / nfft)} as 64-bit fixed-point cycles; rot:
// [n_pix][n_ant] exp(2 pi j n1 B tau / nfft), the weight's step along a row.
cudaError_t launch_td_spectra(const float2* spec, float2* Y, long long b0, int nb, int np,
                              int p_base, int n_ant, const GroupGeom& g, const void* ph,
                              const float2* rot, cudaStream_t st);
// Column pass of nb x np beam sequences (from the row pass of Y with the DM's
// chirp), |y|^2 of the owned samples in [t_lo, t_hi) added to P[t / dump_len][p].
cudaError_t launch_inverse_cols_pow(const float2* Z, float* P, long long n_samp, long long b0,
                                    int nb, int np, int p_base, int n_pix, const GroupGeom& g,
                                    long long n_hi, long long n_lo, int dump_len, long long t_lo,
                                    long long t_hi, TwiddlePtrs tw, cudaStream_t st);

// ---- Chirpolator pre-integrator image on the tensor cores (cpi_tc.cu) ----
// Bytes of the dense split-BF16 filter image (all DMs) and window-DFT image.
long long cpi_tc_a_bytes(int n_dm, int n_pix, int nk, int n_pair);
long long cpi_tc_b_bytes(int n_dm, long long n_blk, int nk, int n_pair);
// Filter image from the sparse filter W [n_dm][n_pair][nj][n_pix] and its
// first bins K0 [n_dm][n_pair][n_pix] (clears the image first).
cudaError_t launch_cpi_tc_aimg(const float2* W, const short* K0, int n_dm, int n_pair, int nj,
                               int nk, int n_pix, uint8_t* aimg, cudaStream_t st);
// E [n_dm][n_blk][n_pix] = |A X|^2 from the window DFTs X [n_dm][n_blk][nk][n_pair]
// (zero while m < n_win[d] - 1); bimg is the plan's window-DFT image buffer.
cudaError_t launch_cpi_tc_image(const float2* X, uint8_t* bimg, const uint8_t* aimg,
                                const int* n_win, int n_dm, long long n_blk, int nk, int n_pair,
                                int n_pix, float* E, int* err, cudaStream_t st);

// ---- back-ends (backends.cu) ----
// Up to kCorrBatchMax DMs' back-ends in one launch (grid dimension z = DM):
// the correlator over DM j's voltages y (float2, or BF16 pairs), dumps
// m_base .. m_base + n_m - 1 or dump_list[0 .. n_m) (device), into vis; and
// the beams from visibilities V of rows first .. first + n_rows - 1 or
// dump_list[0 .. n_rows) into pow.
constexpr int kCorrBatchMax = kMaxChirps;
struct CorrJob {
  const void* y;
  float2* vis;
  long long m_base, n_m, first, last;
  const int* dump_list;
};
struct VisJob {
  const float2* V;
  float* pow;
  long long first, n_rows;
  const int* dump_list;
};
cudaError_t launch_correlate_batch(const CorrJob* jobs, int n_jobs, bool bf16, long long n_samp,
                                   int n_ant, int dump_len, cudaStream_t st);
// max_ctas > 0: at most that many CTAs, striding over the tiles.
cudaError_t launch_beam_from_vis_batch(const VisJob* jobs, int n_jobs, const float* wvis,
                                       int n_ant, int n_pix, cudaStream_t st, int max_ctas = 0);
// dumps m_base .. m_base + n_m - 1, or dump_list[0 .. n_m) when dump_list is a
// device array (zeros for dumps outside [first, last])
cudaError_t launch_correlate(const float2* y, long long n_samp, int n_ant, int dump_len,
                             long long m_base, long long n_m, long long first, long long last,
                             float2* vis, cudaStream_t st, const int* dump_list = nullptr);
// The same from dedispersed voltages rounded to BF16: y16 is [n_ant][n_samp]
// pairs (re, im) of BF16 (__nv_bfloat162); products and sums in FP32.
cudaError_t launch_correlate_bf16(const void* y16, long long n_samp, int n_ant, int dump_len,
                                  long long m_base, long long n_m, long long first, long long last,
                                  float2* vis, cudaStream_t st, const int* dump_list = nullptr);
// Beams from the visibility matrix V [n_dump][n_pair] of one DM: dumps
// first..last, or the n_list dumps of dump_list (device) when given.  wvis is
// the real pair-weight matrix [beam_vis_rows(n_ant)][beam_vis_ld(n_pix)]:
// row 2i = Re w_p,i, row 2i+1 = -Im w_p,i, zero padding.
int beam_vis_rows(int n_ant);
int beam_vis_ld(int n_pix);
cudaError_t launch_beam_from_vis(const float2* V, const float* wvis, int n_ant, int n_pix,
                                 long long first, long long last, float* pow, cudaStream_t st,
                                 const int* dump_list = nullptr, long long n_list = 0);
cudaError_t launch_beamform_simt(const float2* y, long long n_samp, int n_ant, int dump_len,
                                 long long m_base, long long n_m, long long first, long long last,
                                 const float2* W, int n_pix, float* pow, cudaStream_t st);

// ---- incoherent filterbank path (incoherent.cu) ----
// scratch holds a copy of the voltages ([n_ant] rows of seq_stride samples) and
// is transformed in place; S [n_chan][T_fb], D [n_dm][T_fb]; shift [n_dm][n_chan]
// y[a][t] = scale[a] * complex int8 x[a][t] as complex64 (scale NULL = 1)
cudaError_t launch_unpack_ci8(const void* x, const float* scale, int n_ant, long long n_samp,
                              float2* y, cudaStream_t st);
cudaError_t launch_incoherent(float2* scratch, long long seq_stride, int n_ant, int n_chan,
                              int n_int, long long T_fb, const int* shift, int n_dm, float* S,
                              float* D, TwiddlePtrs tw, cudaStream_t st);

// ---- tensor-core beamformer (beamform_tc.cu) ----
// terms = 3: split-BF16 (A_h B_h + A_h B_l + A_l B_h); terms = 1: plain BF16
int beam_tc_groups(int n_ant);                // 8-wide real-K groups per head/tail part
int beam_tc_bgroups(int n_ant, int terms);    // 8-wide k-groups of one B tile
int beam_tc_ksteps(int n_ant, int terms);     // 16-wide MMA K steps
// Kernel shape: 1 = 128-sample tiles, weights in shared memory; 2 = 256-sample
// tiles (dump_len % 256 == 0); 3 = 128-sample tiles, weights in TMEM.
// forced = 0 picks the preferred shape that fits; a forced shape that does
// not fit, or no fitting shape, gives 0.
int beam_tc_pick(int n_ant, int n_pix, int dump_len, int terms, int forced);
int beam_tc_tile_samples(int shape);                          // samples per B tile
long long beam_tc_tile_bytes(int n_ant, int shape, int terms);  // bytes of one B tile
std::vector<uint8_t> build_beam_a_image(const double* W, int n_ant, int n_pix, int terms);
// t_origin: sample of column 0 of B tile 0 (dump-aligned for 256-sample tiles)
cudaError_t launch_beam_tc(const uint8_t* b_img, const uint8_t* a_img, int n_ant, int n_pix,
                           int dump_len, long long first, long long last, long long t_origin,
                           float* pow, int* err, int terms, int shape, cudaStream_t st);

// ---- tensor-core correlator (corr_tc.cu) ----
// terms = 3: split-BF16 ([H; L] H^T), terms = 1: plain BF16 (H H^T)
bool corr_tc_supported(int n_ant, int dump_len, int terms);
// vis[m][pair] for the dumps first..last of one DM (FP32 accumulation)
cudaError_t launch_correlate_tc(const float2* y, long long n_samp, int n_ant, int dump_len,
                                long long first, long long last, float2* vis, int* err, int terms,
                                cudaStream_t st);

// ---- candidate detection (detect.cu) ----
long long detect_chunks(int n_dm, long long n_dump, int n_pix);  // entries of counts / offsets
cudaError_t launch_detect(const float* P, int n_dm, long long n_dump, int n_pix,
                          const long long* first, const long long* last, float snr_min,
                          float2* stats, int* counts, long long* offsets, long long* n_total,
                          chirp_candidate* out, long long max_out, cudaStream_t st);

}  // namespace chirp
