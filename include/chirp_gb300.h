/*
 * chirp_gb300.h -- C ABI of the GB300 (sm_103a) coherent-dedispersion pulse
 * search: per-antenna overlap-save coherent dedispersion for every trial DM,
 * feeding either a per-DM integrate-and-dump correlator ("Chirpolator"
 * back-end) or a per-DM phased-beam detector ("Chimageator" back-end).
 *
 * Paper: K. W. Bannister & T. J. Cornwell, "Two efficient, new techniques for
 * detecting dispersed radio pulses with interferometers: The Chirpolator and
 * The Chimageator" (arXiv:1109.3186).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Voltages are complex baseband, complex-Nyquist sampled at f_s = B
 *    (Sec. 3.2, below Eq. xpq): complex64 (interleaved float re, im),
 *    antenna-major [n_ant][n_samp].
 *  - Dispersion follows Eq. 1 (Sec. 2.1) with constant k_dm (s Hz^2 per
 *    pc cm^-3; mu ~ 4.15 ms GHz^2 in the paper).  Dedispersion multiplies the
 *    spectrum of each overlap-save block by
 *        H_DM(f) = exp(-2 pi j k_dm DM f^2 / (f0^2 (f0 + f)))
 *    (the inverse ISM response of Sec. 2.3.2 about f0); the forward DFT
 *    has the paper's sign exp(-2 pi j n k / N) (Eq. dft); the inverse
 *    includes 1/Nfft.
 *  - Per DM: n_hi = ceil(k DM (f0^-2 - (f0+B/2)^-2) B),
 *            n_lo = ceil(k DM ((f0-B/2)^-2 - f0^-2) B);
 *    Nfft = max(nfft_min, min(pow2ceil(2 (n_hi + n_lo)), pow2ceil(n_samp)));
 *    DMs with equal Nfft share one block grid of step
 *    S = Nfft - max n_hi - max n_lo, rounded down to a multiple of 8 when at
 *    least 8.  Output sample t refers to the arrival
 *    at f0 and is valid for t in [n_hi, n_samp - n_lo).
 *  - Dumps are the absolute grid [m L, (m+1) L), m < floor(n_samp / L).  A
 *    dump is valid for a DM only if it lies inside that DM's valid range;
 *    invalid dumps are written as zeros.
 *  - Return codes: CHIRP_OK (0) or a negative CHIRP_E*; the message of the
 *    last failure on the calling thread is in chirp_last_error().  No C++
 *    exception crosses this boundary.
 *  - Ownership: the caller owns every input and output buffer; the plan
 *    owns its device workspace and frees it in chirp_plan_destroy.  The
 *    library never frees caller memory.
 *  - Streams: all device work of a plan is ordered on the CUDA stream given
 *    at creation (NULL = legacy default stream).  A call whose outputs are
 *    on the device returns once the work is queued; a call with any host
 *    output synchronises that stream before returning.
 */
#ifndef CHIRP_GB300_H
#define CHIRP_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

#define CHIRP_OK 0
#define CHIRP_EINVAL (-1)      /* bad argument or size                     */
#define CHIRP_ENOMEM (-2)      /* device or host allocation failed          */
#define CHIRP_ECUDA (-3)       /* a CUDA runtime call or launch failed      */
#define CHIRP_ETIMEOUT (-4)    /* a bounded device wait gave up              */
#define CHIRP_EUNSUPPORTED (-5)/* valid request the library does not handle */

/* where a caller buffer lives */
#define CHIRP_HOST 0
#define CHIRP_DEVICE 1

/* contraction used by the Chimageator back-end */
#define CHIRP_BEAM_AUTO 0      /* the faster exact form for the shape, by a
                                  cost model of both: CHIRP_BEAM_VIS when its
                                  correlation + quadratic form is estimated
                                  cheaper than the split-BF16 GEMM (e.g. 12
                                  antennas, 1024 pixels), or when no tensor-core
                                  shape fits; else CHIRP_BEAM_TC_3XBF16       */
#define CHIRP_BEAM_FP32_SIMT 1 /* plain FP32 FMA on the CUDA cores           */
#define CHIRP_BEAM_TC_3XBF16 2 /* tcgen05, 3-term bf16 split, FP32 accumulate
                                  (above 60 antennas the weights are held in
                                  TMEM instead of shared memory)             */
#define CHIRP_BEAM_VIS 3       /* exact identity sum_t |w.y|^2 = w^H V w: the
                                  per-dump visibilities V (Chirpolator output)
                                  are formed first, then a quadratic form per
                                  pixel; FP32 CUDA cores                      */
#define CHIRP_BEAM_TC_BF16 4   /* reduced-precision form: tcgen05, operands
                                  rounded once to BF16 (one product), FP32
                                  accumulate; relative error of a beam power
                                  ~1e-3 (held to 1e-2)                        */
#define CHIRP_BEAM_VIS_BF16 5  /* reduced-precision visibility identity: the
                                  inverse column pass rounds the dedispersed
                                  voltages once to BF16 (4 bytes per antenna-
                                  sample instead of 8), the correlator and the
                                  quadratic form run in FP32 on the CUDA cores;
                                  relative error of a beam power ~1e-4 (held
                                  to 1e-2)                                    */

/* contraction used by the Chirpolator back-end (and by CHIRP_BEAM_VIS) */
#define CHIRP_CORR_AUTO 0      /* CHIRP_CORR_TC_3XBF16 from 17 antennas up where
                                  supported (dump length a multiple of 128, or
                                  a divisor of 256 that is a multiple of 16; up
                                  to 48 antennas),
                                  else CHIRP_CORR_FP32_SIMT; the visibility
                                  beam mode then keeps FP32 products (its sum
                                  over M^2 pairs amplifies the ~1e-6 relative
                                  error of split-BF16 visibilities by up to M) */
#define CHIRP_CORR_FP32_SIMT 1 /* FP32 FMA on the CUDA cores                  */
#define CHIRP_CORR_TC_3XBF16 2 /* tcgen05, [H; L] H^T split-BF16, FP32 acc    */
#define CHIRP_CORR_TC_BF16 3   /* reduced precision: tcgen05, H H^T in BF16,
                                  FP32 accumulate (relative error ~1e-3)      */

/* element type of the voltage input (chirp_config.in_type) */
#define CHIRP_IN_C64 0         /* complex64: interleaved FP32 (re, im)        */
#define CHIRP_IN_CI8 1         /* complex int8: interleaved (re, im) bytes,
                                  value = in_scale[a] * (re + j im); converted
                                  to FP32 inside the first FFT pass           */

typedef struct chirp_plan chirp_plan;

/* Everything that fixes the shape of a search.  All pointers are HOST
 * memory and are copied at plan creation. */
typedef struct {
  int n_ant;               /* M antennas, 1..84                                  */
  const double* xyz_m;     /* [n_ant][3] positions, metres, (u,v,w) frame with w
                              towards the phase centre (App. A.1, Eq. tau3D);
                              only the Chimageator reads them (may be NULL
                              otherwise)                                        */
  double f0_hz;            /* band centre                                       */
  double bw_hz;            /* bandwidth = complex sample rate                   */
  double k_dm;             /* dispersion constant; <= 0 selects 4.148808e15     */
  long long n_samp;        /* samples per antenna, >= 1                         */
  const double* dm;        /* [n_dm] trial DMs, pc cm^-3, each >= 0             */
  int n_dm;                /* >= 1                                              */
  int dump_len;            /* L samples per integrate-and-dump, 1..n_samp       */
  long long nfft_min;      /* power of two, 256 .. 2^24                         */
  const double* pix_lm;    /* [n_pix][2] beam direction cosines (l, m), or NULL */
  int n_pix;               /* 0 when no Chimageator runs are wanted             */
  int beam_mode;           /* CHIRP_BEAM_*                                      */
  /* incoherent filterbank search (chirp_incoherent_run); fb_chan = 0: off    */
  int fb_chan;             /* channels per antenna, power of two 16..4096       */
  int fb_int;              /* spectra integrated per filterbank sample, >= 1    */
  const double* fb_dm;     /* [fb_n_dm] trial DMs of the incoherent search      */
  int fb_n_dm;
  int flags;               /* CHIRP_FLAG_* bits                                 */
  int in_type;             /* CHIRP_IN_*: element type of every voltage input
                              of this plan's runs ([n_ant][n_samp] elements) */
  const float* in_scale;   /* [n_ant] scale of CHIRP_IN_CI8 input; NULL = 1   */
  int corr_mode;           /* CHIRP_CORR_*; a tensor-core mode the shape does not
                              allow gives CHIRP_EUNSUPPORTED                  */
  int beam_shape;          /* tensor-core beam kernel shape: 0 = the library's
                              choice; 1 = 128-sample tiles, weights in shared
                              memory; 2 = 256-sample tiles (dump_len % 256 ==
                              0); 3 = 128-sample tiles, weights in TMEM.  A
                              shape that does not fit: CHIRP_EUNSUPPORTED    */
  int fft_row;             /* 0: row length of the two-pass FFT chosen by the
                              library (or the autotuner); else a power of two
                              in 256..4096 forced for every FFT-length group
                              whose column length Nfft/fft_row lies in
                              16..4096 (other groups keep the default)        */
} chirp_config;

/* chirp_config.flags */
#define CHIRP_FLAG_GRAPHS 1   /* replay full device-buffer searches as CUDA graphs:
                                 the first call with a given (input, output,
                                 back-end) runs eagerly, the second captures the
                                 launch sequence, later calls launch the graph.
                                 Needs a non-default plan stream.  Stage timing
                                 does not see inside graph launches.          */
#define CHIRP_FLAG_LEAN 4     /* hold the forward spectra of one FFT-length
                                 group at a time (one buffer sized for the
                                 largest group, each group's spectra formed
                                 right before its DMs) instead of every
                                 group's: less device memory, the forward
                                 passes re-run when a search revisits a group
                                 (same outputs)                               */
#define CHIRP_FLAG_AUTOTUNE 2 /* time the candidate FFT factorisations (row
                                 length 512..4096) of every FFT-length group on
                                 the device at plan creation and keep the
                                 fastest; results differ from the default split
                                 only by rounding.  Cached per process.       */

typedef struct {
  long long n_dump;        /* floor(n_samp / dump_len)                          */
  int n_pair;              /* n_ant (n_ant + 1) / 2                             */
  int n_group;             /* distinct FFT lengths                              */
  long long workspace_bytes;/* device memory owned by the plan (grows on the
                              first run that needs the dedispersed-voltage
                              buffer -- one n_ant x n_samp slot per DM of a
                              row-pass chunk, so that the chunk's back-ends
                              run as one launch, unless the plan is lean or
                              the slots would pass 4 GB -- or host-buffer
                              staging)                                       */
  long long ifft_points;   /* sum over DMs of n_ant * n_blk * Nfft              */
  long long valid_samples; /* sum over DMs of n_ant * (n_samp - n_hi - n_lo)^+  */
  int beam_mode;           /* CHIRP_BEAM_* actually used (AUTO resolved)        */
  long long fb_samples;    /* T_fb of the incoherent search (0 when off)        */
  int beam_shape;          /* tensor-core beam kernel shape used (0: none)      */
  int corr_mode;           /* CHIRP_CORR_* actually used (AUTO resolved)        */
  int dm_chunk;            /* trial DMs of one FFT-length group whose inverse
                              row passes a full search runs in one launch (the
                              group's spectra are read once for them); the
                              staged FP32 correlator and the visibility beams
                              of those DMs also run as one launch each       */
} chirp_plan_info;

/* Create a plan: validates cfg, derives the per-DM FFT lengths and block
 * grids (header conventions), allocates the device workspace, builds the
 * FP64 chirp-phase tables, twiddle tables and beam weights on the device.
 * stream: a cudaStream_t (or NULL).  On success *plan is set.
 * Errors: CHIRP_EINVAL (bad shape), CHIRP_ENOMEM, CHIRP_ECUDA. */
int chirp_plan_create(chirp_plan** plan, const chirp_config* cfg, void* stream);

/* Destroy a plan (NULL is ignored).  Synchronises the plan's stream first. */
void chirp_plan_destroy(chirp_plan* plan);

/* Sizes derived at creation.  Errors: CHIRP_EINVAL on NULL. */
int chirp_plan_query(const chirp_plan* plan, chirp_plan_info* info);

/* FFT length and two-pass split of every FFT-length group: nfft[g] =
 * n_col[g] * n_row[g] (arrays of chirp_plan_info.n_group entries, caller
 * owned).  Errors: CHIRP_EINVAL on NULL arguments. */
int chirp_plan_fft_split(const chirp_plan* plan, long long* nfft, int* n_col, int* n_row);

/* Block grid of DM number d: out7 = {Nfft, n_hi, n_lo, max n_hi of the group,
 * max n_lo of the group, step S, number of blocks}.  Errors: CHIRP_EINVAL. */
int chirp_dm_layout(const chirp_plan* plan, int d, long long* out7);

/* Valid dump range of every DM: first[d] .. last[d] inclusive (last < first
 * when a DM has no valid dump).  first, last: host arrays of n_dm. */
int chirp_dump_range(const chirp_plan* plan, long long* first, long long* last);

/* Coherent dedispersion of one trial DM (Sec. 2.3.2), the shared first stage
 * of both searches.  volt: [n_ant][n_samp] elements of the plan's in_type
 * (complex64 or complex int8, the same for every run below) at volt_loc; y_out:
 * complex64 [n_ant][n_samp] at y_loc; samples outside the DM's valid range
 * are zero.  Errors: CHIRP_EINVAL, CHIRP_ECUDA. */
int chirp_dedisperse_run(chirp_plan* plan, const void* volt, int volt_loc, int d, void* y_out,
                         int y_loc);

/* Chirpolator back-end: for every trial DM and dump, the zero-lag
 * visibilities V_pq = sum_t y_p(t) y_q(t)^* of the dedispersed voltages
 * (pair mixing x_pq = s_p s_q^* of Eq. xpq, integrated and dumped; autos
 * included).  vis_out: complex64 [n_dm][n_dump][n_pair], pairs p <= q in
 * row-major order (0,0),(0,1),..,(0,M-1),(1,1),...  Errors: CHIRP_EINVAL,
 * CHIRP_ECUDA. */
int chirpolator_run(chirp_plan* plan, const void* volt, int volt_loc, void* vis_out, int vis_loc);

/* Chimageator back-end in its phased-sum form: for every trial DM, dump and
 * pixel, P = sum_t |sum_a W_pa y_a(t)|^2 with narrowband weights
 * W_pa = exp(+2 pi j f0 tau_a(l_p, m_p)), tau from Eq. tau3D (direct
 * beamforming, Sec. 2.4.2, detected and integrated).  pow_out: float32
 * [n_dm][n_dump][n_pix].  Needs n_pix > 0 at plan creation.  With the
 * tensor-core mode the contraction runs as three BF16 products (head x head,
 * head x tail, tail x head) accumulated in FP32; with CHIRP_BEAM_VIS the same
 * powers come from the per-dump visibility matrix (identical up to rounding).  Errors: CHIRP_EINVAL,
 * CHIRP_EUNSUPPORTED, CHIRP_ECUDA, CHIRP_ETIMEOUT (host outputs only; see
 * chirp_plan_status). */
int chimageator_run(chirp_plan* plan, const void* volt, int volt_loc, float* pow_out, int pow_loc);

/* True-delay (wideband) beams of the dedispersed voltages (Sec. 2.4.2
 * direct beamforming with each antenna's geometric delay of Eq. tau3D applied
 * at every frequency rather than as one phase at f0).  In overlap-save block
 * b of DM d, with X_ab the block's spectrum and H the DM's chirp,
 *   Y_pb(f) = H(f) sum_a exp(+2 pi j (f0 + f) tau_a(l_p, m_p)) X_ab(f),
 * f = i B / Nfft for bin i < Nfft/2, (i - Nfft) B / Nfft from there; the beam
 * is the inverse transform (1/Nfft included) over the samples block b owns,
 * and P[d][m][p] = sum over dump m of |beam|^2 for the DM's valid dumps, zero
 * elsewhere.  Block grid, chirp, ownership and valid dumps are those of the
 * phased beams; the geometric delays (at most B max|tau| samples) wrap inside
 * a block like the chirp's tail does.  The weights' phases are formed in
 * 64-bit fixed point from FP64 (exact modulo one cycle), the sums in FP32
 * (dump sums by atomic adds, so the last bits may differ between runs).
 * Costs n_pix / n_ant times the phased beams' inverse-FFT work; the sums
 * over antennas do not depend on the DM and are formed once per FFT-length
 * group (and chunk of pixels) for all of the group's DMs.
 *  pow_out: float32 [n_dm][n_dump][n_pix] at pow_loc (chimageator_run's
 *  layout).  Needs pixels and antenna positions at plan creation.  The first
 *  call allocates the beam spectra of one group's pixel chunk (at most 8 GB),
 *  a 1 GB chunk buffer of the inverse and the per-group phase tables.
 *  Errors: CHIRP_EINVAL, CHIRP_EUNSUPPORTED, CHIRP_ENOMEM, CHIRP_ECUDA. */
int chirp_truedelay_run(chirp_plan* plan, const void* volt, int volt_loc, float* pow_out,
                        int pow_loc);

/* Antenna-incoherent search (Sec. 2.3.1 incoherent dedispersion of the power
 * beam of Sec. 2.4.1), the cheap stage that proposes where the coherent path
 * should look.  Each antenna's series is cut into blocks of fb_chan samples
 * and transformed (e^{-2 pi j n k / L}); channels are in ascending frequency
 * f_c = f0 + (c - fb_chan/2) B / fb_chan; |X|^2 is summed over antennas and
 * fb_int blocks:  S[c][tau], tau < T_fb = floor(n_samp / (fb_chan fb_int)).
 * Then D[d][t] = sum_c S[c][t + s_c(d)] with the Eq. dmdelay lag relative to
 * f0 in filterbank samples, s_c = floor(k DM (f_c^-2 - f0^-2) / t_fb + 1/2),
 * t_fb = fb_chan fb_int / B; D is zero outside [-min s, T_fb - max s).
 *  volt: [n_ant][n_samp] of the plan's in_type at volt_loc (not modified);
 *  S_out: float32 [fb_chan][T_fb] or NULL;  D_out: float32 [fb_n_dm][T_fb];
 *  both at out_loc.  Needs fb_chan > 0 at plan creation.
 * Errors: CHIRP_EINVAL, CHIRP_EUNSUPPORTED, CHIRP_ECUDA. */
int chirp_incoherent_run(chirp_plan* plan, const void* volt, int volt_loc, float* S_out,
                         float* D_out, int out_loc);

/* ---- learned proposer: a 1-D convolutional network over the incoherent
 * dedispersed power (trial DMs as channels, filterbank samples as time) that
 * scores every (DM, time) cell; the coherent path then runs only where the
 * score is high.  Layers: h1 = relu(conv(x, W1, b1, k1/2)), h2 =
 * relu(conv(h1, W2, b2, k2/2)), z = conv(h2, W3, b3, 0) with width 1, where
 * conv(x, W, b, pad)[b, o, t] = b[o] + sum_{i,k} W[o, i, k] x[b, i, t + k - pad]
 * (zero padding).  Loss: mean class-weighted BCE with logits; optimiser Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).  All FP32, all on the device.  Not an
 * operation of the paper: the proposal stage of the search.
 * Parameters are one flat FP32 vector in the order W1 [hidden][n_dm][k1],
 * b1 [hidden], W2 [hidden][hidden][k2], b2 [hidden], W3 [n_dm][hidden], b3 [n_dm].
 * Activations x, logits, labels: DEVICE float32 [batch][n_dm][n_time]. */
typedef struct chirp_propnet chirp_propnet;
/* k1, k2 odd and <= 15; buffers for up to max_batch segments of n_time. */
int chirp_propnet_create(chirp_propnet** net, int n_dm, int hidden, int k1, int k2, int max_batch,
                         int n_time, void* stream);
void chirp_propnet_destroy(chirp_propnet* net);
long long chirp_propnet_param_count(const chirp_propnet* net);
/* host float32 [param_count]; set_params also resets the Adam state */
int chirp_propnet_set_params(chirp_propnet* net, const float* params);
int chirp_propnet_get_params(const chirp_propnet* net, float* params);
/* The trainer's whole state, for checkpoint and resume: parameters, Adam's
 * first and second moments (host float32 [param_count] each) and the Adam
 * step count (the bias corrections of the next step use step + 1).  After
 * set_state the next train_step continues exactly as the saved trainer
 * would have.  Errors: CHIRP_EINVAL (NULL buffer, negative step), CHIRP_ECUDA. */
int chirp_propnet_get_state(const chirp_propnet* net, float* params, float* m, float* v,
                            long long* step);
int chirp_propnet_set_state(chirp_propnet* net, const float* params, const float* m,
                            const float* v, long long step);
/* gradients of the last backward / train step, host float32 [param_count] */
int chirp_propnet_get_grads(const chirp_propnet* net, float* grads);
int chirp_propnet_forward(chirp_propnet* net, const float* x, int batch, float* logits);
/* forward + backward (gradients kept on the device); loss_host may be NULL */
int chirp_propnet_backward(chirp_propnet* net, const float* x, const float* y, int batch,
                           float pos_weight, float* loss_host);
/* forward + backward + one Adam step of learning rate lr */
int chirp_propnet_train_step(chirp_propnet* net, const float* x, const float* y, int batch,
                             float pos_weight, float lr, float* loss_host);
/* x[d][t] = (D[d][t] - mean_d) / std_d over the nonzero (valid) samples of
 * each row; zeros stay zero.  D, x: DEVICE float32 [n_dm][n_time]. */
int chirp_propnet_normalize(const float* D, int n_dm, long long n_time, float* x, void* stream);
/* mask[d][w] = 1 where the largest logit of window w (win samples) of DM d
 * exceeds thr.  logits: DEVICE float32 [n_dm][n_time]; mask: DEVICE int32
 * [n_dm][ceil(n_time / win)]. */
int chirp_propose_windows(const float* logits, int n_dm, long long n_time, int win, float thr,
                          int* mask, void* stream);

/* Per-stage device time.  Stages: */
#define CHIRP_STAGE_FORWARD 0   /* forward FFT passes of every group            */
#define CHIRP_STAGE_INV_ROWS 1  /* chirp multiply + inverse row pass, per DM    */
#define CHIRP_STAGE_INV_COLS 2  /* inverse column pass + discard, per DM        */
#define CHIRP_STAGE_CORRELATE 3 /* Chirpolator back-end, per DM                 */
#define CHIRP_STAGE_BEAMFORM 4  /* Chimageator back-end, per DM                 */
#define CHIRP_STAGE_SPLIT 5     /* not timed: the BF16 image of the voltages is
                                   written by the inverse column pass        */
#define CHIRP_STAGE_CHIRP 6     /* FP64-phase chirp table H_DM, per DM           */
#define CHIRP_STAGE_INCOHERENT 7 /* filterbank + incoherent dedispersion        */
#define CHIRP_STAGE_DETECT 8    /* candidate detection (chirp_detect)            */
#define CHIRP_STAGE_TD_SPECTRA 9 /* true-delay beam spectra (chirp_truedelay_run) */
#define CHIRP_N_STAGES 10
/* Returns the milliseconds and launch counts accumulated per stage since the
 * previous call (ms, launches: host arrays of CHIRP_N_STAGES, either may be
 * NULL), resets them, and switches event timing on (enable != 0) or off for
 * later runs: enable = 1 times every stage; CHIRP_TIMING_SELECT | mask times
 * only the stages whose bit (1 << CHIRP_STAGE_*) is set in mask.  Timing
 * records one CUDA event pair around every timed launch on the plan's stream
 * (a few microseconds each); reading the totals synchronises that stream.
 * Not a paper operation: instrumentation for the roofline report.
 * Errors: CHIRP_EINVAL. */
#define CHIRP_TIMING_SELECT 0x40000000
int chirp_stage_timing(chirp_plan* plan, int enable, double* ms, long long* launches);

/* Allocation-free dedispersion of one trial DM.  No counterpart in the
 * paper: it exists for callers that cannot allocate device memory -- code
 * running while another library holds the stream in capture (allocation is
 * illegal there), real-time pipelines that reserve all GPU memory at start-up,
 * and hosts that must avoid the implicit device synchronisation of
 * cudaMalloc/cudaFree.  It computes exactly what chirp_dedisperse_run computes
 * for a plan whose DM list is {dm} alone, with every intermediate kept in a
 * fixed array of CHIRP_NOALLOC_SCRATCH_BYTES that the library holds on every
 * GPU that loads it, until the process exits.
 *  volt:  DEVICE complex64 [n_ant][n_samp];  y_out: DEVICE complex64
 *         [n_ant][n_samp], zero outside the DM's valid range; both must be
 *         device or managed memory (a host pointer gives CHIRP_EINVAL);
 *  stream: cudaStream_t (NULL = legacy default stream); work is queued on it.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  The first
 * call on a device looks up the array's device address and fills its twiddle
 * tables, synchronising the stream: make that first call before any stream
 * capture.  All calls share the one array and it keeps the previous call's
 * contents, so calls whose work overlaps on the GPU (other streams, other
 * threads) race and corrupt each other; serialise them.
 * Errors: CHIRP_EINVAL (bad argument, or a shape whose scratch need exceeds
 * CHIRP_NOALLOC_SCRATCH_BYTES, with the need in the message),
 * CHIRP_EUNSUPPORTED, CHIRP_ECUDA. */
#define CHIRP_NOALLOC_SCRATCH_BYTES (32u << 20)
int chirp_dedisperse_noalloc(const void* volt, int n_ant, long long n_samp, double f0_hz,
                             double bw_hz, double k_dm, double dm, long long nfft_min, void* y_out,
                             void* stream);

/* Synchronises the plan's stream and reports whether any bounded device wait
 * of an earlier run gave up (the tensor-core beamformer never spins without
 * a limit).  Returns CHIRP_OK, or CHIRP_ETIMEOUT when outputs of some run are
 * invalid; the flag stays raised for the plan's lifetime.  Host-output runs
 * of chimageator_run check it themselves.  Errors: CHIRP_EINVAL, CHIRP_ECUDA. */
int chirp_plan_status(chirp_plan* plan);

/* Selective searches: as chirpolator_run / chimageator_run but only for the
 * (DM, dump) cells whose byte in cell_mask (HOST uint8 [n_dm][n_dump]) is
 * nonzero -- e.g. the cells proposed by the learned proposer.  The back-end
 * runs only on selected dumps; every other output cell is zero.  Per
 * FFT-length group, when the selected DMs need at least 85 % of their
 * (DM, overlap-save block) pairs the group's inverse transforms run in full
 * with the multi-DM row pass (one spectrum read for up to 4 DMs); otherwise
 * only the blocks that own a selected dump are inverse transformed, each DM
 * over its own blocks, up to dm_chunk DMs of the group per launch.  The
 * selected cells hold exactly what the full search computes there.
 * Errors: as the full searches. */
int chirpolator_run_selective(chirp_plan* plan, const void* volt, int volt_loc,
                              const unsigned char* cell_mask, void* vis_out, int vis_loc);
int chimageator_run_selective(chirp_plan* plan, const void* volt, int volt_loc,
                              const unsigned char* cell_mask, float* pow_out, int pow_loc);

/* Several searches (observations of any shapes) queued together: search i
 * runs plans[i] (backend 0 = chirpolator_run, 1 = chimageator_run) on volts[i]
 * into outs[i] with the given buffer locations.  Plans created on distinct
 * streams overlap on the device; calls with host outputs synchronise their
 * own stream.  Errors: as the single searches (the first failure stops the
 * batch). */
int chirp_batch_run(chirp_plan* const* plans, const void* const* volts, const int* volt_locs,
                    void* const* outs, const int* out_locs, const int* backends, int n);

/* One detection: trial DM index, dump, pixel, its S/N and dump power. */
typedef struct {
  long long dump;
  int dm;
  int pix;
  float snr;
  float power;
} chirp_candidate;

/* Candidate detection on Chimageator dump powers (thresholding of the
 * detection metric, Sec. 3.3 after Eq. eth; the best of a bank of trial
 * filters over DM, time and direction, App. A.3).  Per (DM, pixel) series
 * over the DM's valid dumps: med = median (even count: mean of the two
 * middle values), sigma = 1.4826 * median(|x - med|), S/N = (x - med) / sigma
 * (0 where sigma == 0), each an IEEE-rounded FP32 operation.  A candidate is
 * a valid cell with S/N >= snr_min that no valid cell among its 26 neighbours
 * (DM +- 1, dump +- 1, pixel index +- 1) exceeds.
 *  pow:   float32 [n_dm][n_dump][n_pix] at pow_loc (chimageator_run's layout);
 *  cand:  [max_cand] at cand_loc, filled in (DM, dump, pixel) order with the
 *         first min(*n_cand, max_cand) candidates;
 *  n_cand: HOST, receives the total number of candidates;
 *  stats_out: NULL or float32 [n_dm][n_pix][2] (med, sigma) at cand_loc.
 * Synchronises the plan's stream.  Errors: CHIRP_EINVAL, CHIRP_EUNSUPPORTED
 * (plan without pixels), CHIRP_ENOMEM, CHIRP_ECUDA. */
int chirp_detect(chirp_plan* plan, const float* pow, int pow_loc, float snr_min,
                 chirp_candidate* cand, long long max_cand, int cand_loc, long long* n_cand,
                 float* stats_out);

/* Self-test of the device watchdog (no GPU fault, trap or endless loop): a
 * one-CTA kernel runs the bounded mbarrier wait of the tensor-core kernels'
 * roles on a barrier that nothing arrives at, with a limit of `polls` polls
 * (1 .. 2^24; each poll after the 32nd sleeps ~64 ns).  The wait must give up
 * and raise the device error word the host reads.  Returns CHIRP_ETIMEOUT --
 * the code a run whose wait gave up reports through chirp_plan_status -- and
 * the kernel's duration in *waited_ms (HOST, may be NULL), with the context
 * still usable; CHIRP_ECUDA if the wait wrongly succeeded or a CUDA call
 * failed; CHIRP_EINVAL for a poll count out of range.  Synchronises stream. */
int chirp_watchdog_selftest(unsigned int polls, double* waited_ms, void* stream);

/* ------------------------------------------------------------------------
 * The paper's own Chirpolator pre-integrator (Sec. 3, App. A.3) on the RAW
 * voltages, for every trial DM:
 *   mixing       x_pq[n] = y_p[n] y_q[n]^*, p < q (Eq. xpq)
 *   partial DFTs V_k[m] = sum_{n<L} exp(-2 pi j (n + mL) k / N) x_pq[n + mL]
 *                (Sec. A.3.2), k in [-K, K], blocks m < n_blk = floor(n_samp / L)
 *   moving sum   S_k[m] = S_k[m-1] + V_k[m] - V_k[m - n_win] (Eq. block_cic)
 *   window DFT   X_k[m] = exp(2 pi j (m + 1 - n_win) k / n_win) S_k[m], the
 *                DFT of samples [(m + 1 - n_win) L, (m + 1) L) in their own
 *                time; zero while m < n_win - 1
 *   image        P = sum_{p<q} sum_{k = k0'-F}^{k0'+F} w_pq,k X_pq,k (Eq. pth
 *                with the 2F+1-bin matched filter of Sec. 3.4), E = |P|^2
 *                (Eq. eth)
 * A trial DM is a linear chirp (Sec. 2.1, Eq. freqvst2, about the sweep's
 * temporal midpoint): T = k_dm DM ((f0 - B/2)^-2 - (f0 + B/2)^-2),
 * alpha = ((f0 - B/2)^-2 + (f0 + B/2)^-2) / 2, a0 = alpha^-1/2 (Hz),
 * fdot = a1 = -alpha^-3/2 / (2 k_dm DM) (Hz/s), window
 * n_win = max(1, floor(B T / L + 1/2)) blocks, N = n_win L.  For direction
 * (l, m) with delays tau from Eq. tau3D: kappa = -fdot (tau_p - tau_q) N / B
 * (Eq. f0Bt), k0' = rint(kappa), and the filter is the conjugate response of
 * a unit chirp whose midpoint is at the window centre,
 *   w_pq,k = conj(phi exp(-pi j kappa) exp(-pi j (k - kappa)(N-1)/N))
 *            D_N(k - kappa) / N,
 *   phi = exp(pi j fdot (tau_p^2 - tau_q^2) - 2 pi j a0 (tau_p - tau_q)),
 * D_N the Dirichlet kernel (Eq. dn).  Pair pq needs bins |k| <= K_pq =
 * max over DMs and pixels of |k0'| + F (Sec. A.3.1); bins beyond it are not
 * computed and read as zero.
 * All arithmetic is FP32 on the CUDA cores; the moving sums carry each sum as
 * two floats (compensated, TwoSum) and the filter table is built in FP64 and
 * rounded once.  The partial DFTs are evaluated by a
 * Taylor expansion inside sub-blocks whose truncation is below 1e-9 of the
 * sub-block's sum of |x_pq| (chirp_cpi_info.sub_len, .n_terms).
 * ---------------------------------------------------------------------- */
typedef struct chirp_cpi_plan chirp_cpi_plan;

/* All pointers are HOST memory, copied at plan creation. */
typedef struct {
  int n_ant;             /* M, 2..84                                          */
  const double* xyz_m;   /* [n_ant][3] positions, metres ((u,v,w), Eq. tau3D)  */
  double f0_hz;          /* band centre                                        */
  double bw_hz;          /* bandwidth = complex sample rate                    */
  double k_dm;           /* <= 0 selects 4.148808e15 s Hz^2 / (pc cm^-3)       */
  long long n_samp;      /* samples per antenna, >= blk_len                    */
  const double* dm;      /* [n_dm] trial DMs, each > 0                          */
  int n_dm;              /* >= 1                                               */
  int blk_len;           /* L, power of two 16..65536                          */
  const double* pix_lm;  /* [n_pix][2] direction cosines                       */
  int n_pix;             /* >= 1                                               */
  int half_width;        /* F, 0..8                                            */
  int max_bin;           /* K (0: the smallest that holds every pixel's bins);
                            at most 64                                         */
  int image_mode;        /* 0: the image as a dense contraction on the tcgen05
                            tensor cores (the filter densified over all 2K+1
                            bins, split-BF16 operands: A_h B_h + A_h B_l +
                            A_l B_h, FP32 accumulate; about 2.4 GB of operand
                            images on the bench workload); 1: the sparse
                            2F+1-bin gathers on the CUDA cores               */
} chirp_cpi_config;

typedef struct {
  int n_pair;            /* M (M - 1) / 2, order (0,1), (0,2), ..., (M-2,M-1)   */
  long long n_blk;       /* floor(n_samp / L)                                  */
  int max_bin;           /* K in use                                           */
  int n_freq;            /* distinct frequencies k / N over (DM, |k| <= K),
                            f = 0 included (the factorised partial DFTs)       */
  int sub_len, n_terms;  /* Taylor evaluation: sub-block length, terms         */
  long long work_bytes;  /* device workspace                                   */
} chirp_cpi_info;

/* Creates a plan (device workspace, FP64 filter table) whose work is queued
 * on `stream` (a cudaStream_t, NULL = legacy default stream).  Errors:
 * CHIRP_EINVAL (bad size, DM <= 0, a pixel with l^2 + m^2 > 1, max_bin below
 * what the pixels need),
 * CHIRP_EUNSUPPORTED (more than 1024 sub-blocks per block would be needed),
 * CHIRP_ENOMEM, CHIRP_ECUDA.  *out is NULL on failure. */
int chirp_cpi_create(chirp_cpi_plan** out, const chirp_cpi_config* cfg, void* stream);
int chirp_cpi_query(const chirp_cpi_plan* plan, chirp_cpi_info* info);
/* Per DM d: n_win and fdot (Hz/s); pair_bins (may be NULL): [n_pair] K_pq. */
int chirp_cpi_layout(const chirp_cpi_plan* plan, int d, int* n_win, double* fdot, int* pair_bins);
/* E [n_dm][n_blk][n_pix] float (|P|^2; zero for incomplete windows) from
 * complex64 voltages [n_ant][n_samp].  volt_loc / out_loc: CHIRP_HOST or
 * CHIRP_DEVICE.  A host output synchronises the plan's stream and returns
 * CHIRP_ETIMEOUT if a bounded wait of the tensor-core image pass gave up
 * (chirp_cpi_timing reports the same). */
int chirp_cpi_run(chirp_cpi_plan* plan, const void* volt, int volt_loc, float* energy, int out_loc);
/* The intermediate spectra of the same search, both complex64
 * [n_dm][n_blk][2K+1][n_pair] (bin k at index k + K): V the partial DFTs,
 * X the window DFTs; bins beyond K_pq are zero.  Either may be NULL. */
int chirp_cpi_spectra(chirp_cpi_plan* plan, const void* volt, int volt_loc, void* V, void* X,
                      int out_loc);
/* Milliseconds of the last run's four passes (moments, partial DFTs, moving
 * sums, image), CUDA events on the plan's stream; synchronises it. */
int chirp_cpi_timing(chirp_cpi_plan* plan, double ms[4]);
void chirp_cpi_destroy(chirp_cpi_plan* plan);

/* ------------------------------------------------------------------------
 * The paper's own Chimageator pre-integrator (Sec. 4.2, App. B.2) on a
 * uniform linear array: antennas p = 0..M-1 at p * spacing_m along u, for
 * every trial DM:
 *   mixing       x_{p,p+l}[n] = y_p[n] y_{p+l}[n]^* (Eq. xpq_chimg)
 *   gridding     x'_l[n] = sum_{p<M-l} w_l x_{p,p+l}[n], l = 1..M-1, with
 *                w_l = 1/(M-l) (weights = 0, the paper's "natural") or 1
 *   spatial DFT  X_k[n] = sum_l exp(-2 pi j k l / Ns) x'_l[n], k < Ns
 *   integrate    Y_k[m] = sum_{i<L} X_k[i + mL], m < n_dump = floor(n_samp / L)
 *   trajectory   P = sum_{r<n_win} sum_{k = k0'(r)-F}^{k0'(r)+F} w Y_k[m-n_win+1+r]
 *                (Eq. chimg_pth, App. B.2.3), E = |P|^2 (Eq. eth)
 * The trial chirp and its window follow the Chirpolator pre-integrator's
 * conventions (rate a1, centre a0, n_win = max(1, floor(B T / L + 1/2))
 * dumps, the chirp's temporal midpoint at the window centre).  For direction
 * cosine l_dir (tau = spacing_m l_dir / c) the spatial tone is
 * nu(t) = tau (a0 + a1 (t - t_c)) cycles per spacing, k0'(r) = rint(Ns nu) mod Ns
 * at dump r's centre, and w = conj(Yhat) / ((M - 1) L), Yhat the expected Y
 * of a unit chirp (closed form in FP64).  Gridding, DFT and integration
 * commute: the GPU sums each dump first (FP32).
 * ---------------------------------------------------------------------- */
typedef struct chirp_chimg_plan chirp_chimg_plan;
typedef struct {
  int n_ant;             /* M, 2..32                                           */
  double spacing_m;      /* element spacing D, metres                          */
  double f0_hz, bw_hz;   /* band centre; bandwidth = complex sample rate        */
  double k_dm;           /* <= 0 selects 4.148808e15                           */
  long long n_samp;      /* samples per antenna, >= dump_len                   */
  const double* dm;      /* [n_dm] trial DMs, each > 0 (HOST)                  */
  int n_dm;
  int dump_len;          /* L                                                  */
  const double* l_dir;   /* [n_pix] direction cosines along the array (HOST)   */
  int n_pix;
  int n_spatial;         /* Ns, n_ant..1024                                    */
  int half_width;        /* F, 0..8, 2F+1 <= Ns                                */
  int weights;           /* 0: 1/(M-l), 1: 1                                   */
} chirp_chimg_config;
/* Errors: CHIRP_EINVAL (bad size, DM <= 0, |l_dir| > 1, a sweep longer than
 * the data), CHIRP_EUNSUPPORTED (2^31 or more dumps x directions),
 * CHIRP_ENOMEM, CHIRP_ECUDA; *out is NULL on failure. */
int chirp_chimg_create(chirp_chimg_plan** out, const chirp_chimg_config* cfg, void* stream);
/* n_dump, and n_win of every DM ([n_dm], may be NULL). */
int chirp_chimg_query(const chirp_chimg_plan* plan, long long* n_dump, int* n_win);
/* Y [n_dump][Ns] complex64 from complex64 voltages [n_ant][n_samp]. */
int chirp_chimg_grid(chirp_chimg_plan* plan, const void* volt, int volt_loc, void* Y, int out_loc);
/* E [n_dm][n_dump][n_pix] float; zero for incomplete windows. */
int chirp_chimg_run(chirp_chimg_plan* plan, const void* volt, int volt_loc, float* energy, int out_loc);
void chirp_chimg_destroy(chirp_chimg_plan* plan);

/* The partial-sum recursion of the imaging step (App. B.2.1): trajectories
 * of one gradient (Eq. chimg_grad) and one intercept lie on one line, and
 * every trial on it is a prefix of one cumulative sum along the line.  This
 * holds in the paper's own model of Sec. 4.2 -- natural weights, Eq.
 * chimg_xpq without its tau^2 term, a baseband chirp sweeping 0..B from the
 * window start -- where a unit chirp puts the tone nu(t) = rate t cycles per
 * spacing on the grid (rate = fdot tau, t from the window start) and every
 * trajectory starts at k = 0; it does not hold in the carrier-aware model of
 * chirp_chimg_run, whose trials of equal gradient differ in intercept.
 * For line g (rate[g], HOST [n_line]) and dump r of a window the taps are
 * the 2F+1 bins around rint(Ns rate t_r) mod Ns at the dump's centre t_r,
 * w = conj(Yhat) / ((M - 1) L) with Yhat the expected Y of the unit chirp
 * (FP64 closed form).  One cumulative sum per (line, window start s) over
 * Y (DEVICE complex64 [n_dump][Ns], as chirp_chimg_grid writes it with
 * natural weights) gives each trial t of the line, of n_t dumps,
 * energy[t][s + n_t - 1] = |P|^2 (Eq. eth); energy is DEVICE float
 * [n_trial][n_dump], zero where a window is incomplete.  Trials are given in
 * CSR form: trial_off (HOST [n_line + 1], trial_off[0] = 0) and trial_len
 * (HOST [n_trial], >= 1, ascending within a line).  Allocates and frees its
 * own device scratch and synchronises stream.  CHIRP_EINVAL for a bad shape,
 * lengths or non-device Y / energy; CHIRP_EUNSUPPORTED past 2^26 taps rows;
 * CHIRP_ENOMEM, CHIRP_ECUDA. */
int chirp_chimg_lines_run(const void* Y, long long n_dump, int n_ant, int n_spatial, int dump_len,
                          double bw_hz, int half_width, const double* rate, int n_line,
                          const int* trial_off, const int* trial_len, float* energy,
                          void* stream);

/* ------------------------------------------------------------------------
 * The same pre-integrator on a uniform RECTANGULAR array (Sec. 4.2 in two
 * dimensions, App. B.2): antenna a = iy n_x + ix at (ix dx_m, iy dy_m, 0).
 *   mixing + gridding  x'_s[n] = w_s sum_{(p,q) in s} y_p[n] y_q[n]^* over the
 *                half-plane spacings s = (lx, ly) = pos(q) - pos(p) with
 *                ly > 0, or ly = 0 and lx > 0 (ordered by ly, then lx);
 *                w_s = 1 / (pairs of s) (weights 0, "natural") or 1
 *   spatial DFT  X[kx][ky][n] = sum_s exp(-2 pi j (kx lx / Nx + ky ly / Ny)) x'_s[n]
 *   integrate    Y[m][kx][ky] = sum_{i<L} X[kx][ky][i + mL]
 *   trajectory   P = sum_{r<n_win} sum_{|jx|<=Fx, |jy|<=Fy} w Y[m-n_win+1+r][kx0+jx][ky0+jy]
 *                (indices mod Nx, Ny), (kx0, ky0) = (rint(Nx dx_m l nu / c),
 *                rint(Ny dy_m m nu / c)) at dump r's centre, nu = a0 + a1 (t - t_c),
 *                w = conj(Yhat) / (S L), Yhat the expected Y of a unit chirp
 *                from (l, m), S the number of spacings;  E = |P|^2 (Eq. eth).
 * Trial chirps and windows as in chirp_chimg_*.  The GPU forms the per-dump
 * products of every pair on the raw voltages first (FP32; the DM-independent
 * visibilities), then grids and transforms each dump.  With n_y = 1 and
 * Ny = 1 every step is the uniform linear array's.
 * ---------------------------------------------------------------------- */
typedef struct chirp_chimg2d_plan chirp_chimg2d_plan;
typedef struct {
  int n_x, n_y;          /* antennas along u and v; 2 <= n_x n_y <= 84          */
  double dx_m, dy_m;     /* element spacings, metres                           */
  double f0_hz, bw_hz;   /* band centre; bandwidth = complex sample rate        */
  double k_dm;           /* <= 0 selects 4.148808e15                           */
  long long n_samp;      /* samples per antenna, >= dump_len                   */
  const double* dm;      /* [n_dm] trial DMs, each > 0 (HOST)                  */
  int n_dm;
  int dump_len;          /* L                                                  */
  const double* pix_lm;  /* [n_pix][2] direction cosines (l, m) (HOST)         */
  int n_pix;
  int n_spatial_x;       /* Nx >= 2 n_x - 1 (n_x when n_y = 1): no two spacings
                            share a bin                                         */
  int n_spatial_y;       /* Ny >= n_y; Nx Ny <= 16384                          */
  int half_width_x;      /* Fx, 0..8, 2 Fx + 1 <= Nx                           */
  int half_width_y;      /* Fy, 0..8, 2 Fy + 1 <= Ny                           */
  int weights;           /* 0: 1 / (pairs of the spacing), 1: 1                */
} chirp_chimg2d_config;
/* Errors: CHIRP_EINVAL (bad size, a grid that aliases spacings, DM <= 0,
 * l^2 + m^2 > 1, a sweep longer than the data), CHIRP_EUNSUPPORTED,
 * CHIRP_ENOMEM, CHIRP_ECUDA; *out is NULL on failure.  Work is queued on
 * stream (a cudaStream_t, NULL = legacy default stream). */
int chirp_chimg2d_create(chirp_chimg2d_plan** out, const chirp_chimg2d_config* cfg, void* stream);
/* n_dump; n_win of every DM ([n_dm], may be NULL); the number of spacings S. */
int chirp_chimg2d_query(const chirp_chimg2d_plan* plan, long long* n_dump, int* n_win,
                        int* n_spacing);
/* Y complex64 [n_dump][Nx][Ny] from complex64 voltages [n_ant][n_samp]; a
 * host output synchronises the stream. */
int chirp_chimg2d_grid(chirp_chimg2d_plan* plan, const void* volt, int volt_loc, void* Y,
                       int out_loc);
/* E [n_dm][n_dump][n_pix] float; zero for incomplete windows. */
int chirp_chimg2d_run(chirp_chimg2d_plan* plan, const void* volt, int volt_loc, float* energy,
                      int out_loc);
void chirp_chimg2d_destroy(chirp_chimg2d_plan* plan);

/* ------------------------------------------------------------------------
 * Combination of coarse channels (post-integration, Sec. 2.1 Eq. 1 applied
 * between channel centres): a wide band searched as n_chan coarse channels
 * of equal bandwidth bw_hz and dump length (one Chimageator plan per channel,
 * each dedispersing about its own centre f_c), aligned to the top channel
 * (f_ref = max f_c) and added incoherently:
 *   E[d][m][pix] = sum_c P_c[d][m + s_c(d)][pix],
 *   s_c(d) = rint(k_dm DM_d (f_c^-2 - f_ref^-2) bw_hz / dump_len)  (FP64),
 * where every channel's dump m + s_c(d) is below n_dump and inside that
 * channel's valid dumps [first_c[d], last_c[d]]; E = 0 elsewhere.
 *  P:     HOST array of n_chan DEVICE pointers, each float32
 *         [n_dm][n_dump][n_pix] (chimageator_run's layout);
 *  first, last: HOST int64 [n_chan][n_dm] (chirp_dump_range of each plan);
 *  f_c:   HOST [n_chan] channel centres, Hz;  dm: HOST [n_dm], pc cm^-3;
 *  k_dm <= 0 selects 4.148808e15;  E: DEVICE float32 [n_dm][n_dump][n_pix].
 * Sums are FP32 in channel order.  Work is queued on stream (a cudaStream_t,
 * NULL = legacy default stream); a small stream-ordered workspace holds the
 * shifts.  Errors: CHIRP_EINVAL (NULL or bad size; n_chan above
 * CHIRP_MAX_CHANNELS), CHIRP_ENOMEM, CHIRP_ECUDA. */
#define CHIRP_MAX_CHANNELS 64
int chirp_combine_channels(const float* const* P, int n_chan, int n_dm, long long n_dump,
                           int n_pix, const long long* first, const long long* last,
                           const double* f_c, double bw_hz, int dump_len, double k_dm,
                           const double* dm, float* E, void* stream);

/* Message of the last failure on the calling thread ("" if none). */
const char* chirp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CHIRP_GB300_H */
