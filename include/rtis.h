/*
 * rtis.h -- C ABI of the eRTIS energyscape library (one GB300, sm_103a).
 *
 * The library turns one recording of the eRTIS in-air imaging sonar (32
 * microphones, int16 samples, 450 kHz) into an energyscape: an image of
 * reflector intensity over range x steering direction.  The processing chain
 * follows the paper's Fig. 3 and Sec. 4.1 (matched filter against the emitted
 * broadband FM sweep, delay-and-sum beamforming per direction of interest,
 * envelope detection with the time axis as range) and Sec. 4.3 (filters as
 * FFT convolutions with their group delay removed, subsampling after the
 * envelope, device memory allocated once per fixed configuration).
 *
 * Definitions used by every entry point (x: int16 input, s: chirp, M mics,
 * N samples per mic, D directions, L chirp samples, R decimation):
 *   F        = smallest power of two >= N + L - 1
 *   k_lo/hi  = ceil(band_lo F/fs), floor(band_hi F/fs)     (in-band FFT bins)
 *   a_m[n]   = IFFT_F( 2 FFT_F(x_m/32768) conj(FFT_F(s)) on k_lo..k_hi )[n]
 *   delta_dm = fs (Delta_m - (p_m . u_d)/c)                 (samples)
 *   TD:  b_d[n] = sum_m g_m sum_{q=-1..2} w_q(mu) a_m[j+q],  j = floor(n+delta_dm),
 *        mu = n + delta_dm - j, Catmull-Rom weights, a = 0 outside [0, N)
 *   FD:  b_d = IFFT_F( sum_m g_m exp(+2 pi i k delta_dm/F) A_m[k] )[0:N)
 *   E[d][i]  = sum_j h[j] |b_d|[R i + j - (len(h)-1)/2],  i < floor(N/R),
 *        |b| = 0 outside [0, N)
 *
 * Conventions
 *   - Pointers named d_* are DEVICE pointers owned by the caller; they must
 *     stay valid until the work queued on `stream` has finished.  Host
 *     arrays passed to rtis_plan_create are copied; the caller keeps them.
 *   - Complex arrays are interleaved (re, im) float32 pairs.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Every call except create/destroy/sync is asynchronous and
 *     stream-ordered; none synchronises the device.
 *   - No C++ exception crosses this interface.  Arguments are checked before
 *     any launch; a failing call returns a status != RTIS_OK, launches
 *     nothing, and leaves a message for rtis_last_error() (thread-local).
 *   - Device-side checks (a steering delay outside the plan's staged range,
 *     a bounded wait that ran out) never trap: they set bits in the plan's
 *     status word, which rtis_plan_sync() reads and clears.
 *   - A plan is not thread-safe: calls on one plan must not overlap on
 *     different streams, because they share the plan's workspaces.
 */
#ifndef RTIS_H
#define RTIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rtis_plan rtis_plan;

typedef enum rtis_status {
    RTIS_OK = 0,
    RTIS_ERR_INVALID_ARG = 1,   /* null pointer, bad size, misaligned pointer */
    RTIS_ERR_CUDA = 2,          /* a CUDA runtime call failed (message says which) */
    RTIS_ERR_OOM = 3,           /* device allocation failed in rtis_plan_create */
    RTIS_ERR_UNSUPPORTED = 4,   /* valid request outside what this build implements */
    RTIS_ERR_TIMEOUT = 5,       /* a bounded device wait ran out (status word) */
    RTIS_ERR_NONFINITE = 6,     /* non-finite geometry, chirp or taps */
    RTIS_ERR_DEVICE = 7,        /* a device-side range check failed (status word) */
    RTIS_ERR_BUSY = 8           /* no free slot (rtis_stream_submit) */
} rtis_status;

/* Device status-word bits reported by rtis_plan_sync(). */
#define RTIS_DEV_DELAY_RANGE 0x1u   /* |floor(delta)| beyond the plan's staged halo */
#define RTIS_DEV_TIMEOUT     0x2u   /* a bounded mbarrier wait ran out */
#define RTIS_DEV_NONFINITE   0x4u   /* an energyscape value came out NaN or infinite */

/*
 * Host-side fault injection (testing the error paths; nothing faults the GPU).
 * The environment variable RTIS_FAULT, read at each call, selects:
 *   "alloc"   -- rtis_plan_create, rtis_batch_create and rtis_fd_gemm_create
 *                fail with RTIS_ERR_OOM before allocating anything;
 *   "launch"  -- the entry points that launch kernels fail with RTIS_ERR_CUDA
 *                before launching anything;
 *   "stall"   -- the time-domain beamformer withholds the first TMA copy of
 *                each CTA and waits for it with a short bound (thousands of
 *                polls): every CTA gives up, sets RTIS_DEV_TIMEOUT, lets its
 *                other copies land and returns; the next sync reports
 *                RTIS_ERR_TIMEOUT and the context stays usable.
 */

enum { RTIS_PATH_TD = 0, RTIS_PATH_FD = 1, RTIS_PATH_BB = 2 };
enum { RTIS_PREC_FP32 = 0, RTIS_PREC_BF16 = 1, RTIS_PREC_FP16 = 2 };

typedef struct rtis_options {
    double c;                    /* speed of sound, m/s (default 343) */
    int decim;                   /* R, envelope subsampling factor (default 10) */
    int lpf_len;                 /* odd number of envelope low-pass taps; 0 -> 4R+1 */
    const float* lpf_taps;       /* host [lpf_len]; NULL -> sinc(t/R) x Hann, sum 1 */
    double band_lo_hz;           /* matched-filter band (default 20e3) */
    double band_hi_hz;           /* (default 80e3) */
    int path;                    /* RTIS_PATH_TD (default), RTIS_PATH_FD or RTIS_PATH_BB */
    int precision;               /* storage of the analytic signal a on the TD path:
                                    RTIS_PREC_FP32 (default) or RTIS_PREC_BF16 (a rounded
                                    to BF16 pairs, half the staged bytes; products and sums
                                    stay FP32).  The FD path takes FP32 only. */
    double max_delay_s;          /* bound on |Delta_m| set by calibration (default 10e-6) */
    double position_slack_m;     /* bound on calibrated mic displacement (default 0.01) */
    int max_batch;               /* most measurements one rtis_process_many call takes through
                                    the batched FD GEMM (0: none, <= 64); sizes its buffers */
    int td_layout;               /* time-domain beamformer stage layout: 0 = autotune at creation
                                    (default), k = layout k-1 of rtis_plan_info.td_layout_ms */
    int bb_layout;               /* the same for the baseband beamformer (RTIS_PATH_BB) */
    int grid_mode;               /* with a forced layout: 0 or 1 = one CTA per tile, 2 = the CTAs
                                    resident at once looping over the tiles.  Every layout and grid
                                    gives the same results bit for bit (only the staging differs) */
    int fd_ifft;                 /* inverse transform of rtis_process_many's frequency-domain path:
                                    RTIS_FD_IFFT_AUTO (default: the faster form as measured on
                                    GB300, today the FFT), RTIS_FD_IFFT_FFT (radix-16/32 FFTs
                                    on the FP32 pipe), RTIS_FD_IFFT_TC (two dense DFT stages on the
                                    tcgen05 tensor cores in FP32 as three BF16 products; needs
                                    F = 32768, at most 4608 in-band bins and a low-pass of at most
                                    127 taps, else rtis_plan_create returns RTIS_ERR_UNSUPPORTED) */
} rtis_options;

#define RTIS_FD_IFFT_AUTO 0
#define RTIS_FD_IFFT_FFT 1
#define RTIS_FD_IFFT_TC 2

/* Fills *opt with the defaults listed above. */
void rtis_options_default(rtis_options* opt);

typedef struct rtis_plan_info {
    int n_mics, n_samples, n_dirs, chirp_len;
    int fft_len;                 /* F */
    int k_lo, k_hi;              /* in-band bins */
    int decim, lpf_len, n_out;   /* n_out = floor(N/R): energyscape row length */
    int halo;                    /* staged samples each side of a TD tile */
    int max_shift;               /* largest |floor(delta)| the TD kernel accepts */
    size_t workspace_bytes;      /* device memory the plan holds */
    int td_variant;              /* time-domain beamformer stage layout chosen at creation */
    int td_grid;                 /* and its grid (CTAs) */
    float td_tuned_ms;           /* its time on this device when tuned */
    int n_coarse;                /* RTIS_PATH_BB: n_samples/4 coarse samples per channel (else 0) */
    int k_c;                     /* RTIS_PATH_BB: demodulation bin floor((k_lo + k_hi)/2) (else 0) */
    int bb_variant;              /* RTIS_PATH_BB: baseband beamformer stage layout chosen at creation */
    int bb_grid;                 /* and its grid (CTAs) */
    float bb_tuned_ms;           /* its time on this device when tuned */
    float td_layout_ms[16];      /* the time-domain autotuner's measurements: mean ms of layout v with
                                    one CTA per tile at [2v], with the resident persistent grid at
                                    [2v + 1]; 0 where not tried */
    float bb_layout_ms[16];      /* the same for the baseband beamformer (RTIS_PATH_BB) */
    int fd_ifft;                 /* the inverse transform rtis_process_many's frequency-domain path
                                    runs: RTIS_FD_IFFT_FFT or RTIS_FD_IFFT_TC (0 without max_batch) */
} rtis_plan_info;

/*
 * rtis_plan_create -- validate the configuration and allocate, once, every
 * device buffer the chain needs (Sec. 4.3: preallocation for fixed sizes).
 *   mic_xyz     host float [n_mics][3], metres, array frame (faces +z)
 *   fs          sampling rate, Hz (> 0)
 *   chirp       host float [chirp_len], the emitted sweep s[n]
 *   directions  host float [n_dirs][3], unit steering vectors
 *   n_samples   N, samples per channel; a multiple of 4, 64 <= N <= 65536
 *   opt         NULL -> defaults
 * Limits: 1 <= n_mics <= 32; 1 <= n_dirs; chirp_len >= 1; the in-band bins
 * must number at most F/4 and lie below F/4.  On success *out owns the plan
 * (free with rtis_plan_destroy); on failure *out is NULL.  Synchronises the
 * device (table upload) and autotunes the time-domain beamformer's stage
 * layout and grid by timing the candidates on the plan's zeroed workspace
 * (a few ms).
 */
rtis_status rtis_plan_create(rtis_plan** out, const float* mic_xyz, int n_mics, double fs,
                             const float* chirp, int chirp_len, const float* directions,
                             int n_dirs, int n_samples, const rtis_options* opt);

/* Frees the plan and its device memory (synchronises the device). NULL is a no-op. */
void rtis_plan_destroy(rtis_plan* plan);

/* Sizes derived at creation. */
rtis_status rtis_plan_get_info(const rtis_plan* plan, rtis_plan_info* info);

/*
 * rtis_process -- whole chain for one recording (Fig. 3): matched filter,
 * delay-and-sum on the plan's path, envelope, low-pass, subsample.
 *   RTIS_PATH_TD  Catmull-Rom fractional delays on the full-rate analytic signal.
 *   RTIS_PATH_FD  exact phase ramps on the in-band spectrum; needs F <= 65536 with
 *                 its spectrum, FFT buffer and outputs in shared memory (N up to
 *                 about 46000 at R = 10; larger N: RTIS_ERR_UNSUPPORTED).
 *   RTIS_PATH_BB  complex baseband: the paper subsamples before its filters
 *                 (Sec. 4.3); this path subsamples after the matched filter.
 *                 The analytic signal, demodulated by the mid-band bin
 *                 k_c = floor((k_lo + k_hi)/2), is kept at every 4th sample:
 *                 z_m[j] = a_m[4j] e^{-2 pi i k_c 4j/F}.  The beam is formed on
 *                 that grid, b_d[j] = sum_m g_m e^{+2 pi i k_c delta_dm/F}
 *                 I(z_m, j + delta_dm/4) with I the Catmull-Rom interpolation.
 *                 The result is E[d][i] = sum_j h_i(4j - R i) |b_d[j]|, with h_i
 *                 the plan's low-pass taps at those offsets, renormalised to
 *                 sum 1.  It approximates the TD/FD energyscape to about 1e-2 of
 *                 its peak, at 2.7x fewer multiply-adds.
 * With opt.precision = RTIS_PREC_BF16 the TD path beamforms from a BF16 copy
 * of a (relative error ~2^-9 per sample; energyscape within 1e-2 of the peak).
 *   d_in   device int16 [n_mics][n_samples], 8-byte aligned
 *   d_out  device float [n_dirs][n_out]
 */
rtis_status rtis_process(rtis_plan* plan, const int16_t* d_in, float* d_out, void* stream);

/*
 * rtis_process_many -- the whole chain for n measurements of the plan's
 * geometry, d_in [n][n_mics][n_samples], one matched filter per measurement
 * feeding either or both delay-and-sum forms:
 *   d_out_td  [n][n_dirs][n_out]: time-domain energyscapes (or NULL);
 *   d_out_fd  [n][n_dirs][n_out]: frequency-domain energyscapes (or NULL;
 *             needs n <= opt.max_batch and F <= 65536).
 * The frequency-domain delay-and-sum of all n runs as ONE batched complex
 * GEMM on the tensor cores (the phase-ramp form of Fig. 3 / Sec. 4.1 with the
 * measurements as frames: Y[d][k][t] = sum_m g_m e^{+2 pi i k delta_dm/F} A_m^t[k],
 * FP32 operands as three BF16 products), followed by the per-direction phase
 * IFFTs, envelope, low-pass and subsampling of each measurement.  Results
 * match rtis_process to the FP32 energyscape tolerance.
 *   d_in   device int16, 8-byte aligned
 */
rtis_status rtis_process_many(rtis_plan* plan, const int16_t* d_in, int n, float* d_out_td, float* d_out_fd,
                              void* stream);

/*
 * rtis_matched_filter -- the matched-filter stage alone (Sec. 4.1/4.3).
 *   d_in   device int16 [n_mics][n_samples]
 *   d_a    device complex float [n_mics][n_samples]: a_m[n] as defined above
 * d_a may be NULL when only the band spectrum is wanted.
 *   d_A    device complex float [n_mics][k_hi-k_lo+1]: A_m[k] = 2 X_m[k] conj(S[k])/F
 *          (already divided by F; NULL to skip)
 */
rtis_status rtis_matched_filter(rtis_plan* plan, const int16_t* d_in, float* d_a, float* d_A,
                                void* stream);

/*
 * rtis_beamform_td -- time-domain delay-and-sum with the fused envelope,
 * low-pass and subsampling epilogue, from a matched-filter output (always
 * complex float, whatever opt.precision).
 *   d_a    device complex float [n_mics][n_samples], 16-byte aligned
 *   d_out  device float [n_dirs][n_out]
 */
rtis_status rtis_beamform_td(rtis_plan* plan, const float* d_a, float* d_out, void* stream);

/*
 * rtis_beamform_fd -- frequency-domain delay-and-sum with the envelope,
 * low-pass and subsampling, from the in-band matched-filter spectra
 * (rtis_matched_filter's d_A).  Needs F <= 65536 (as RTIS_PATH_FD).
 *   d_A    device complex float [n_mics][k_hi-k_lo+1], 8-byte aligned
 *   d_out  device float [n_dirs][n_out]
 */
rtis_status rtis_beamform_fd(rtis_plan* plan, const float* d_A, float* d_out, void* stream);

/*
 * rtis_baseband_signal -- the matched filter of a RTIS_PATH_BB plan, ending in
 * the demodulated analytic signal on the coarse grid (see rtis_process):
 *   d_in   device int16 [n_mics][n_samples], 8-byte aligned
 *   d_z    device complex float [n_mics][n_samples/4], 8-byte aligned:
 *          z_m[j] = a_m[4j] e^{-2 pi i k_c 4j/F}, k_c = floor((k_lo + k_hi)/2)
 * RTIS_ERR_UNSUPPORTED on a plan of another path.
 */
rtis_status rtis_baseband_signal(rtis_plan* plan, const int16_t* d_in, float* d_z, void* stream);

/*
 * rtis_beamform_bb -- the baseband delay-and-sum with the fused envelope and
 * coarse-grid low-pass of a RTIS_PATH_BB plan, from rtis_baseband_signal's z.
 *   d_z    device complex float [n_mics][n_samples/4], 16-byte aligned;
 *          n_samples/4 must be even (16-byte rows) -- else RTIS_ERR_UNSUPPORTED
 *          (rtis_process has no such limit)
 *   d_out  device float [n_dirs][n_out]
 */
rtis_status rtis_beamform_bb(rtis_plan* plan, const float* d_z, float* d_out, void* stream);

/*
 * rtis_steering_table -- the plan's per-(direction, mic) fractional-delay
 * table, computed on the device in FP64 from the current geometry:
 *   d_shift   device int32 [n_dirs][n_mics]  floor(delta_dm)
 *   d_weight  device float [n_dirs][n_mics][4]  g_m w_q(mu), q = -1..2
 */
rtis_status rtis_steering_table(rtis_plan* plan, int32_t* d_shift, float* d_weight, void* stream);

/*
 * rtis_set_calibration -- replaces the array calibration the plan steers
 * with (positions p_m, gains g_m, per-mic delays Delta_m in seconds); each
 * pointer is a device array ([n_mics][3], [n_mics], [n_mics]) or NULL to
 * keep the current values (initially: the create-time positions, gains 1,
 * delays 0).  Stream-ordered; the steering tables are rebuilt on `stream`.
 * Delays beyond opt.max_delay_s or positions moved by more than
 * opt.position_slack_m can exceed the staged halo: the affected entries
 * then contribute nothing and rtis_plan_sync reports RTIS_ERR_DEVICE.
 */
rtis_status rtis_set_calibration(rtis_plan* plan, const float* d_mic_xyz, const float* d_gain,
                                 const float* d_delay_s, void* stream);

/*
 * rtis_backward -- reverse pass of the time-domain energyscape with respect
 * to the calibration (not in the paper, which has no gradient): given the
 * cotangent G = dL/dE it returns
 *   d_grad_xyz [n_mics][3] = dL/dp_m,  d_grad_gain [n_mics] = dL/dg_m,
 *   d_grad_delay [n_mics] = dL/dDelta_m (per second)
 * (any of them may be NULL).  With t = n + delta_dm and Catmull-Rom value
 * and slope weights: dL/d delta_dm = g_m sum_n Re(conj(G_b) I'), where
 * G_b = (transposed low-pass of G) * b / |b| (0 where b = 0).  The matched
 * filter and the beams are recomputed from d_in; nothing per direction is
 * stored.  Reductions run in a fixed order (deterministic).
 *   d_in        device int16 [n_mics][n_samples]
 *   d_grad_out  device float [n_dirs][n_out]
 */
rtis_status rtis_backward(rtis_plan* plan, const int16_t* d_in, const float* d_grad_out, float* d_grad_xyz,
                          float* d_grad_gain, float* d_grad_delay, void* stream);

/*
 * rtis_loss_l2 -- the self-calibration objective (not in the paper): with E
 * the energyscape of a recording and E_ref that of the known scene,
 *   *d_loss = sum_{d,i} (E[d][i] - E_ref[d][i])^2,  d_grad_out = 2 (E - E_ref)
 * (d_grad_out may be NULL).  d_E, d_E_ref, d_grad_out: device float
 * [n_dirs][n_out]; d_loss: one device float.  The sum runs in a fixed order
 * (deterministic).  Uses the plan's adjoint scratch: do not overlap with
 * rtis_backward on another stream.
 */
rtis_status rtis_loss_l2(rtis_plan* plan, const float* d_E, const float* d_E_ref, float* d_grad_out, float* d_loss,
                         void* stream);

/*
 * rtis_plan_sync -- waits for the device, then reads and clears the plan's
 * device status word.  Returns RTIS_ERR_DEVICE / RTIS_ERR_TIMEOUT if a
 * device-side check fired since the last sync (bits in *bits if non-NULL).
 */
rtis_status rtis_plan_sync(rtis_plan* plan, unsigned* bits);

/*
 * Many sensors at once (the paper's multi-sensor network, Sec. 3; several
 * sensors on one GPU, Sec. 5): plans with their own geometry, record length
 * and direction set, processed on the time-domain path.  Every sensor's
 * matched filter runs, then ONE persistent beamformer launch walks the tiles
 * of all sensors (at most 16 plans per batch).
 *
 * rtis_process_batch -- plain launches on `stream`; allocates nothing.
 *   plans  [n] plans (not owned); d_in [n] device int16 [M_s][N_s];
 *   d_out [n] device float [D_s][n_out_s].
 *   Device-side checks report into plans[0]'s status word.
 *
 * rtis_batch_create / rtis_batch_run / rtis_batch_destroy -- a reusable
 * batch.  The first run autotunes the beamformer (every stage layout of
 * rtis_plan_info.td_layout_ms that fits x two grids: one persistent CTA per
 * SM, or one CTA per tile, each timed on the real inputs; the outputs are
 * written several times); every run replays the batch as a CUDA graph on an
 * internal stream, ordered after and before `stream` with events.  A new set
 * of input/output pointers re-captures the graph.  The plans must outlive
 * the batch; rtis_batch_sync waits for it and reads its status word.
 */
typedef struct rtis_batch rtis_batch;
typedef struct rtis_batch_info {
    int n_sensors, total_tiles;
    int tuned;        /* 1 once the first run has autotuned */
    int variant;      /* beamformer stage layout v, timed at rtis_plan_info.td_layout_ms[2v] */
    int grid;         /* beamformer CTAs */
    float tuned_ms;   /* beamformer time of the chosen candidate */
} rtis_batch_info;
rtis_status rtis_process_batch(rtis_plan* const* plans, int n, const int16_t* const* d_in, float* const* d_out,
                               void* stream);
rtis_status rtis_batch_create(rtis_batch** out, rtis_plan* const* plans, int n);
rtis_status rtis_batch_run(rtis_batch* b, const int16_t* const* d_in, float* const* d_out, void* stream);
rtis_status rtis_batch_get_info(const rtis_batch* b, rtis_batch_info* info);
rtis_status rtis_batch_sync(rtis_batch* b, unsigned* bits);
void rtis_batch_destroy(rtis_batch* b);

/*
 * Frequency-domain delay-and-sum as a batched complex GEMM (the phase-ramp
 * form of the paper's delay-and-sum, Fig. 3 / Sec. 4.1, evaluated per
 * frequency), on the tcgen05 tensor cores:
 *
 *   Y[k][d][t] = sum_m W[k][d][m] X[k][m][t],
 *   W[k][d][m] = g_m exp(+2 pi i f_k tau_dm),  tau_dm = Delta_m - (p_m . u_d)/c
 *
 * The steering matrix W is generated on the device (phase in compensated
 * FP32) and never stored.  precision: RTIS_PREC_BF16 or RTIS_PREC_FP16
 * operands with FP32 accumulation and per-channel power-of-two scaling, or
 * RTIS_PREC_FP32 (three BF16 products hi.hi + hi.lo + lo.hi).
 *
 * rtis_fd_gemm_create
 *   mic_xyz    host float [n_mics][3] (n_mics <= 32), directions host float [n_dirs][3]
 *   freqs_hz   host double [n_bins], bin frequencies f_k
 *   n_frames   T, 1 <= T <= 64
 *   gain, delay_s  host float [n_mics] or NULL (1 and 0)
 * rtis_fd_gemm_run
 *   d_X  device complex float [n_bins][n_mics][n_frames], 8-byte aligned
 *   d_Y  device complex float [n_bins][n_dirs][n_frames], 16-byte aligned
 */
typedef struct rtis_fd_gemm rtis_fd_gemm;
rtis_status rtis_fd_gemm_create(rtis_fd_gemm** out, const float* mic_xyz, int n_mics, const float* directions,
                                int n_dirs, const double* freqs_hz, int n_bins, int n_frames, double c,
                                const float* gain, const float* delay_s, int precision);
rtis_status rtis_fd_gemm_run(rtis_fd_gemm* g, const float* d_X, float* d_Y, void* stream);
void rtis_fd_gemm_destroy(rtis_fd_gemm* g);

/*
 * Streaming service: the paper's sensor-to-processor queue (Sec. 3:
 * measurements arrive at a fixed rate and are turned into images as they come)
 * as a ring of `depth` pinned host slots around one plan.
 *   rtis_stream_submit -- copies host_in (int16 [M][N], host memory, free again on
 *                         return) into the next slot and queues its input copy,
 *                         rtis_process and the copy of the energyscape (float
 *                         [D][n_out]) into host_out; returns the ticket.  host_out
 *                         must stay valid until the ticket is collected; page-locked
 *                         memory keeps its copy asynchronous.  RTIS_ERR_BUSY when
 *                         that slot's previous ticket has not been collected
 *                         (collect tickets in submission order).
 *   rtis_stream_wait   -- waits at most timeout_ms until `ticket`'s energyscape is
 *                         in its host_out, then frees the slot; RTIS_ERR_TIMEOUT if
 *                         not ready (the ticket stays valid).
 * Input and result copies run on per-slot streams, the chain on one compute
 * stream, so copies overlap other measurements' processing.  rtis_stream_create
 * captures each slot's chain (the plan's path) into a CUDA graph that submit
 * replays; the graphs read the plan's steering tables in place, so
 * rtis_set_calibration between measurements takes effect.  While tickets are
 * outstanding the plan's workspaces belong to the service: do not run the plan
 * on another stream then.  Calls on one stream object are serialised
 * internally.
 */
typedef struct rtis_stream rtis_stream;
rtis_status rtis_stream_create(rtis_stream** out, rtis_plan* plan, int depth);
rtis_status rtis_stream_submit(rtis_stream* s, const int16_t* host_in, float* host_out, int64_t* ticket);
rtis_status rtis_stream_wait(rtis_stream* s, int64_t ticket, int timeout_ms);
void rtis_stream_destroy(rtis_stream* s);

/*
 * Comparison baseline (not the product path): the time-domain chain built the
 * way the paper's GPU implementation is described (Sec. 4.3) -- cuFFT
 * convolutions for the matched filter, one thread per (direction, sample) for
 * the delay-and-sum with the beam's envelope in device memory, then a separate
 * low-pass/subsample kernel.  Same definitions and plan tables as
 * rtis_process on the time-domain path; results agree to FP32 rounding.
 *   rtis_baseline_create   -- cuFFT plans and work buffers for `plan`
 *                             (M F floats, M (F/2+1) + M F complex, D N floats)
 *   rtis_baseline_process  -- d_in int16 [M][N] -> d_out float [D][n_out]; the
 *                             plan must have run once (its steering table)
 */
typedef struct rtis_baseline rtis_baseline;
rtis_status rtis_baseline_create(rtis_baseline** out, const rtis_plan* plan);
rtis_status rtis_baseline_process(rtis_baseline* b, const int16_t* d_in, float* d_out, void* stream);
void rtis_baseline_destroy(rtis_baseline* b);

/*
 * rtis_pdm_demodulate -- the PDM front end: the microphones record through a
 * 1-bit sigma-delta ADC (Sec. 2) and the bits are unpacked and low-pass
 * filtered before the matched filter (Sec. 4.3).  Produces the int16 PCM
 * recording that rtis_process takes:
 *   b_m[k] = +1 for bit m of word k set, -1 for clear, 0 for k outside [0, n_words)
 *   x_m[n] = sat16((sum_j g[j] b_m[decim n + j - c] + r) >> shift),
 *            c = (n_taps - 1)/2, r = 2^(shift-1) for shift > 0 (halves round up)
 * The arithmetic is integer, so the result is exact.
 *   d_words  device uint32 [n_words], one word per bit-clock tick, bit m = mic m
 *            (4-byte aligned; bits above n_mics are ignored)
 *   taps     host int32 [n_taps], n_taps <= 256, sum |g| <= 2^30; or NULL for the
 *            order-4 CIC kernel (the length-decim boxcar convolved 4 times, sum
 *            decim^4: 10^4 at decim = 10, so no shift is needed)
 *   decim    bit ticks per output sample, 1..64 (10: 4.5 MHz bits -> 450 kHz)
 *   shift    right shift 0..30
 *   d_x      device int16 [n_mics][n_samples], 2-byte aligned
 * Stream-ordered; needs no plan and allocates nothing.
 */
rtis_status rtis_pdm_demodulate(const uint32_t* d_words, long long n_words, int n_mics, int n_samples, int decim,
                                const int32_t* taps, int n_taps, int shift, int16_t* d_x, void* stream);

/*
 * rtis_matched_filter_noalloc -- the matched filter of rtis_matched_filter
 * for callers that may not allocate device memory: code that runs where
 * cudaMalloc is not allowed or not wanted (a real-time loop that must never
 * block in the allocator, a host framework that owns all device memory and
 * only lends buffers, a process without a plan created beforehand).  The
 * paper has no counterpart; it allocates once per configuration instead.
 *
 * Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 * The twiddle table, the chirp spectrum and the half-size spectra live in
 * one static device array of RTIS_NOALLOC_SCRATCH_BYTES, which every GPU
 * that loads this library holds until the process exits.  The first call on
 * a device looks up that array's device address (cudaGetSymbolAddress, with
 * that device current) and keeps it for that device's context; make that
 * first call before any stream capture.  A call after cudaDeviceReset sees a
 * new context and looks the address up again (again a first call).
 * All calls share the array and it keeps the last call's contents (each call
 * rewrites everything it reads), so calls whose work overlaps on the GPU --
 * on different streams, or from different threads -- race and corrupt each
 * other's results: serialise them.
 *   d_in       device int16 [n_mics][n_samples], 8-byte aligned
 *   d_chirp    device float [chirp_len], the emitted sweep
 *   band_*_hz  matched-filter band (the plan default is 20e3 .. 80e3)
 *   d_a        device complex float [n_mics][n_samples] (or NULL), as rtis_matched_filter
 *   d_A        device complex float [n_mics][k_hi-k_lo+1] (or NULL), as rtis_matched_filter
 * Sizes needing more than RTIS_NOALLOC_SCRATCH_BYTES
 * (8 F + 8 ceil256(K_b) + 16 n_mics F/4 bytes, F = nextpow2(N + L - 1)) are
 * rejected with RTIS_ERR_INVALID_ARG before anything is launched; 32 mics
 * with N + L - 1 <= 32768 fit.
 */
#define RTIS_NOALLOC_SCRATCH_BYTES (8u << 20)
rtis_status rtis_matched_filter_noalloc(const int16_t* d_in, int n_mics, int n_samples, const float* d_chirp,
                                        int chirp_len, double fs, double band_lo_hz, double band_hi_hz,
                                        float* d_a, float* d_A, void* stream);

/*
 * Kernel tracing (CUDA-event timing of the library's own launches).
 * rtis_plan_set_tracing(plan, 1) creates RTIS_TRACE_MAX pairs of CUDA events
 * (once; 0 destroys them).  While tracing is on, every call on the plan that
 * launches kernels (rtis_process, rtis_process_many, rtis_matched_filter,
 * rtis_beamform_td, rtis_beamform_fd, rtis_beamform_bb, rtis_backward,
 * rtis_set_calibration, and the steering-table refresh they may trigger) starts
 * a new list and records an
 * event pair around each of its kernel launches on the caller's stream, in
 * launch order.  Calls on a stream that is being captured are not traced.
 * rtis_plan_get_trace waits for the last traced call's final event and copies
 * up to `capacity` entries {kernel id, launch index in the call, milliseconds};
 * *n_out is the number of entries recorded (a call with more than
 * RTIS_TRACE_MAX launches keeps the first RTIS_TRACE_MAX).  Errors:
 * RTIS_ERR_INVALID_ARG (NULL plan, or get_trace while tracing is off),
 * RTIS_ERR_CUDA (event creation or timing failed).
 */
#define RTIS_TRACE_MAX 32
typedef enum {
    RTIS_KERNEL_STEERING_TABLE = 1,
    RTIS_KERNEL_MF_FORWARD = 2,
    RTIS_KERNEL_MF_INVERSE = 3,
    RTIS_KERNEL_TD_BEAMFORM = 4,
    RTIS_KERNEL_FD_GEMM = 5,           /* the per-channel |X| maxima and the tcgen05 GEMM */
    RTIS_KERNEL_FD_ENERGYSCAPE = 6,
    RTIS_KERNEL_BB_BEAMFORM = 7,
    RTIS_KERNEL_ADJOINT = 8            /* the adjoint and its two reductions */
} rtis_kernel_id;
typedef struct rtis_trace_entry {
    int kernel;                  /* rtis_kernel_id */
    int index;                   /* position among the call's launches */
    float ms;                    /* CUDA-event time of the launch */
} rtis_trace_entry;
rtis_status rtis_plan_set_tracing(rtis_plan* plan, int enable);
rtis_status rtis_plan_get_trace(rtis_plan* plan, rtis_trace_entry* out, int capacity, int* n_out);

const char* rtis_status_string(rtis_status s);
const char* rtis_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RTIS_H */
