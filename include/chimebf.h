/*
 * chimebf.h -- C ABI of the GB300 CHIME/FRB fan-beam library (arXiv 1702.04728).
 *
 * One coarse frequency channel carries 4+4-bit complex voltages from 2048
 * inputs (4 cylinders x 256 feeds x 2 polarisations; Sec. 2, Table 1).  The
 * library turns them into Stokes-I intensity for 1024 beams (256 N-S x 4 E-W)
 * at 16 sub-channels x one frame per 384 samples (Sec. 3, Table 1):
 *
 *   1. N-S beams: 2x zero-padded 512-point FFT of each 256-feed line, kept at
 *      the 256 bins of the clamp table of Eq. (1) (Sec. 3.1);
 *   2. 4 E-W beams by exact phasing across the cylinders (Sec. 3);
 *   3. up-channelisation by a 128-point FFT over time (Sec. 3.2);
 *   4. |.|^2 summed over polarisation (Sec. 3);
 *   5. sums over 8 fine channels x 3 blocks (24 kHz, 0.983 ms; Sec. 3, Table 1).
 *
 * Data layouts (all row-major, C order):
 *   input  uint8 [n_chan][n_samples][2048]; byte (cyl*256 + feed)*2 + pol;
 *          high nibble = real + 8, low nibble = imaginary + 8.
 *   output float [1024][16*n_chan][n_frames]; beam = 256*ew + ns,
 *          sub-channel = 16*chan + s with s = 0 the lowest frequency.
 *
 * Error behaviour: every call returns an int status; negative values are
 * errors, no call aborts the process, and bf_last_error() gives a message for
 * the calling thread's last failure.
 */
#ifndef CHIMEBF_H
#define CHIMEBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BF_OK          0
#define BF_PENDING     1   /* bf_poll: not finished within the timeout              */
#define BF_EQUEUED     2   /* bf_submit: accepted, waiting for memory or a slot     */
#define BF_EINVAL     -1   /* bad argument or unsupported geometry                  */
#define BF_ENOMEM     -2   /* request larger than the plan's whole memory budget    */
#define BF_ECUDA      -3   /* a CUDA call failed (message in bf_last_error)         */
#define BF_ETIMEDOUT  -4   /* a bounded device-side wait expired                    */
#define BF_ENOTICKET  -5   /* unknown, already collected or cancelled ticket        */
#define BF_ESHUTDOWN  -6   /* plan is being destroyed                               */

/* N-S transform forms (bf_config.form).  The BF_TC_DFT256* forms evaluate the
 * clamped zero-padded FFT (Sec. 3.1, Eq. 1) as the equivalent DFT over the 256
 * kept rows on tcgen05 (FP16 operands, FP32 accumulation); the E-W phased feed
 * line is split into FP16 hi + lo, the twiddles are FP16 hi (+ lo).
 * BF_TC_DFT512 evaluates all 512 rows of the zero-padded transform (the 512
 * redundant beams of Sec. 3.1) with one GEMM term and applies the clamp to the
 * result: the same output as BF_TC_DFT256_X1 at twice the GEMM and
 * up-channelisation work.  Its plans refuse the stage dumps and the stall
 * check (BF_EINVAL). */
#define BF_FP32_FFT      0 /* FP32 zero-padded FFT on the CUDA cores                */
#define BF_TC_DFT256     1 /* 3 GEMM terms: twiddles hi+lo x data hi+lo             */
#define BF_TC_DFT512     2 /* all 512 padded rows, 1 GEMM term, clamp at the output */
#define BF_TC_DFT256_X2  3 /* 2 GEMM terms: twiddles hi x data hi+lo                */
#define BF_TC_DFT256_X1  4 /* 1 GEMM term: twiddles hi x data hi                    */

/* execution modes (bf_config.mode) */
#define BF_MODE_DIRECT   0 /* bf_submit launches at once on cuda_stream             */
#define BF_MODE_SERVING  1 /* a plan thread batches queued requests into launches   */

/* request flags */
#define BF_END_OF_STREAM 1 /* drop the stream's leftover samples after this request */

typedef struct bf_plan_s* bf_plan_t;

/*
 * Plan configuration.  Geometry follows Sec. 1 (4 cylinders, 256 feeds at
 * 0.3048 m, dual polarisation), Sec. 3.1 (padding P = 2), Sec. 3 (4 E-W
 * beams) and Sec. 3.2 / Table 1 (128-point up-channelisation, 16 output
 * sub-channels, 0.983 ms = 3 blocks of 128 samples).  The kernels are built
 * for exactly this geometry; other integer values return BF_EINVAL.  The
 * spacings and pointings are free (Sec. 3.1: the N-S tiling is tunable).
 */
typedef struct {
    int n_cyl;              /* 4   */
    int n_feed;             /* 256 */
    int n_pol;              /* 2   */
    int pad;                /* 2   */
    int n_ew;               /* 4   */
    int upchan;             /* 128 */
    int f_ds;               /* 8   */
    int t_ds;               /* 3   */
    double feed_spacing_m;  /* N-S feed spacing d, 0.3048                         */
    double cyl_spacing_m;   /* E-W cylinder spacing, 20.0                         */
    double dt_s;            /* sample cadence, 2.56e-6 (bookkeeping only)         */
    const double* ns_sin;   /* host [n_feed] sin(theta_m) of the N-S pointings, or
                               NULL for (m - 127.5)/128; copied by bf_plan        */
    const double* ew_sin;   /* host [n_ew] sin of the E-W beam angles, or NULL for
                               sin({-0.6, -0.2, 0.2, 0.6} deg); copied            */
    int form;               /* BF_FP32_FFT, a BF_TC_DFT256* form or BF_TC_DFT512  */
    int mode;               /* BF_MODE_DIRECT | BF_MODE_SERVING                   */
    size_t mem_budget;      /* serving admission budget in bytes (0 = unlimited)  */
    int max_streams;        /* distinct stream_ids held at once (0 = 1024)        */
    void* cuda_stream;      /* cudaStream_t for the launches, or NULL: the plan
                               creates its own non-blocking stream                */
    int device;             /* CUDA device ordinal, or -1 for the current device  */
    int max_tables;         /* per-frequency table slots (clamp table, E-W phases,
                               tensor-core twiddle image) held at once, 0 = 4096
                               (the largest); a new frequency reuses the least
                               recently used slot that no open stream and no
                               running batch references, else BF_ENOMEM          */
} bf_config;

/* Fill *cfg with the CHIME defaults above.  Returns BF_OK or BF_EINVAL. */
int bf_config_default(bf_config* cfg);

/*
 * Create a plan: validates cfg, precomputes in FP64 the twiddle tables and
 * allocates device memory for per-frequency tables (clamp table of Eq. (1)
 * and E-W phases, filled lazily per channel frequency) and stream carry state.
 * On success *out owns everything and must be released with bf_destroy.
 */
int bf_plan(const bf_config* cfg, bf_plan_t* out);

/*
 * One request: n_samples new samples of n_chan channels of stream stream_id.
 * vin   device pointer, uint8 [n_chan][n_samples][2048], caller-owned.
 * out   device pointer, float [1024][16*n_chan][n_frames_out], caller-owned,
 *       n_frames_out = floor((carry + n_samples) / 384) where carry (< 384) is
 *       the number of samples the stream left over from earlier requests.
 * chan_freq_hz  host [n_chan] coarse-channel centre frequencies (they select
 *       the clamp table of Eq. (1) and the E-W phases); a stream keeps the
 *       frequencies of its first request.
 * Both buffers must stay valid until bf_poll returns BF_OK for the ticket.
 */
typedef struct {
    uint64_t stream_id;
    int n_chan;
    const double* chan_freq_hz;
    int64_t n_samples;
    const uint8_t* vin;
    float* out;
    int flags;              /* 0 or BF_END_OF_STREAM */
    const double* ew_sin_frames; /* tracking E-W beams (Sec. 3.1: "static or
                               tracking"): host [n_frames_out][n_ew] sin of the
                               E-W beam angles for each output frame of this
                               request, or NULL for the plan's static beams */
} bf_request;

/* Frames a request will produce given the stream's current carry (host-side). */
int bf_frames_out(bf_plan_t p, uint64_t stream_id, int64_t n_samples, int64_t* n_frames_out);

/*
 * Submit a request.  DIRECT mode: the work is enqueued on the plan's stream
 * before returning (BF_OK).  SERVING mode: the request is queued (BF_OK if it
 * was admitted at once, BF_EQUEUED if it waits for memory); the plan thread
 * batches admitted requests of different streams into one launch.  *ticket
 * identifies the request for bf_poll.  Requests of one stream run in order.
 * Results do not depend on batching: a stream cut into requests anywhere, or
 * run alone or in a mixed batch, gives the same output bits (every sum runs
 * in a fixed order, whichever CTAs take its parts).
 */
int bf_submit(bf_plan_t p, const bf_request* r, uint64_t* ticket);

/*
 * Wait up to timeout_us microseconds (0 = just test, <0 = forever) for a
 * ticket.  BF_OK: output written, *n_frames_out set, ticket released.
 * BF_PENDING: still running.  Negative: error (the ticket is released).
 */
int bf_poll(bf_plan_t p, uint64_t ticket, int64_t timeout_us, int64_t* n_frames_out);

/*
 * bf_poll plus the request's timeline, for latency breakdowns of a serving
 * plan (no counterpart in the paper).  When the call collects the ticket (BF_OK
 * or an error), times (host array of 5 doubles) receives, in seconds on the
 * host's monotonic clock: [0] bf_submit accepted the request; [1] its batch's
 * kernels were enqueued; [2] the runtime saw the batch's completion event (the
 * plan thread checks every 20 us while batches run, and every poll checks);
 * [3] this call collected it; and [4] the batch's device time, from CUDA
 * events recorded on the plan's stream before its first and after its last
 * operation (0 if the batch failed).  So [1] - [0] is the wait in the queue,
 * [2] - [1] - [4] the wait behind earlier batches on the stream (plus launch
 * and event latency), [4] the batch itself, [3] - [2] the caller's delay in
 * collecting.  On BF_PENDING times is left unchanged.  A null times is
 * BF_EINVAL.
 */
int bf_poll_timed(bf_plan_t p, uint64_t ticket, int64_t timeout_us, int64_t* n_frames_out, double* times);

/* Drain outstanding work, free all plan-owned memory and the plan thread. */
int bf_destroy(bf_plan_t p);

/* Message for the calling thread's last error ("" if none). */
const char* bf_last_error(void);

/* ---- products of the intensity output (enqueued on the plan's stream) ---- */

/*
 * Frequency- and time-summed sky map (the map of Fig. 3, Sec. 3.3): for each of
 * the 1024 beams, the sum over its n_sub sub-channels and n_frames frames of a
 * bf_submit output float [1024][n_sub][n_frames] (device, d_out) into
 * d_map float [1024] (device).  Enqueued after earlier work on the plan's
 * stream; returns at once.  FP32 accumulation in a fixed order.
 */
int bf_skymap(bf_plan_t p, const float* d_out, int64_t n_sub, int64_t n_frames, float* d_map);

/*
 * Incoherent dedispersion to one nominal DM (the fourth kernel proposed in
 * Sec. 3.2).  d_out is a bf_submit output float [1024][16*n_chan][n_frames] of
 * channels chan_freq_hz (host [n_chan]).  Sub-channel s of channel c sits at
 * f_c + (8 s + 3.5 - 64) * 390625/128 Hz; its delay in frames relative to the
 * highest sub-channel is floor(((4.148808e3 * dm) * (1/(f f) - 1/(fmax fmax)))
 * / 0.98304e-3 + 1/2) with f in MHz (FP64, that order).  Writes
 * d_series float [1024][n_out] with n_out = n_frames - max delay (0 if
 * negative; *n_out reports it): series[b][t] = sum_s out[b][s][t + d_s].
 * The delay table goes to plan-owned device memory; the kernel is enqueued
 * on the plan's stream and the call returns at once.
 */
int bf_dedisperse(bf_plan_t p, const float* d_out, int n_chan, const double* chan_freq_hz, int64_t n_frames,
                  double dm, float* d_series, int64_t* n_out);

/*
 * bf_dedisperse without any device allocation (the paper has no counterpart).
 * bf_dedisperse keeps its delay table in plan memory that it grows with
 * cudaFree + cudaMalloc, and cudaFree waits for the whole device; callers whose
 * device memory is owned by someone else (a framework's pool reserved up
 * front, an embedding application that forbids allocation after start-up) or
 * that run a latency-bound loop beside other streams cannot make those calls.
 * This entry point takes the same arguments and gives the same result, for
 * n_chan <= 4096 (at most 65536 sub-channels; more is rejected with BF_EINVAL
 * before any work).  The delay table lives in one file-scope device array of
 * 65536 ints (256 KB) that every device loading the library holds until the
 * process exits:
 *   - the array is shared by every plan and thread of the process on that
 *     device, so calls that overlap on the GPU (other streams or threads) race
 *     on it; serialise them;
 *   - it keeps the last call's delays; nothing in it has to start at zero,
 *     because each call writes the n_chan * 16 entries it reads (a copy from
 *     host memory, in stream order on the plan's stream) before its kernel runs;
 *   - the first call on a device looks the array's address up
 *     (cudaGetSymbolAddress, with the device current, return code checked);
 *     make that first call before any stream capture.
 * No cudaMalloc, cudaFree or other allocating call is made.
 */
int bf_dedisperse_static(bf_plan_t p, const float* d_out, int n_chan, const double* chan_freq_hz,
                         int64_t n_frames, double dm, float* d_series, int64_t* n_out);

/*
 * 8-bit intensity (Table 1 lists 8-bit integer output; the paper gives no
 * scaling rule).  For each of n_rows rows of n_frames floats (a bf_submit
 * output viewed as [1024 * n_sub][n_frames]): mean and standard deviation over
 * the row, code = clip(floor(64 + 16 (x - mean) (1/std) + 1/2), 0, 255) (a constant
 * row gives 64), evaluated in FP32 with sums frame by frame, each operation
 * rounded once.  d_codes uint8 [n_rows][n_frames] and optional d_stats float
 * [n_rows][2] (mean, std), both
 * device, caller-owned.  Enqueued on the plan's stream; returns at once.
 */
int bf_rescale_u8(bf_plan_t p, const float* d_out, int64_t n_rows, int64_t n_frames, uint8_t* d_codes,
                  float* d_stats);

/* ---- inspection entry points (used by the parity tests) ------------------ */

/* Host-only: the clamp table (Eq. 1) [n_feed] and E-W weights [n_ew][n_cyl]
 * complex (interleaved re, im; FP32 rounding of FP64 values) that a plan with
 * configuration cfg uses for one frequency.  Needs no GPU; either output may
 * be NULL. */
int bf_debug_tables(const bf_config* cfg, double freq_hz, int32_t* lut_out, float* ew_out);

/* Host-only: the order in which the FP32 form's consumer threads take the 256
 * N-S beams for one frequency: order_out[ell + 128 h] (int16, host, 256
 * entries, caller-owned) is the beam of TMEM lane ell, bin half h.  A
 * permutation of 0..255 chosen so that each group of eight consecutive
 * slots gathers bins from distinct 16-byte shared-memory bank groups (or
 * shares a bin); no paper counterpart (an implementation detail exposed for
 * tests).  BF_EINVAL on a null argument or a non-positive frequency. */
int bf_debug_gather_order(const bf_config* cfg, double freq_hz, int16_t* order_out);

/* Tensor-core forms only: the GEMM output (N-S beams after E-W phasing) as
 * float2 [block][pol][ew][ns][t], t = 0..127, for n_samples a multiple of 384. */
int bf_debug_gemm(bf_plan_t p, double freq_hz, const uint8_t* d_vin, int64_t n_samples, float* d_out);

/* Failure-detection check of the device-side waits (no counterpart in the
 * paper): runs a tensor-core kernel on one frame (d_vin: device, 384 x 2048
 * bytes, 16-byte aligned) with its MMA thread idle, so no pipeline stage is
 * ever released, and every mbarrier wait bounded by wait_ns (1 .. 2e9).  The
 * kernel is the plan's own for the 1-term and 512-row forms (one cluster of
 * two or four CTAs, which also exchange data-tile copies before their waits
 * run out) and the single-CTA tensor-core kernel for every other form.  It
 * neither traps nor spins unbounded: its waits run out, it frees its tensor
 * memory and reports through the plan's status word, and the call returns
 * BF_ETIMEDOUT, after which the plan and the CUDA context remain usable.
 * BF_OK would mean a wait did not expire.  Any plan form may call it; it
 * synchronises the plan's stream. */
int bf_debug_stall(bf_plan_t p, const uint8_t* d_vin, int64_t wait_ns);

/* Device unpack of n bytes into 2n floats (re, im), with the same device
 * code the fused kernel uses.  d_in, d_out device pointers. */
int bf_debug_unpack(bf_plan_t p, const uint8_t* d_in, float* d_out, int64_t n);

/* Stages 1+2 for one channel: complex beams float2 [T][pol][ew][ns] from
 * uint8 [T][2048], computed by the fused kernel's N-S/E-W device code. */
int bf_debug_beams(bf_plan_t p, double freq_hz, const uint8_t* d_vin, int64_t n_samples, float* d_out);

/* Stages 1-3 for one channel: up-channelised complex voltages float2
 * [block][pol][ew][ns][q'] (q' fftshifted) for n_samples a multiple of 384,
 * computed by the fused kernel with detection replaced by a dump. */
int bf_debug_upchan(bf_plan_t p, double freq_hz, const uint8_t* d_vin, int64_t n_samples, float* d_out);

/* ---- measurement aid (no counterpart in the paper) ------------------------ */

/* Throughput probe of the FP32 FMA pipe, the unit that bounds the FP32 form:
 * enqueues on cuda_stream (cudaStream_t; NULL = the legacy default stream) one
 * kernel of 4 CTAs per SM (at most n_sink / 256 CTAs) x 256 threads on the
 * current device; each thread runs iters (rounded up to a multiple of 4) steps
 * of 16 independent packed FFMA2 chains (paired != 0) or 32 scalar FFMA chains,
 * so the pipe and not latency sets the rate.  d_sink: device float [n_sink],
 * n_sink >= 256, caller-owned, receives one value per thread.  *flop_out = the
 * flops the kernel issues (2 per FMA); the caller times the launch on its
 * stream.  Returns at once. */
int bf_fp32_fma_probe(void* cuda_stream, int paired, int64_t iters, float* d_sink, int64_t n_sink,
                      double* flop_out);

#ifdef __cplusplus
}
#endif

#endif /* CHIMEBF_H */
