/*
 * gwstream.h -- C ABI of the GB300 streaming inference library for detector
 * time series (DeepClean-shaped noise regression -> subtraction -> resample
 * -> whitening -> BBHnet-shaped detection), after arXiv 2108.12430.
 *
 * Conventions for every entry point
 *  - Returns GW_OK (0) or a negative GW_E* code; gw_last_error() gives a
 *    thread-local message for the last failure on the calling thread.
 *    No C++ exception crosses this boundary.
 *  - "device" pointers are CUDA device memory on the context's device (for
 *    example a torch CUDA tensor's data_ptr()); "host" pointers are CPU memory
 *    (pinned memory makes the copies asynchronous-capable but is not
 *    required).  The caller owns every buffer it passes; the library owns the
 *    objects it creates and all device memory behind them (weights, stream
 *    state, workspaces) until the matching *_destroy.
 *  - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device-pointer entry points are stream-ordered and return
 *    before the GPU finishes; host-pointer entry points return after their
 *    outputs have been written to host memory.
 *  - Sample layouts are row-major, time innermost: [batch][channel][time].
 *  - Layers whose input size fails the checks stated below return GW_EINVAL
 *    and launch nothing.
 */
#ifndef GWSTREAM_H
#define GWSTREAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define GW_OK          0
#define GW_EINVAL     -1  /* bad argument: null pointer, size or mode out of range */
#define GW_EBUDGET    -2  /* the object would exceed the context's HBM budget */
#define GW_ENOMEM     -3  /* cudaMalloc failed */
#define GW_ECUDA      -4  /* a CUDA runtime call or kernel launch failed */
#define GW_ETIMEOUT   -5  /* a bounded wait ran out (host or device side) */
#define GW_ESTATE     -6  /* object in the wrong state (e.g. destroyed, or faulted) */
#define GW_ENOTIMPL   -7  /* combination not implemented (e.g. a precision for a model kind) */
#define GW_ENONFINITE -8  /* NaN or Inf found in an input snapshot */

/* ---- enumerations ------------------------------------------------------ */
enum gw_precision { GW_FP32 = 0, GW_BF16 = 1, GW_FP8 = 2 };
enum gw_model_kind { GW_MODEL_DEEPCLEAN = 0, GW_MODEL_BBHNET = 1 };
enum gw_agg_mode { GW_AGG_LATEST = 0, GW_AGG_AVERAGE = 1 };
enum gw_mem { GW_MEM_HOST = 0, GW_MEM_DEVICE = 1 };

typedef struct gw_ctx* gw_ctx_t;
typedef struct gw_model* gw_model_t;
typedef struct gw_fir* gw_fir_t;
typedef struct gw_stream* gw_stream_t;

const char* gw_last_error(void);
const char* gw_version(void);

/* ---- context ------------------------------------------------------------
 * One context per GPU.  `hbm_budget_bytes` caps the device memory of every
 * object created under the context (0 = no cap); a create that would exceed
 * it returns GW_EBUDGET and allocates nothing.  Creates make the context's
 * device current on the calling thread; every other call launches on the
 * calling thread's current CUDA device, which must be the one of the objects
 * it is given (a thread that did not create them selects it first).  The
 * destroy calls switch to the object's device themselves and give the
 * caller's back.  A server's own threads select its device.
 * gw_ctx_destroy frees the context alone: destroy every object created
 * under it first (an object destroyed after its context reads freed memory).
 */
int gw_ctx_create(int device, size_t hbm_budget_bytes, gw_ctx_t* out);
int gw_ctx_destroy(gw_ctx_t ctx);
size_t gw_ctx_bytes_in_use(gw_ctx_t ctx);

/* ---- models -------------------------------------------------------------
 * DeepClean-shaped autoencoder (Sec. 1, "DeepClean"): 21 -> 8 (k7 s1),
 * 8 -> 16 -> 32 -> 64 (k7 s2 p3), transposed 64 -> 32 -> 16 -> 8 (k7 s2 p3,
 * output padding 1), each with eval BatchNorm + tanh; output conv 8 -> 1 (k7
 * p3).  BBHnet-shaped classifier (Sec. 1, "BBHnet"): stem 2 -> 32 (k16, pad
 * 7/8) + BN + ReLU, 4 residual blocks (32, 64, 128, 256 channels; conv k7 s2,
 * conv k7 s1, shortcut k1 s2, BN after each), global average pool, linear
 * 256 -> 1.
 *
 * `params` (host, FP32) holds the raw, unfolded parameters in canonical
 * order: per layer w (PyTorch layout: conv [C_out][C_in][K], transposed conv
 * [C_in][C_out][K]), b [C_out], then BatchNorm gamma, beta, running mean,
 * running var [C_out] each; BBHnet appends the head w [256], b [1].  Its
 * length must equal gw_model_param_count(kind, n_in).  BatchNorm (eps 1e-5)
 * is folded into the weights in FP64 on the host at create time, then the
 * weights are cast to the model's precision and copied to the device.
 * `in_mean` / `in_std` (host, n_in floats, may be NULL) standardise the
 * input per channel, (x - mean) / std, inside the first kernel.
 * FP8 (BBHnet only): weights are e4m3 with a per-output-channel scale (max
 * |w| -> 448); activations are e4m3 with static per-tensor scales s (stored
 * value e4m3(x s)), accumulation is FP32.  `act_scales` (host, may be NULL):
 * n_layers + 1 entries, the scale of each conv layer's input (a block
 * shortcut's entry is not used: its input is its block's input, quantised
 * with the block's first conv's scale; its output is stored with the block
 * output's scale) and, last, the scale of the final block's output that the
 * pooling head reads.  Without act_scales an FP8 model refuses to run until
 * gw_model_calibrate sets them.
 */
typedef struct gw_model_desc {
  int kind;               /* enum gw_model_kind */
  int precision;          /* enum gw_precision */
  int n_in;               /* input channels: 21 for DeepClean, 2 for BBHnet */
  const float* params;    /* host */
  size_t n_params;
  const float* in_mean;   /* host [n_in] or NULL */
  const float* in_std;    /* host [n_in] or NULL */
  const float* act_scales;/* host [n_layers + 1] or NULL (FP8) */
  int n_act_scales;
} gw_model_desc;

size_t gw_model_param_count(int kind, int n_in);
int gw_model_create(gw_ctx_t ctx, const gw_model_desc* desc, gw_model_t* out);
int gw_model_destroy(gw_model_t m);
/* Synchronises cuda_stream and reports whether a tensor-core kernel of this
 * model gave up a bounded device-side wait (GW_ETIMEOUT) since creation. */
int gw_model_status(gw_model_t m, void* cuda_stream);
/* Test of the failure path of the bounded device-side waits (no GPU fault is
 * involved).  Runs one DeepClean forward (1 window of 4096 samples, zero input)
 * of a BF16 model in which one CTA of the first layer never arms one input
 * stage, so that its MMA thread's wait runs out after about 1 s and the
 * launch unwinds; *observed receives what the host then reads
 * (GW_ETIMEOUT expected).  The model's error flag is cleared and a normal
 * forward is run on the same stream: the call returns GW_OK when it succeeds
 * (GW_ETIMEOUT if the flag is set again).  Synchronises cuda_stream; not to be
 * called concurrently with other work of the same model. */
int gw_model_test_wait_timeout(gw_model_t m, int* observed, void* cuda_stream);

/* DeepClean forward over B windows of L samples (L a multiple of 8).
 * x: device FP32; channel c of window b is the L samples starting at
 *    x + c * ld + b * window_stride, so B consecutive snapshots of one stream
 *    are overlapping views of one [C][ld] buffer (window_stride = stride S).
 * y: device FP32 [B][L], the predicted noise.
 * Output per window: the network of gw_model_create applied to that window
 * alone, zero padding at its edges (Methods, "Streaming IaaS": every
 * snapshot goes through the static model on its own). */
int gw_deepclean_forward(gw_model_t m, const float* x, int64_t ld, int64_t window_stride,
                         int B, int L, float* y, void* cuda_stream);

/* The same FP32 DeepClean forward for callers that cannot allocate device
 * memory -- for example a real-time loop that reserved its memory at start-up
 * and must never block in cudaMalloc, or a host framework that forbids
 * allocations by plug-in libraries.  The paper has no counterpart: this is a
 * deployment variant.  It calls no cudaMalloc/cudaFree and no allocating
 * library routine; its scratch is a fixed 2 MiB array inside the library
 * image, held by every GPU that loads the library until the process exits.
 * Limits: FP32 models only (GW_ENOTIMPL otherwise) and B * L <= 32768 samples
 * (GW_EINVAL beyond).  The first call on each device looks up the array's
 * device address on the current device; make that first call before any
 * CUDA stream capture.  The current CUDA device must be the model's
 * (GW_EINVAL otherwise).  All calls share the one array, so calls that overlap
 * on the GPU (different streams, or different host threads) race and must be
 * serialised by the caller; the array needs no clearing, because each layer
 * overwrites what the next layer reads.  Arguments as gw_deepclean_forward. */
int gw_deepclean_forward_noalloc(gw_model_t m, const float* x, int64_t ld, int64_t window_stride,
                                 int B, int L, float* y, void* cuda_stream);

/* BBHnet logits.  x: device FP32 [B][2][L] whitened strain (L a multiple of
 * 16, L >= 16); logits: device FP32 [B]. */
int gw_bbhnet_score(gw_model_t m, const float* x, int B, int L, float* logits, void* cuda_stream);

/* Static FP8 activation scales from a calibration batch (FP8 BBHnet models;
 * GW_EINVAL otherwise): runs the model's folded FP32 weights on x (device
 * [B][2][L]), records max |.| of every quantised tensor, and sets each scale
 * to 448 / (headroom * max) (headroom >= 1).  scales_out (host, may be NULL)
 * receives the n_layers + 1 scales in the act_scales order.  Synchronises
 * cuda_stream. */
int gw_model_calibrate(gw_model_t m, const float* x, int B, int L, float headroom, float* scales_out,
                       void* cuda_stream);

/* ---- whitening FIR --------------------------------------------------------
 * Linear-phase whitening filter designed in FP64 on the host from a
 * one-sided PSD sampled on f_j = j fs / nfft, j = 0 .. nfft/2 (n_psd =
 * nfft/2 + 1, nfft even): target amplitude sqrt(2 / (fs S_j)) (unit-variance
 * output), zero-phase inverse DFT, centred, truncated to `ntaps` (odd,
 * <= nfft) and Hann-windowed.  `precision` selects FP32 SIMT or BF16
 * tensor-core application. */
int gw_fir_create_whitening(gw_ctx_t ctx, const double* psd, int n_psd, double fs, int ntaps,
                            int precision, gw_fir_t* out);
int gw_fir_destroy(gw_fir_t f);
int gw_fir_ntaps(gw_fir_t f);
/* Anti-alias low-pass for resampling by 2 (the paper resamples its 4096 Hz
 * cleaned strain before BBHnet in the end-to-end ensemble, Methods,
 * "Offline Deployment"; the filter itself is unspecified, so this is a
 * reading): a Hann-windowed sinc with cutoff fc at sample rate fs,
 * h[j] ~ (2 fc / fs) sinc(2 fc / fs (j - (ntaps-1)/2)) w_Hann[j], normalised to
 * sum 1 (unit DC gain), designed in FP64.  ntaps odd.  BF16 needs
 * ntaps = 8 q + 1 (GW_ENOTIMPL otherwise). */
int gw_fir_create_lowpass(gw_ctx_t ctx, double fc, double fs, int ntaps, int precision, gw_fir_t* out);
/* Host copy of the FP64 taps (ntaps doubles). */
int gw_fir_taps(gw_fir_t f, double* taps_out);
/* Valid-mode filtering y[b][c][n] = sum_k h[k] x[b][c][n + k],
 * n < L_in - ntaps + 1.  x: device FP32 [B][C][L_in]; y: device FP32
 * [B][C][L_in - ntaps + 1]. */
int gw_whiten(gw_fir_t f, const float* x, int B, int C, int L_in, float* y, void* cuda_stream);

/* ---- streams ---------------------------------------------------------------
 * A stream keeps the snapshot state of one or two detectors on the device
 * (Methods, "Streaming IaaS": the state holds the previous snapshot and each
 * request brings only floor(f_s / r) = stride new samples).  Snapshot k is
 * the last `window` samples ending after push k; before the stream has
 * `window` samples the missing past is zero.  Each push of n_snap snapshots
 * runs DeepClean on the n_snap windows (one batch), subtracts the aggregated
 * prediction from strain and returns stride cleaned samples per snapshot
 * (Methods, "Data aggregation" and "Aggregation latency"):
 *   emitted times of snapshot k: [k*stride - agg_delay, (k+1)*stride - agg_delay)
 *   GW_AGG_LATEST : the newest window's prediction on those times;
 *   GW_AGG_AVERAGE: the mean over every window pushed so far that covers a
 *                   time, summed in window order (agg_delay = window - stride
 *                   gives full overlap-add over window/stride windows).
 * Strain before time 0 counts as zero.  Constraints: stride a multiple of 8,
 * window a multiple of 8 and of stride, 0 <= agg_delay <= window - stride,
 * 1 <= n_snap <= max_batch. */
typedef struct gw_stream_desc {
  int n_det;       /* detectors, 1 or 2; one DeepClean model each (may be the same object) */
  int n_witness;   /* witness channels per detector (the model's n_in) */
  int window;      /* W samples per snapshot */
  int stride;      /* S new samples per snapshot */
  int max_batch;   /* largest n_snap of one push */
  int agg_mode;    /* enum gw_agg_mode */
  int agg_delay;   /* aggregation latency in samples */
  /* optional post-processing FIR of K (odd) taps applied to the aggregated
   * prediction before subtraction (gw_fir_create_bandpass; FP32; the taps are
   * copied at create, the handle may be destroyed afterwards; NULL = none):
   *   cleaned[t] = strain[t] - sum_k h[k] p[t + k - c],  c = (K - 1) / 2,
   * with p the aggregated prediction (0 before time 0).  The samples returned
   * by a push are then c samples later: [k S - delta - c, k S + S - delta - c). */
  gw_fir_t post;
} gw_stream_desc;

int gw_stream_create(gw_ctx_t ctx, const gw_stream_desc* desc, const gw_model_t* deepclean,
                     gw_stream_t* out);
int gw_stream_destroy(gw_stream_t s);
/* Push n_snap snapshots.
 * witness: [n_det][n_witness][n_snap*stride]; strain: [n_det][n_snap*stride];
 * clean_out: [n_det][n_snap*stride] (snapshot-major within each detector).
 * mem = GW_MEM_HOST: host pointers; the call copies in, runs, copies out and
 *   returns when clean_out is written.
 * mem = GW_MEM_DEVICE: device pointers; stream-ordered on cuda_stream.
 * Non-finite input samples are rejected with GW_ENONFINITE and the stream
 * state is left unchanged (host mode: the staged input is checked on the
 * device before any state update, clean_out is then unspecified; device mode
 * checks on the device and reports through gw_stream_status). */
int gw_stream_push(gw_stream_t s, int n_snap, const float* witness, const float* strain,
                   float* clean_out, int mem, void* cuda_stream);
/* Queued host-buffer pushes for a pipelined client: the same computation as
 * gw_stream_push in host mode (Methods, "Streaming IaaS", "Data aggregation"
 * and "Aggregation latency"), with the client's requests overlapping.  gw_stream_push_async queues push k: the copy
 * of its inputs to the device, the device-side check, the snapshot update,
 * DeepClean, the subtraction and the copy of its cleaned samples to
 * clean_out, all stream-ordered on cuda_stream, and returns without waiting;
 * the host can queue push k + 1 while the device still works on push k.
 * witness / strain / clean_out are host buffers in the layouts of
 * gw_stream_push; they should be page-locked (cudaHostAlloc or a pinned
 * allocator: pageable buffers make the copies synchronous) and must stay
 * valid, the inputs unmodified and clean_out unread, until gw_stream_sync
 * returns.  All pushes queued before a gw_stream_sync use one cuda_stream
 * (GW_EINVAL otherwise); at most GW_STREAM_MAX_PENDING are pending
 * (GW_ESTATE beyond).  gw_stream_push returns GW_ESTATE while pushes are
 * pending.  The head advances at every queued push.
 * gw_stream_sync waits for every pending push.  If one of them held a
 * non-finite sample it returns GW_ENONFINITE and stores its index among the
 * pending pushes (0 = the oldest) in *first_rejected (may be NULL; -1 when
 * none): that push and every later pending one left the stream state
 * unchanged and their clean_out is unspecified, the earlier ones completed,
 * and the head is rewound to that before the rejected push. */
#define GW_STREAM_MAX_PENDING 1024
int gw_stream_push_async(gw_stream_t s, int n_snap, const float* witness, const float* strain,
                         float* clean_out, void* cuda_stream);
int gw_stream_sync(gw_stream_t s, int* first_rejected);
/* Samples pushed so far per detector. */
int64_t gw_stream_head(gw_stream_t s);
/* Device-side status of the stream: GW_OK or GW_ENONFINITE (sticky until reset). */
int gw_stream_status(gw_stream_t s, void* cuda_stream);

/* ---- serving loop ------------------------------------------------------------
 * Many streams, each of n_det detectors, served by one persistent loop that
 * batches the pending snapshots of different streams into one device tick
 * (the paper's inference service answers many concurrent clients whose
 * requests each carry one snapshot of new samples, with the snapshot state
 * kept on the GPU: Methods, "Streaming IaaS", "Online Deployment", and the
 * end-to-end ensemble of "Offline Deployment").  A snapshot of stream s runs
 * the whole path:
 *   1. ring update of the witness and strain state (stride S new samples);
 *   2. DeepClean on the window of the last `window` samples (one model per
 *      detector);
 *   3. subtraction and aggregation as for gw_stream (agg_mode, agg_delay),
 *      giving S cleaned samples c[tau], tau in [k S - agg_delay, (k+1) S - agg_delay);
 *      with desc.post (K taps, c = (K-1)/2) the aggregated estimate is
 *      band-passed before it is subtracted and the S samples are those of
 *      tau in [k S - agg_delay - c, (k+1) S - agg_delay - c), as for gw_stream;
 *   4. 2x resampling with the decimator FIR f (Kf taps, odd):
 *      d[m] = sum_j f[j] c[2 m + j - (Kf-1)/2], c[tau < 0] = 0; d[m] is
 *      computed as soon as every c it reads has been emitted;
 *   5. whitening with the FIR h (Kh taps, odd), centred:
 *      w[n] = sum_j h[j] d[n + j - (Kh-1)/2], d[m < 0] = 0, computed as soon
 *      as its inputs exist;
 *   6. BBHnet on the newest bbh_len whitened samples of every detector
 *      (channel = detector, w[n < 0] = 0), giving one logit.
 * Steps 4-6 are readings: the paper gives neither the resampler nor the exact
 * sample alignment.  Snapshots of one stream run in submission order, at most
 * one per tick; snapshots of different streams share ticks.  Each tick is one
 * CUDA-graph launch (when use_graphs) of the batch rounded up to a bucket.
 *
 * Ownership: the server copies weights handles (the models and FIRs must
 * outlive it); submit copies the inputs before it returns; clean_out and
 * score_out are written by the server's completion thread and must stay
 * valid until gw_server_wait for the ticket returns GW_OK (or the server is
 * destroyed).  All calls are thread-safe. */
typedef struct gw_server* gw_server_t;
typedef struct gw_server_desc {
  int n_det;        /* detectors per stream, 1 or 2 (BBHnet's input channels) */
  int n_witness;    /* witness channels per detector */
  int window;       /* DeepClean window W (samples at the input rate) */
  int max_stride;   /* largest stride a stream may open with (multiple of 8) */
  int max_streams;  /* slot-table size: streams open at once */
  int max_batch;    /* most snapshots in one tick (1 .. max_streams) */
  int max_pending;  /* request slots: submitted, not yet completed (>= max_batch) */
  int agg_mode;     /* enum gw_agg_mode */
  int agg_delay;    /* 0 <= agg_delay <= window - max_stride */
  int bbh_len;      /* BBHnet input length at the resampled rate */
  int max_wait_us;  /* a tick waits up to this long for max_batch snapshots (0 = launch when the device is free) */
  int max_inflight; /* ticks queued on the device at once, 1 .. 4 */
  int use_graphs;   /* 1 = each tick is one CUDA-graph launch; 0 = eager launches */
  int form_lead_us; /* 0 = the next tick is formed as soon as a device slot is free; > 0 = while a tick runs, the
                       next one is formed only when the running tick is expected to end within this many
                       microseconds (its duration estimated from completed ticks of the same batch bucket), or
                       once max_batch snapshots are queued: snapshots that arrive meanwhile join it */
  gw_fir_t post;    /* optional (NULL = none): FP32 FIR of odd length K with which the aggregated noise estimate
                       is post-processed before it is subtracted (Methods, online deployment), as in
                       gw_stream_desc.post; a snapshot then returns the cleaned samples of its emitted times less
                       c = (K - 1) / 2, and resampling, whitening and BBHnet follow that delayed series */
} gw_server_desc;
typedef struct gw_server_stats {
  int64_t snapshots;      /* completed since the last reset */
  int64_t ticks;          /* device ticks since the last reset */
  int64_t kernels;        /* kernels launched by those ticks */
  double mean_batch;      /* snapshots per tick */
  double p50_us, p99_us, mean_us, max_us;  /* submit -> result latency */
  double busy_s;          /* wall time from the first submit to the last completion */
  /* Where a slow request's time went (maxima since the last reset): the
   * device time of a tick (both stages, from events around each stage), the
   * wait from a tick's oldest request's arrival to the tick's launch (the
   * formation loop, or a backlog of ticks), for gw_server_replay how late the
   * load generator queued a request after its scheduled time (0 otherwise),
   * and the host time of one tick's launch calls.  The first stage's start
   * event is recorded before its launch, so a host pause inside the launch
   * calls shows in both the tick's device time and max_launch_call_us. */
  double max_tick_device_us, max_launch_wait_us, max_submit_late_us, max_launch_call_us;
} gw_server_stats;
/* deepclean: n_det models (same precision, n_in = n_witness); bbhnet: a
 * BBHnet with n_in = n_det, or NULL to skip scoring (score_out gets NaN);
 * decimator / whitening: FIRs with odd tap counts (their FP32 taps are used).
 * Preallocates the tick workspace for max_batch snapshots (GW_EBUDGET if it
 * does not fit) and captures the graphs. */
int gw_server_create(gw_ctx_t ctx, const gw_server_desc* d, const gw_model_t* deepclean, gw_model_t bbhnet,
                     gw_fir_t decimator, gw_fir_t whitening, gw_server_t* out);
/* Opens a stream with the given stride (a multiple of 8, and of the first
 * DeepClean layer's phase count for BF16; <= max_stride; divides window).
 * Its device state is allocated now against the context's budget:
 * GW_EBUDGET if it does not fit, GW_ESTATE if every slot is taken. */
int gw_server_open(gw_server_t s, int stride, int* stream_id);
/* Waits for the stream's snapshots in flight, then frees its state and slot.
 * GW_ESTATE if snapshots of it are still pending. */
int gw_server_close(gw_server_t s, int stream_id);
/* Bytes of device state one stream of this stride takes. */
int64_t gw_server_stream_bytes(gw_server_t s, int stride);
/* Queues one snapshot: witness [n_det][n_witness][stride], strain
 * [n_det][stride] (host FP32); results: clean_out [n_det][stride] (host),
 * score_out one float (host, may be NULL).  Blocks while every request slot
 * is taken (GW_ETIMEOUT after 10 s).  GW_ENONFINITE: a non-finite input
 * sample (nothing is queued). */
int gw_server_submit(gw_server_t s, int stream_id, const float* witness, const float* strain, float* clean_out,
                     float* score_out, uint64_t* ticket);
/* GW_OK once the ticket's results are written; GW_ETIMEOUT after timeout_us
 * (< 0 = no limit); GW_EINVAL for a ticket never issued; the server's sticky
 * device error (GW_ETIMEOUT / GW_ECUDA) if a tick failed. */
int gw_server_wait(gw_server_t s, uint64_t ticket, int64_t timeout_us);
int gw_server_stats_read(gw_server_t s, int reset, gw_server_stats* out);
/* Replays an arrival schedule from a host thread of the library (a load
 * generator whose pace does not depend on the caller's language): request i
 * of stream ids[i] is submitted at t0 + t_us[i] (non-decreasing), with the
 * inputs witness[i], strain[i] and outputs clean[i], score[i]; then all are
 * waited for.  latency_us[i] (may be NULL) receives submit -> completion
 * time.  Returns GW_OK or the first error. */
int gw_server_replay(gw_server_t s, int n, const int* ids, const double* t_us, const float* const* witness,
                     const float* const* strain, float* const* clean, float* score, double* latency_us);
/* Stops the loop after the queued work, frees every stream and the workspace. */
int gw_server_destroy(gw_server_t s);

/* ---- one scored stream ---------------------------------------------------
 * The problem statement's call shape for one stream: create a stream with its
 * window and stride, push a snapshot of new samples, get back the cleaned
 * strain and the detection score (Methods, "Streaming IaaS": each request
 * carries floor(f_s / r) = stride new samples and the state stays on the
 * device; "Data aggregation": the response is the newest cleaned samples;
 * the end-to-end ensemble of "Offline Deployment": the two detectors'
 * cleaned strain is resampled, whitened and scored by BBHnet).  It is the
 * serving loop above with one stream in one slot, so a push computes exactly
 * what gw_server_submit computes (steps 1-6 there):
 *   gw_scored_stream_create = gw_server_create (max_streams = max_batch = 1)
 *                             + gw_server_open(stride);
 *   gw_scored_stream_push   = gw_server_submit: witness [n_det][n_witness]
 *                             [stride], strain [n_det][stride] (host FP32,
 *                             copied before it returns); clean_out
 *                             [n_det][stride] and score_out (one float) are
 *                             host buffers written when the ticket
 *                             completes (they must stay valid until then);
 *   gw_scored_stream_wait   = gw_server_wait (GW_ETIMEOUT after timeout_us,
 *                             < 0 = no limit);
 *   gw_scored_stream_destroy closes the stream and frees the server.
 * Pushes run in order; up to max_pending may be queued (a push blocks while
 * all are taken, GW_ETIMEOUT after 10 s).  Arguments and errors otherwise as
 * gw_server_create / _open / _submit / _wait. */
typedef struct gw_scored_stream* gw_scored_stream_t;
int gw_scored_stream_create(gw_ctx_t ctx, const gw_model_t* deepclean, gw_model_t bbhnet, gw_fir_t decimator,
                            gw_fir_t whitening, int n_det, int n_witness, int window, int stride, int agg_mode,
                            int agg_delay, int bbh_len, int max_pending, gw_scored_stream_t* out);
int gw_scored_stream_push(gw_scored_stream_t s, const float* witness, const float* strain, float* clean_out,
                          float* score_out, uint64_t* ticket);
int gw_scored_stream_wait(gw_scored_stream_t s, uint64_t ticket, int64_t timeout_us);
int gw_scored_stream_destroy(gw_scored_stream_t s);

/* ---- stream placement over devices ------------------------------------------
 * Streams are independent and only each stream's own state update is
 * sequential (Methods, "Streaming IaaS"), so serving shards by stream with no
 * collective: each stream lives on one device (one context and server per
 * device).  gw_partition_streams places n streams on n_dev devices (host only,
 * no GPU call):
 *   stride[i]   stride of stream i (its real-time load is proportional to
 *               1 / stride: snapshots per second at a fixed sample rate);
 *   bytes[i]    its device state (gw_server_stream_bytes);
 *   budget[d]   free bytes on device d, or < 0 when the device is not
 *               available (for example a rank that left);
 *   current     (may be NULL) the present placement: a stream keeps its
 *               device while that device is available and has room, so a
 *               rebalance after a device leaves moves only that device's
 *               streams;
 *   device_out  receives the device of every stream (-1: placed nowhere);
 *   load_out    (n_dev, may be NULL) receives each device's summed 1/stride.
 * The streams to place go, in decreasing load (ties by index), to the
 * available device with the least load so far that has room (ties by
 * index): the placement is a deterministic function of the arguments, so
 * every rank of a job computes the same one.  GW_EBUDGET when some stream
 * fits on no device (the others are still placed). */
int gw_partition_streams(int n, const int* stride, const int64_t* bytes, int n_dev, const int64_t* budget,
                         const int* current, int* device_out, double* load_out);

/* ---- training ---------------------------------------------------------------
 * DeepClean is retrained regularly on recent data (main text, on the model's
 * validity and retraining; no loss is given).  Loss (a reading): the
 * band-limited, inverse-PSD-weighted mean square error
 *   L = (1 / N) sum_{b,n} r[b][n]^2,   r = g (*) (strain - y_hat)  (valid mode,
 *   N = B (L - Kg + 1)),
 * where g is designed by gw_fir_create_band_loss.  BatchNorm uses its running
 * statistics, so it folds into the weights; the trained parameters are every
 * layer's raw w, b, gamma, beta in the canonical order of gw_model_create
 * (running mean / var get gradient 0).  Training calls are stream-ordered on
 * device pointers; the arithmetic is FP32 (SIMT FMA), except that with
 * precision GW_BF16 the weight gradients of every layer run on the tensor
 * cores (operands rounded to BF16, FP32 accumulation), and with tc_data also
 * every layer's forward conv and data gradient (the layer inputs and output
 * gradients are rounded to BF16 for the MMAs; activations and gradients are
 * kept in FP32 between layers). */
typedef struct gw_trainer* gw_trainer_t;
typedef struct gw_trainer_desc {
  int n_in;        /* witness channels */
  int max_batch;   /* largest B of a forward */
  int length;      /* window length L (multiple of 8) */
  int checkpoint;  /* 1: keep only the four block inputs and recompute inside the backward */
  int precision;   /* GW_FP32, or GW_BF16: weight gradients on the tensor cores (sm_103a) */
  int tc_data;     /* with GW_BF16: 1 = the forward convs and the data gradients on the tensor cores too
                      (BF16 operands, FP32 activations and gradients between layers) */
} gw_trainer_desc;
/* in_mean / in_std: host [n_in] input standardisation (may be NULL). */
int gw_trainer_create(gw_ctx_t ctx, const gw_trainer_desc* d, const float* in_mean, const float* in_std,
                      gw_trainer_t* out);
int gw_trainer_destroy(gw_trainer_t t);
/* GW_ETIMEOUT if a tensor-core kernel of this trainer gave up a bounded wait
 * (synchronises cuda_stream), else GW_OK. */
int gw_trainer_status(gw_trainer_t t, void* cuda_stream);
/* Length of the flat raw parameter vector (= gw_model_param_count). */
int64_t gw_trainer_param_count(gw_trainer_t t);
int64_t gw_trainer_bytes(gw_trainer_t t);
/* Training forward: params device FP32 raw parameters (caller-owned, read
 * again by the backward), x device [B][n_in][L] raw witness windows, y_hat
 * device [B][L].  Folds BatchNorm on the device and keeps the tape for the
 * next gw_trainer_backward (one forward in flight per trainer). */
int gw_trainer_forward(gw_trainer_t t, const float* params, const float* x, int B, float* y_hat, void* cuda_stream);
/* dy_hat device [B][L] = dLoss/dy_hat; dparams device [param_count] receives
 * dLoss/dparams of the last forward's parameters (overwritten). */
int gw_trainer_backward(gw_trainer_t t, const float* dy_hat, float* dparams, void* cuda_stream);
/* Loss-weight FIR: linear phase, |G(f)|^2 = T(f) S(f_ref) / S(f), T = 1 on
 * [f1 + ramp, f2 - ramp] with raised-cosine ramps to 0 at f1 and f2, S(f_ref)
 * interpolated linearly; designed like the whitening filter (centred inverse
 * real DFT, Hann window, FP64). */
int gw_fir_create_band_loss(gw_ctx_t ctx, const double* psd, int n_psd, double fs, int ntaps, double f1, double f2,
                            double ramp, double f_ref, int precision, gw_fir_t* out);
/* Post-processing band-pass for the DeepClean prediction (Methods, online
 * deployment: the noise estimate is post-processed, then subtracted from the
 * strain; the post-processing itself is not specified, here it keeps the band
 * the network was trained on): zero-phase, |H(f)| = T(f) on the grid
 * f_j = j fs / nfft with T the raised-cosine band of gw_fir_create_band_loss;
 * centred inverse real DFT, Hann window, FP64 design, FP32 taps (ntaps odd,
 * <= nfft).  Used through gw_stream_desc.post. */
int gw_fir_create_bandpass(gw_ctx_t ctx, double fs, int nfft, int ntaps, double f1, double f2, double ramp,
                           int precision, gw_fir_t* out);
/* loss: device scalar; r: device [B][L - ntaps + 1] (kept for the backward);
 * strain, y_hat: device [B][L]. */
int gw_band_loss(gw_fir_t g, const float* strain, const float* y_hat, int B, int L, float* loss, float* r,
                 void* cuda_stream);
/* dy_hat = dloss * dL/dy_hat = -(2 dloss / N) sum_k g[k] r[m - k]; dloss a
 * device scalar or NULL (1). */
int gw_band_loss_backward(gw_fir_t g, const float* r, int B, int L, const float* dloss, float* dy_hat,
                          void* cuda_stream);
/* Adjoint of gw_whiten: dx[b][c][m] = sum_k h[k] dy[b][c][m - k], m < L_in,
 * dy [B][C][L_in - ntaps + 1]; FP32 taps whatever the FIR's precision. */
int gw_fir_backward(gw_fir_t f, const float* dy, int B, int C, int L_in, float* dx, void* cuda_stream);
/* Adam with bias correction on FP32 master parameters (device arrays of n);
 * step counts from 1. */
int gw_adam_step(float* params, const float* grads, float* m, float* v, int64_t n, int step, float lr, float beta1,
                 float beta2, float eps, void* cuda_stream);
/* The same update with the step count in device memory: *step (a device int,
 * the number of steps taken so far) is incremented on the device before the
 * update, which then uses the new value, so a CUDA graph that captured a
 * training step replays successive Adam steps.  Two launches on the stream. */
int gw_adam_step_dev(float* params, const float* grads, float* m, float* v, int64_t n, int* step, float lr,
                     float beta1, float beta2, float eps, void* cuda_stream);

/* ---- instrumentation ---------------------------------------------------------
 * Process-wide, for benchmarks.  gw_profile_enable(1) clears the record and
 * brackets every kernel launch the library makes with a pair of CUDA events on
 * the launching stream (adds a little host overhead per launch);
 * gw_profile_read synchronises those events and writes, per kernel name, the
 * summed device time and the launch count.  `names` receives up to
 * `names_len` bytes of '\n'-separated names in the order of the other two
 * arrays (at most `max_entries` each).  Returns the number of names, or a
 * negative code.  gw_launch_count returns the number of kernels launched by
 * the library since load (always counted); gw_alloc_count the number of
 * device allocations (cudaMalloc calls) the library has made since load. */
/* Host-only inspection of how the tensor-core path lowers one conv layer
 * (no GPU is touched): `spec` = {transposed, c_in, c_out, k, stride, pad_left,
 * pad_right, out_pad}; `wfold` = folded weights [c_out][c_in][k] (FP64);
 * `lin` = input length; in_P / out_P = phase planes of input (0 = the
 * layer's own) and output; `batch` = items the launch plan is made for.
 * Writes the packed B-operand image (per K-step: 2 K-halves x npad rows x 16
 * bytes), the 2-word-per-step table and 26 ints of meta: n_steps, npad,
 * groups, input phases, output positions per row (Q), tap span, min tap
 * shift, M sub-tiles per tile, rows per plane, A stage bytes, steps per
 * weight stage, weight stages, step bytes, TMEM columns, tiles per item,
 * valid rows, channels per position, instruction descriptor, dynamic shared
 * memory bytes, output length, output-column slices per tile, bytes per
 * K-step in a weight stage, packed slice stages (0/1), weight-stage producer
 * warps, input stages, CTAs per SM. */
int gw_tc_inspect(const int* spec, int precision, const double* wfold, int lin, int in_P, int out_P, int batch,
                  void* img_out, size_t img_cap, uint32_t* table_out, int table_cap, int* meta_out);
int gw_profile_enable(int on);
int gw_profile_read(char* names, size_t names_len, double* total_ms, int64_t* launches, int max_entries);
int64_t gw_launch_count(void);
int64_t gw_alloc_count(void);

#ifdef __cplusplus
}
#endif
#endif /* GWSTREAM_H */
