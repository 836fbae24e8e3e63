/*
 * filark.h -- C-ABI of the GB300 chunked DAS filter chain.
 *
 * The chain is the streaming operator chain of FiLark (arxiv 2605.20132):
 *   1. a causal IIR bandpass given as cascaded second-order sections (SOS),
 *      each section in transposed direct form II, with the filter state carried
 *      from one call to the next (Sec. 3.4: stateful-compatible operators and
 *      the realtime SOS filter; Table 1, "IIR (offline & realtime SOS)");
 *   2. a spatial running mean over the 2h+1 neighbouring channels, which needs
 *      a halo of h channels on each side of every channel block (Sec. 3.4:
 *      overlap-aware execution with halo regions; Table 1, "Spatial ... running
 *      mean");
 *   3. an energy detector, the classic STA/LTA ratio of cf = y^2 over trailing
 *      windows, with running sums carried across calls (Sec. 3.4: threshold
 *      energy detectors behind the monitor interface).
 *
 * Streaming contract (Sec. 3.4 and Sec. 6.2): the concatenation of the outputs
 * of any sequence of pushes equals the output of one push of the whole
 * recording, and every push returns exactly as many samples as it was given.
 * The state after create/reset is zero (x[n<0] = y[n<0] = 0), which keeps the
 * start-up transient of the first chunk that Sec. 6.2 describes.
 *
 * Data layout (every sample buffer, host or device): time-major float32,
 * sample t of channel c at buf[t * ld + c], ld >= n_channels -- the paper's
 * `nt_nc` dimension order (Sec. 3.5, custom loader listing).
 *
 * Exact definitions (the CPU oracle computes these in FP64):
 *   IIR, per channel and section, coefficients divided by a0:
 *       y = b0*u + z1;  z1 = b1*u - a1*y + z2;  z2 = b2*u - a2*y
 *   spatial:  y_sp[n,c] = mean of y_bp[n,c'] over c' in [c-h, c+h] ∩ [0, C)
 *   detector: cf = y_sp^2; STA[n] = (1/ns) sum_{k=n-ns+1..n} cf[k], LTA alike
 *             with nl; R[n] = STA/LTA when n >= nl-1 and the long window holds
 *             a nonzero cf, else 0.  n counts samples since create/reset.
 *
 * Threading: one chain must not be used from two threads at once.  Different
 * chains are independent.  All calls that take a stream enqueue work on it and
 * return without waiting, unless stated otherwise.  Error messages are kept
 * per thread (filark_last_error_string).
 */
#ifndef FILARK_H
#define FILARK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FILARK_ABI_VERSION 1u

/* The same type as the CUDA runtime's cudaStream_t; NULL is the legacy
   default stream. */
typedef struct CUstream_st *filark_stream_t;

typedef enum {
    FILARK_OK = 0,
    FILARK_EINVAL = 1,     /* an argument or configuration value is invalid   */
    FILARK_ENOMEM = 2,     /* host or device allocation failed                */
    FILARK_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed     */
    FILARK_EUNSTABLE = 4,  /* an SOS section has a pole on/outside |z| = 1    */
    FILARK_ETIMEOUT = 5,   /* a bounded device-side wait gave up              */
    FILARK_ESTATE = 6,     /* the chain is in an error state: reset it        */
    FILARK_ENOSYS = 7      /* the configuration is valid but not supported    */
} filark_status;

/* Outputs a chain may be asked to write (bit mask, filark_chain_config.outputs) */
enum {
    FILARK_OUT_RATIO = 1u,     /* STA/LTA ratio R                  */
    FILARK_OUT_BANDPASS = 2u,  /* bandpass output y_bp (stage 1)   */
    FILARK_OUT_SPATIAL = 4u    /* spatial mean y_sp (stage 2)      */
};

/* How the IIR stage carries state between time blocks (see filark_chain_info) */
enum {
    FILARK_PREC_AUTO = 0,      /* planner picks and verifies a mode          */
    FILARK_PREC_MODAL32 = 1,   /* per-pole 2x2 carries in FP32, FP64 across
                                  thread blocks and chunks                   */
    FILARK_PREC_DENSE64 = 2,   /* dense carry in the cascade's own basis,
                                  double-float (~48-bit) arithmetic at every
                                  block, FP64 between chunks (poles very
                                  near 1 or repeated poles)                  */
    FILARK_PREC_ALL32 = 3      /* modal carries in FP32 everywhere, including
                                  the state kept between chunks (comparison
                                  only)                                      */
};

typedef struct {
    uint32_t abi_version;   /* must equal FILARK_ABI_VERSION                      */
    int32_t n_channels;     /* C >= 1                                             */
    double fs;              /* sampling rate in Hz (> 0); metadata only, all
                               windows are given in samples                       */
    int32_t n_sections;     /* S, 0 <= S <= FILARK_MAX_SECTIONS (0 = no IIR)      */
    const double *sos;      /* host, S rows {b0,b1,b2,a0,a1,a2}; copied by create */
    int32_t spatial_width;  /* K = 2h+1, odd, 1 <= K <= FILARK_MAX_SPATIAL_WIDTH;
                               1 = no spatial stage                               */
    int32_t sta_len;        /* ns in samples; 1 <= ns <= nl, or both 0 = detector
                               off                                                */
    int32_t lta_len;        /* nl in samples                                      */
    uint32_t outputs;       /* FILARK_OUT_* mask of the outputs pushes may write  */
    int32_t precision;      /* FILARK_PREC_*                                      */
    int64_t max_chunk;      /* largest n_samples of one push (>= 1); sizes the
                               detector's history ring                            */
} filark_chain_config;

#define FILARK_MAX_SECTIONS 8
#define FILARK_MAX_SPATIAL_WIDTH 33

typedef struct filark_chain filark_chain;

/* Plan details, for diagnostics and benchmarks. */
typedef struct {
    int32_t precision;        /* mode in use (FILARK_PREC_MODAL32, ...)              */
    int32_t block_len;        /* L: samples per time block                           */
    int32_t blocks_per_cta;   /* time blocks per thread block                        */
    int32_t tile_channels;    /* output channels per thread block                    */
    int32_t halo;             /* h = (K-1)/2                                         */
    int32_t n_slots;          /* 2x2 state slots per channel in the kernel           */
    double modal_condition;   /* condition number of the modal basis (inf if none)   */
    double probe_error;       /* planner's FP32-emulation error on its probe signal  */
    int64_t ring_len;         /* detector history ring length in samples (0 = none)  */
    int64_t device_bytes;     /* device memory the chain owns                        */
    int64_t samples;          /* samples pushed since create/reset                   */
} filark_chain_info;

/*
 * Create a chain on CUDA device `cuda_device`.  Validates the configuration
 * (FILARK_EINVAL), checks that every section is stable (FILARK_EUNSTABLE),
 * plans the kernel tables on the host in FP64, allocates the chain's device
 * state and zeroes it.  On success *out receives the chain; on failure *out is
 * set to NULL and nothing is leaked.  Synchronous.
 */
filark_status filark_chain_create(const filark_chain_config *cfg, int cuda_device,
                                  filark_chain **out);

/*
 * Push n_samples new samples of every channel through the chain.
 *   d_in       device, [n_samples][ld_in] float32, ld_in >= C; read only.
 *   d_ratio    device, [n_samples][ld_out] float32, or NULL; STA/LTA ratio.
 *   d_bandpass device, [n_samples][ld_out] float32, or NULL; stage-1 output.
 *   d_spatial  device, [n_samples][ld_out] float32, or NULL; stage-2 output.
 * An output may be non-NULL only if its bit is in cfg.outputs.  Inputs must not
 * overlap outputs.  0 <= n_samples <= max_chunk; 0 is a no-op.  The work is
 * enqueued on `stream`; the caller's buffers must stay valid until it
 * completes.  Returns FILARK_ESTATE if an earlier device-side error was seen
 * (the chain stays in that state until reset), FILARK_ECUDA if a launch fails.
 */
filark_status filark_chain_push_chunk(filark_chain *h, const float *d_in, int64_t ld_in,
                                      int64_t n_samples, float *d_ratio, float *d_bandpass,
                                      float *d_spatial, int64_t ld_out, filark_stream_t stream);

/*
 * As filark_chain_push_chunk, with HOST buffers (pinned memory is fastest).
 * The chain copies the input to its own device staging buffer, runs the push
 * and copies the requested outputs back, all on `stream`, and returns when the
 * outputs are in host memory (synchronous).  Device staging is allocated on the
 * first call (max_chunk samples per buffer).
 */
filark_status filark_chain_push_chunk_host(filark_chain *h, const float *h_in, int64_t ld_in,
                                           int64_t n_samples, float *h_ratio, float *h_bandpass,
                                           float *h_spatial, int64_t ld_out,
                                           filark_stream_t stream);

/*
 * Pipelined host-buffer pushes (no counterpart in the paper, which reads its
 * input on the host and moves it to the device one chunk at a time): the same
 * computation as filark_chain_push_chunk_host, but the call only enqueues the
 * work and returns.  Each push takes the next of FILARK_HOST_SLOTS device
 * staging slots; its input copy runs on a copy stream of the chain, the chain
 * on `stream`, the output copies on a second copy stream, ordered by events,
 * so the copies of one push overlap the computation of its neighbours.  A slot
 * is reused only after the computation and the output copies of its previous
 * push are done.  The host buffers must be page-locked (cudaHostAlloc or
 * registered; pageable memory works but does not overlap) and must stay valid
 * and unmodified until filark_chain_host_sync returns; the outputs are in
 * host memory only then.  Pushes are applied in call order; they may be mixed
 * with filark_chain_push_chunk on the same `stream`.  Call
 * filark_chain_host_sync before filark_chain_reset_state, set_state or reading
 * the outputs.  Argument checks as filark_chain_push_chunk_host.
 */
#define FILARK_HOST_SLOTS 3
filark_status filark_chain_push_host_async(filark_chain *h, const float *h_in, int64_t ld_in,
                                           int64_t n_samples, float *h_ratio, float *h_bandpass,
                                           float *h_spatial, int64_t ld_out,
                                           filark_stream_t stream);
/* Wait for all pipelined host pushes (and `stream`); returns the chain's
   device status as filark_chain_sync_status does. */
filark_status filark_chain_host_sync(filark_chain *h, filark_stream_t stream);

/*
 * Launch geometry (no counterpart in the paper).  Each launch of <= 2048
 * samples cuts every channel tile's samples into 32-sample blocks and gives
 * each CTA of the tile's cluster `blocks_per_cta` consecutive blocks (at most
 * 8 CTAs per tile).  0 selects the default, 8; 1..7 gives a short push more
 * CTAs per tile (raised to ceil(blocks / 8) where a launch would need more
 * than 8 CTAs), which can lower the latency of chains with few channel tiles
 * (512 channels, pushes of 1000 on a GB300: 21.9 -> 17.8 us with 4) and is
 * slower once the tiles fill the GPU.  The dense carry always uses 8.  The
 * outputs are equal within rounding for every setting, and bit-identical for
 * the same setting.  FILARK_EINVAL outside 0..8.
 */
filark_status filark_chain_set_blocks_per_cta(filark_chain *h, int blocks_per_cta);

/*
 * Samples per launch (no counterpart in the paper): a push is cut into
 * launches of at most `samples` samples, a multiple of 256 in 256..2048
 * (0 selects the default, 2048).  A launch's tile runs as a cluster of
 * ceil(samples / 256) CTAs; clusters of 4 pack the SMs more tightly than
 * clusters of 6 or 8, but a push then takes more, smaller launches, and
 * which wins depends on how the lanes' launches interleave.  GB300, 6,000
 * channels, pushes of 1,500: enqueued back to back, one launch per push in
 * two lanes is fastest (85.6 us per push; 1,024 + 476 in three lanes:
 * 94.9 us); with the pushes enqueued about 40 us apart, 1,024 + 476 in three
 * lanes measured 83.3 us against 86.3 us.  The carried state crosses launch
 * boundaries in FP64 / double-float, so outputs are equal within rounding for
 * every setting and bit-identical for the same setting.  FILARK_EINVAL
 * otherwise.  Takes effect at the next push.
 */
filark_status filark_chain_set_launch_samples(filark_chain *h, int samples);

/*
 * Autotuner for the launch geometry above (no counterpart in the paper):
 * times every combination of lanes 1..min(FILARK_MAX_LANES, channel tiles),
 * samples per launch {2048, 1024} and blocks per CTA {8, 4} (the dense carry:
 * 8 only; at most 16 candidates) on the caller's push -- two warm-up pushes,
 * then timed_pushes >= 1 pushes of the same chunk back to back, joined, CUDA
 * events on `stream` -- keeps the fastest and resets the chain's state (the
 * trial pushes advance it).  The outputs are overwritten.  Blocks until done.
 * Arguments as for filark_chain_push_chunk (n_samples >= 1).
 */
filark_status filark_chain_tune(filark_chain *h, const float *d_in, int64_t ld_in, int64_t n_samples, float *d_ratio,
                                float *d_bandpass, float *d_spatial, int64_t ld_out, int timed_pushes,
                                filark_stream_t stream);

typedef struct {
    int32_t n_tuned;              /* candidates timed by the last filark_chain_tune */
    int32_t chosen;               /* index of the one kept (-1: none)               */
    int32_t lanes[16];
    int32_t launch_samples[16];
    int32_t blocks_per_cta[16];   /* 0 = the default, 8                             */
    double ms_per_push[16];
} filark_chain_tuning;
filark_status filark_chain_get_tuning(const filark_chain *h, filark_chain_tuning *out);

/*
 * Lanes (no counterpart in the paper: a throughput mode for pushes that are
 * queued back to back, e.g. a recording replayed from storage).  A launch
 * waits for the whole previous launch before it touches the carried state, so
 * when a push's clusters of channel tiles fill the GPU's SMs 2.4 times over,
 * the third, partly filled wave runs with most SMs idle.  With lanes >= 2 the
 * channel tiles are split into `lanes` contiguous groups, each pushed on an
 * internal stream of the chain, and each tile carries the state of its halo
 * columns itself; the groups do not wait for one another, so one group's
 * pushes fill the other's partial waves.  A push still starts after the work
 * already enqueued on its `stream` (the lanes fork from it), but it does NOT
 * complete on `stream`: its input must stay unmodified, and its outputs are
 * valid, only once a stream made to wait by filark_chain_join has reached that
 * point (or after filark_chain_sync_status / filark_chain_host_sync).  The
 * outputs and the state are bit-identical to lanes = 1.  get_state, set_state,
 * reset_state, sync_status, host_sync and the host-buffer pushes join the
 * lanes into their `stream` first (the host-buffer pushes after each push).
 * Changing the setting waits for the lanes' pending work on the host.
 * lanes = 1 (the default) runs every push on the caller's stream.
 * FILARK_EINVAL outside 1..FILARK_MAX_LANES; FILARK_ECUDA / FILARK_ENOMEM if
 * the streams or the per-tile state (2 x tiles x 64 x 2S doubles) cannot be
 * created.  With fewer channel tiles than lanes, the tiles run one per lane.
 */
#define FILARK_MAX_LANES 4
filark_status filark_chain_set_lanes(filark_chain *h, int lanes);

/* Make `stream` wait (asynchronously) for every push enqueued on the chain's
   lanes; a no-op when none is pending. */
filark_status filark_chain_join(filark_chain *h, filark_stream_t stream);

/* Zero the whole state (IIR, detector sums, history, sample count) on
   `stream`, and clear a sticky error. */
filark_status filark_chain_reset_state(filark_chain *h, filark_stream_t stream);

/* Free everything the chain owns (waits for its work to finish).  NULL is
   accepted. */
filark_status filark_chain_destroy(filark_chain *h);

/*
 * Checkpoint: copy the chain's complete state to host memory.  With
 * host_buf == NULL, *bytes receives the size needed.  The IIR state is written
 * in the canonical layout (per channel, per section z1 then z2, FP64), followed
 * by the detector sums and history.  Synchronous on `stream`.  Restoring it with
 * filark_chain_set_state into a chain of the same configuration continues the
 * stream exactly as if it had not stopped.
 */
filark_status filark_chain_get_state(filark_chain *h, void *host_buf, size_t *bytes,
                                     filark_stream_t stream);
filark_status filark_chain_set_state(filark_chain *h, const void *host_buf, size_t bytes,
                                     filark_stream_t stream);

/* Wait for the chain's work on `stream` and report any device-side error. */
filark_status filark_chain_sync_status(filark_chain *h, filark_stream_t stream);

/* Fill *out with the plan details (host only, no synchronisation). */
filark_status filark_chain_get_info(const filark_chain *h, filark_chain_info *out);

/*
 * Butterworth bandpass design by the bilinear transform (host only).  `order`
 * is the order N of the analog lowpass prototype (the bandpass has order 2N);
 * 0 < f1 < f2 < fs/2.  Writes N SOS rows {b0,b1,b2,a0,a1,a2} to sos_out:
 * conjugate-pole sections with zeros at z = +1 and z = -1, in ascending pole
 * radius, gain spread evenly so that |H| = 1 at the image of the geometric band
 * centre (and 1/sqrt(2) at f1 and f2).
 */
filark_status filark_butter_bandpass_sos(int order, double f1, double f2, double fs,
                                         double *sos_out);

/*
 * Allocation-free variant of the chain (the paper has no counterpart; this is a
 * deployment aid).  For callers that cannot call cudaMalloc -- a real-time
 * acquisition thread whose latency budget rules out allocator calls (cudaMalloc
 * can block and synchronise the device), or a plugin inside a host application
 * that owns all device memory through its own pool.
 *
 * Runs the whole chain over ONE recording of n_samples samples, from a zero
 * state, writing the requested outputs (same layouts and rules as
 * filark_chain_push_chunk; any n_samples >= 0).  An output pointer whose bit is
 * not set in cfg->outputs, an output that overlaps the input or another output,
 * or a stride below n_channels is rejected with FILARK_EINVAL.  The chain's
 * working memory (carried IIR and detector state, cf history ring, dense-carry
 * matrices) lives in a 32 MiB file-scope device array that every GPU which
 * loads the library holds until the process exits; no device memory is
 * allocated or freed (host-side planning uses ordinary heap memory).  A
 * recording whose working memory would exceed the array -- roughly
 * 4 * n_channels * (lta_len + min(n_samples, 2048)) bytes plus the state -- is
 * rejected with FILARK_EINVAL and a message.
 *
 * Every call looks up the array's device address and sets the kernels'
 * attributes on the current device (neither allocates); the first call on a
 * device also loads the library's device code there, so make that first call
 * before any stream capture.  When the plan uses the dense carry
 * (FILARK_PREC_DENSE64, or FILARK_PREC_AUTO for poles very close to z = 1, see
 * filark_chain_get_info of an equivalent chain), the call copies the carry
 * matrices from host memory and waits for `stream` before it returns.  All
 * calls share the array and each call clears the state it starts from, so
 * calls that overlap on the GPU (other streams or host threads) race with each
 * other; serialise them.  Work is enqueued on `stream` on the current CUDA
 * device.
 */
filark_status filark_chain_run_static(const filark_chain_config *cfg, const float *d_in, int64_t ld_in,
                                      int64_t n_samples, float *d_ratio, float *d_bandpass,
                                      float *d_spatial, int64_t ld_out, filark_stream_t stream);

/*
 * Differentiable bandpass: the SOS cascade of the chain's first stage (Sec. 3.4,
 * the SOS filter; Table 1, "IIR (offline & realtime SOS)") as a forward pass
 * with state checkpoints plus its reverse-time adjoint, so that the filter can
 * be fitted or inverted.  Whole records from a zero state (no carried state
 * across calls).  Section s maps u_s to y_s = u_{s+1} by
 *     a0 y[n] + a1 y[n-1] + a2 y[n-2] = b0 u[n] + b1 u[n-1] + b2 u[n-2].
 * Given gy = dL/dy_{S-1}, the backward solves, backwards in time,
 *     a0 w_s[n] + a1 w_s[n+1] + a2 w_s[n+2] = g_s[n]   (w = 0 past the end)
 * and returns
 *     dL/db_i = sum_m u_s[m] w_s[m+i],  dL/da_i = -sum_m y_s[m] w_s[m+i]
 *     (i = 0, 1, 2; a0 included, through the division by a0),
 *     dL/dx = g_0,  g_{s-1}[n] = b0 w_s[n] + b1 w_s[n+1] + b2 w_s[n+2].
 * dL/da0 is formed from the other five of its section: scaling a section's
 * six coefficients by one factor leaves the cascade unchanged, so
 * sum_k c_k dL/dc_k = 0 per section.
 *
 * sos: host, n_sections rows {b0,b1,b2,a0,a1,a2} (raw, not normalised), read
 * during the call only; all finite, a0 != 0; 1 <= n_sections <=
 * FILARK_MAX_SECTIONS.  Signals are time-major float32 as everywhere else
 * (buf[t * ld + c], ld >= n_channels).  Arithmetic is double-float (FP32 pairs, ~48 bits) on the device.
 *
 * Checkpointing: the forward stores only the cascade state (2 * n_sections
 * doubles per channel) at the start of every piece of P ~ sqrt(2 * L) samples
 * of every segment (L the segment length), in the caller's d_ckpt buffer of
 * filark_iir_ckpt_bytes(...) bytes -- about L / P * 2S doubles per channel and
 * segment.  Segments are ckpt_every samples long unless n_channels x
 * ceil(n_samples / ckpt_every) is below 2^17 (too few (segment, channel)
 * threads to fill the GPU): then they are shortened to ceil(ckpt_every / f),
 * f = ceil(2^17 / that product), but not below min(ckpt_every, 128) samples.
 * The backward recomputes the section signals from those checkpoints, one
 * piece at a time, in the caller's d_work buffer of filark_iir_work_bytes(...)
 * bytes -- (P * S + 8S) doubles per channel and segment plus 48S for the
 * reduction of the coefficient gradients -- rather than
 * n_samples * n_sections doubles per channel for all intermediates.  Both
 * size queries return 0 for invalid sizes and depend only on their
 * arguments.
 *
 * Buffers are 8-byte aligned device memory owned by the caller; d_ckpt must
 * hold the checkpoints of a forward with the same sos, sizes and input when the
 * backward runs.  d_y and d_gx may be NULL (skipped).  d_gsos receives
 * n_sections * 6 doubles (device).  Inputs must not overlap outputs.  Work is
 * enqueued on `stream`; argument errors return FILARK_EINVAL before anything is
 * enqueued, launch errors FILARK_ECUDA.
 */
size_t filark_iir_ckpt_bytes(int n_sections, int n_channels, int64_t n_samples, int64_t ckpt_every);
size_t filark_iir_work_bytes(int n_sections, int n_channels, int64_t n_samples, int64_t ckpt_every);
filark_status filark_iir_forward_ckpt(const double *sos, int n_sections, int n_channels, const float *d_x,
                                      int64_t ld_x, int64_t n_samples, float *d_y, int64_t ld_y,
                                      int64_t ckpt_every, void *d_ckpt, size_t ckpt_size,
                                      filark_stream_t stream);
filark_status filark_iir_backward(const double *sos, int n_sections, int n_channels, const float *d_x,
                                  int64_t ld_x, int64_t n_samples, const float *d_gy, int64_t ld_gy,
                                  int64_t ckpt_every, const void *d_ckpt, size_t ckpt_size, void *d_work,
                                  size_t work_size, float *d_gx, int64_t ld_gx, double *d_gsos,
                                  filark_stream_t stream);

/*
 * Batched chains: many independent streams with the same chain configuration
 * (filter, spatial width, detector windows, outputs, precision, max_chunk) but
 * their own channel count, chunk lengths and carried state -- the many
 * concurrent DAS recordings a production deployment serves at once (Sec. 6.2
 * streams one recording; this serves many).  Each push of all streams is ONE
 * persistent kernel: a grid of thread-block clusters walks the (stream,
 * channel tile) work items, longest chunk first, and runs every stream's push
 * with the same arithmetic as filark_chain_push_chunk.  The descriptor upload
 * and the launch are captured once in a CUDA graph and replayed per push.
 *
 * The launch geometry -- time ranges per cluster (1, 2, 4 or 8 CTAs), the
 * scan segment of one CTA (4 .. 8 blocks of 32 samples) and the number of
 * resident clusters -- is chosen by filark_batch_tune, which times the
 * candidates on a caller-given push; until then a fixed default is used.  A
 * stream whose push needs fewer time ranges than the cluster has (a short
 * chunk) shares each cluster among several of its channel tiles.
 */
typedef struct filark_batch filark_batch;

/* One stream's part of a batched push; the same rules as the arguments of
   filark_chain_push_chunk (n_samples may be 0: the stream is skipped). */
typedef struct {
    const float *d_in;
    int64_t ld_in;
    int64_t n_samples;
    float *d_ratio, *d_bandpass, *d_spatial;
    int64_t ld_out;
} filark_chunk_desc;

typedef struct {
    int32_t n_streams;
    int32_t cluster;          /* CTAs (time ranges of 256 samples) per cluster */
    int32_t n_clusters;       /* persistent grid, in clusters                  */
    int32_t use_graph;        /* 1: pushes replay a captured CUDA graph         */
    int64_t n_tiles;          /* work items of a push that feeds every stream  */
    int64_t device_bytes;     /* state, rings, descriptors                     */
    int32_t n_tuned;          /* candidates timed by the last filark_batch_tune */
    int32_t tune_cluster[16];
    int32_t tune_clusters[16];
    double tune_ms[16];       /* mean ms per push of each candidate            */
    int32_t blocks_per_cta;   /* scan blocks of 32 samples per CTA (4 .. 8)     */
    int32_t tune_blocks[16];  /* blocks per CTA of each candidate              */
    double tune_stream_ms;    /* the fastest candidate without the graph       */
} filark_batch_info;

/* cfg is the configuration every stream shares; its n_channels is ignored and
   n_channels[i] (>= 1) is used for stream i.  n_streams >= 1.  Allocates every
   stream's state like filark_chain_create, plus the descriptor buffers and two
   captured graphs. */
filark_status filark_batch_create(const filark_chain_config *cfg, int n_streams, const int32_t *n_channels,
                                  int cuda_device, filark_batch **out);

/* Push descs[0 .. n_streams) (host array, read during the call) on `stream`:
   one launch for all streams.  Returns after enqueueing; the host may block
   briefly until the descriptor upload of the push before last has run. */
filark_status filark_batch_push(filark_batch *b, const filark_chunk_desc *descs, filark_stream_t stream);

/* Time each launch geometry on the push `descs` (warm-up pushes, then
   timed_pushes >= 1 timed ones, CUDA events on `stream`), then the fastest
   once more without the graph; keep the fastest of all and reset every
   stream's state (the trial pushes advance it).  Blocks until done.  The
   outputs of descs are overwritten. */
filark_status filark_batch_tune(filark_batch *b, const filark_chunk_desc *descs, int timed_pushes,
                                filark_stream_t stream);

/* Set the launch geometry by hand: cluster in {1, 2, 4, 8}; n_clusters <= 0
   takes the occupancy limit.  use_graph 1: each push replays a captured graph
   (upload + launch); 0: each push uploads its descriptors on a side stream,
   which overlaps the previous push, and launches with programmatic dependent
   launch, so that its clusters start while the previous push's last items
   drain (the same rule as for filark_chain_push_chunk: work enqueued on
   `stream` between two pushes then runs before the second push's kernel,
   which only reads the caller's input before that push's state is needed). */
filark_status filark_batch_set_launch(filark_batch *b, int cluster, int n_clusters, int use_graph);

/* Scan blocks of 32 samples per CTA, 4 .. 8 (default 8): a unit then spans
   cluster x blocks x 32 samples.  FILARK_EINVAL outside 4 .. 8; FILARK_ENOSYS
   for anything but 8 when the plan uses the dense carry.  Waits for the
   staging buffers' uploads like filark_batch_set_launch. */
filark_status filark_batch_set_blocks_per_cta(filark_batch *b, int blocks);

filark_status filark_batch_reset_state(filark_batch *b, filark_stream_t stream);
filark_status filark_batch_sync_status(filark_batch *b, filark_stream_t stream);
filark_status filark_batch_get_info(const filark_batch *b, filark_batch_info *out);
/* Stream i's chain (owned by the batch; valid until filark_batch_destroy):
   for filark_chain_get_state / get_info.  Pushing it directly is allowed
   between batched pushes. */
filark_status filark_batch_stream(filark_batch *b, int i, filark_chain **out);
filark_status filark_batch_destroy(filark_batch *b);   /* NULL ok */

/*
 * Triggers and events on the detector ratio: the monitor stage behind the
 * energy detector (Sec. 3.4, threshold-based energy detectors behind the
 * monitor interface).
 *
 * Per channel, a hysteresis state carried across pushes (zero after create /
 * reset):  s(n) = 1 if R(n) >= on, 0 if R(n) < off, else s(n-1).  Every
 * maximal run of s = 1 is a channel trigger [t_on, t_off) (sample indices
 * since create/reset, t_off one past the run).  A push reports the triggers
 * that END in it; filark_trigger_flush reports the runs still open (t_off =
 * samples so far, flag FILARK_TRIGGER_OPEN) and keeps the state.  R is
 * compared exactly against the double thresholds.
 *
 * Triggers are appended at d_records[*d_count ...] with one device atomic per
 * trigger: *d_count (device, the caller zeroes it) grows by the number of
 * triggers even past `capacity`; records past capacity are dropped.  Order
 * within a call is unspecified.  Work is enqueued on `stream`.
 *
 * Events: the connected components of a set of triggers, two triggers being
 * joined when their channels differ by one and their intervals share a
 * sample -- the 4-connected regions of the (channel, time) trigger image.
 * Each event is (t_on = earliest start, t_off = latest end, c_min, c_max,
 * n_triggers, flags = OR of the triggers' flags), in unspecified order.
 * filark_events_merge needs a 256-byte aligned device workspace of
 * filark_events_work_bytes(n_triggers, n_channels) bytes and blocks until it
 * is done (it reads back an error flag).  FILARK_EINVAL if a trigger's channel
 * lies outside [0, n_channels).
 */
#define FILARK_TRIGGER_OPEN 1

typedef struct {
    int64_t t_on, t_off;
    int32_t channel;
    int32_t flags;
} filark_trigger_record;

typedef struct {
    int64_t t_on, t_off;
    int32_t c_min, c_max;
    int32_t n_triggers;
    int32_t flags;
} filark_event;

typedef struct filark_trigger filark_trigger;

/* off <= on, both finite; max_chunk: largest n_samples of one push. */
filark_status filark_trigger_create(int n_channels, double on, double off, int64_t max_chunk, int cuda_device,
                                    filark_trigger **out);
/* d_ratio: device [n_samples][ld] float32, ld >= n_channels (e.g. a chain's
   ratio output).  d_count: device, 64-bit. */
filark_status filark_trigger_push(filark_trigger *t, const float *d_ratio, int64_t ld, int64_t n_samples,
                                  filark_trigger_record *d_records, int64_t capacity,
                                  unsigned long long *d_count, filark_stream_t stream);
filark_status filark_trigger_flush(filark_trigger *t, filark_trigger_record *d_records, int64_t capacity,
                                   unsigned long long *d_count, filark_stream_t stream);
filark_status filark_trigger_reset(filark_trigger *t, filark_stream_t stream);

/*
 * Overlap mode (no counterpart in the paper: a throughput mode for pushes
 * queued back to back).  A push is three short dependent kernels: the segment
 * summaries (which read the ratio and depend on nothing else), the per-channel
 * scan (which carries the state from push to push) and the emission of the
 * triggers.  With overlap = 1 they run on two internal streams, so that the
 * summaries of one push run beside the scan and emission of the previous one.
 * A push still starts after the work already enqueued on its `stream` (it
 * forks from it) but does NOT complete on `stream`: the ratio must stay
 * unmodified, and *d_count / d_records are not final, until
 * filark_trigger_join(t, stream) has made `stream` wait for every push so far
 * (flush and reset join first by themselves).  Triggers and their order per
 * channel are the same as without overlap.  Switching the mode waits for the
 * work enqueued so far.  overlap: 0 or 1, else FILARK_EINVAL.
 */
filark_status filark_trigger_set_overlap(filark_trigger *t, int overlap);
filark_status filark_trigger_join(filark_trigger *t, filark_stream_t stream);

/*
 * Chain push with the triggers fused into its detector: the same push as
 * filark_chain_push_chunk with the ratio output (d_ratio required; no
 * bandpass or spatial output), during which the detector also writes the
 * trigger's per-segment summaries from the ratio values it computes, followed
 * by the trigger's scan and emission (filark_trigger_push without its own pass
 * over the ratio).  The ratio and the triggers are the same as those of the
 * two calls made one after the other.  t must have the chain's channel count
 * and n_samples <= its max_chunk.  The scan needs every tile's summaries:
 * with the trigger's overlap mode its scan and emission run on the trigger's
 * stream and wait for this push's launches (in every lane), so a chain in
 * lanes goes on with its next push meanwhile (join both, filark_chain_join
 * and filark_trigger_join, before using the ratio or the triggers); without
 * it the chain's lanes join back into `stream` at the end of the push.
 */
filark_status filark_chain_push_triggers(filark_chain *h, filark_trigger *t, const float *d_in, int64_t ld_in,
                                        int64_t n_samples, float *d_ratio, int64_t ld_out,
                                        filark_trigger_record *d_records, int64_t capacity,
                                        unsigned long long *d_count, filark_stream_t stream);
filark_status filark_trigger_destroy(filark_trigger *t);   /* NULL ok */

size_t filark_events_work_bytes(int64_t n_triggers, int n_channels);
filark_status filark_events_merge(const filark_trigger_record *d_triggers, int64_t n_triggers, int n_channels,
                                  filark_event *d_events, int64_t capacity, unsigned long long *d_n_events,
                                  void *d_work, size_t work_bytes, filark_stream_t stream);

/*
 * Stateful temporal operators on the same streaming contract as the chain
 * (Sec. 3.4, stateful-compatible operators; Table 1, temporal filters and
 * amplitude operators): per channel, x before the stream start is zero, the
 * state is carried across pushes, and the outputs of any sequence of pushes
 * equal one push of the whole recording.
 *
 *   FILARK_TOP_FIR   y[n] = sum_{k<M} h[k] x[n-k]   (realtime FIR; the last M-1
 *                    inputs are carried, overlap-save); `length` = M <= 512,
 *                    `taps` = h (host, M doubles, rounded to float)
 *   FILARK_TOP_MEAN  y[n] = (1/w) sum_{k<w} x[n-k]  (running mean; `length` = w)
 *   FILARK_TOP_AGC   y[n] = x[n] / ((1/w) sum_{k<w} |x[n-k]|), 0 where that mean
 *                    is 0 (running AGC; `length` = w)
 *   FILARK_TOP_EMA   e[n] = (1-a) e[n-1] + a x[n]^2, e[-1] = 0,
 *                    y[n] = x[n] / sqrt(e[n]), 0 where e = 0 (EMA gain
 *                    equalisation; `alpha` = a in (0, 1])
 *
 * Buffers: time-major float32 [n][ld], ld >= n_channels, device; the output
 * must not overlap the input.  Window sums are kept as double-float running
 * prefixes (about 48 significant bits), the EMA state likewise.  Pushes are
 * asynchronous on `stream`; one operator must not be used concurrently.
 */
enum { FILARK_TOP_FIR = 0, FILARK_TOP_MEAN = 1, FILARK_TOP_AGC = 2, FILARK_TOP_EMA = 3 };

typedef struct filark_top filark_top;

filark_status filark_top_create(int kind, int n_channels, int length, const double *taps, double alpha,
                                int64_t max_chunk, int cuda_device, filark_top **out);
filark_status filark_top_push(filark_top *t, const float *d_in, int64_t ld_in, int64_t n_samples,
                              float *d_out, int64_t ld_out, filark_stream_t stream);
filark_status filark_top_reset(filark_top *t, filark_stream_t stream);
filark_status filark_top_destroy(filark_top *t);   /* NULL ok */

/*
 * Overlap-add FFT filtering: the FFT-domain filtering mode the paper benchmarks
 * on the GPU (Table 1, FFT-domain bandpass; Sec. 6.2, overlap-add chunked
 * filtering), with the chain's streaming contract.  Computes
 *     y[n] = sum_{k<M} h[k] x[n-k]   (x before the stream start is zero)
 * for long filters (a windowed-sinc bandpass of thousands of taps): each push
 * is cut into blocks of at most block_len samples, each block is convolved
 * with h through an FFT of N >= block_len + M - 1 points (hand-written Stockham
 * transform, two channels per complex transform), and the M-1 sample overlap
 * tail is carried across blocks and pushes.  block_len <= 0 picks N = the
 * power of two >= 2M.  N is limited to 8192: up to M = 4096 a block_len that
 * does not fit is shortened to 8193 - M; longer filters (M <= 2^24) are cut
 * into partitions of 4096 taps, each block (at most 4096 samples) is
 * transformed once and every partition's product with it is inverse
 * transformed and added at the partition's offset (uniformly partitioned
 * convolution).  filark_fftfilt_get_info reports the largest N and the block
 * length in use.  taps: host, M doubles, rounded to float.  Buffers as for
 * filark_top_push.
 */
typedef struct filark_fftfilt filark_fftfilt;

filark_status filark_fftfilt_create(int n_channels, int n_taps, const double *taps, int block_len,
                                    int64_t max_chunk, int cuda_device, filark_fftfilt **out);
filark_status filark_fftfilt_push(filark_fftfilt *f, const float *d_in, int64_t ld_in, int64_t n_samples,
                                  float *d_out, int64_t ld_out, filark_stream_t stream);
filark_status filark_fftfilt_reset(filark_fftfilt *f, filark_stream_t stream);
filark_status filark_fftfilt_get_info(const filark_fftfilt *f, int *fft_len, int *block_len);
filark_status filark_fftfilt_destroy(filark_fftfilt *f);   /* NULL ok */

/*
 * Headless streaming display path: the paper's ring-buffer texture (Sec. 3.2,
 * ring-buffer streaming visualization -- fixed-size buffer, only the newly
 * exposed columns written, a ring offset for the logical start), the
 * view-dependent downsampling modes of its I/O layer (Sec. 3.5: drop, peak,
 * linear) and the render-time causal display filter whose state is kept
 * across viewport updates (Sec. 3.2) -- as a device buffer, without a graphics
 * API.
 *
 * Per push of n_samples x n_channels (time-major, device):
 *   rows     channels are grouped channels_per_row at a time (the last group
 *            may be shorter) into H = ceil(n_channels / channels_per_row)
 *            display rows, per sample;
 *   filter   with n_sections > 0, the causal SOS filter `sos` (as for the
 *            chain, state carried) runs on the rows at the source rate;
 *   columns  samples are grouped samples_per_column at a time into display
 *            columns counted from the stream start; the samples of an
 *            incomplete column wait for the next push;
 *   ring     column j is stored at ring column j mod width.
 * Group reduction: FILARK_VIEW_DROP the first value, FILARK_VIEW_PEAK the value
 * of largest magnitude (first on ties), FILARK_VIEW_LINEAR the interpolation at
 * the group's centre (the middle value, or the mean of the two middle values).
 * filark_view_image writes the ring as an [H][ld_image] float32 image (device),
 * oldest column at the left, newest at the right, zeros left of the first
 * column.
 */
enum { FILARK_VIEW_DROP = 0, FILARK_VIEW_PEAK = 1, FILARK_VIEW_LINEAR = 2 };

typedef struct filark_view filark_view;

filark_status filark_view_create(int n_channels, int channels_per_row, int samples_per_column, int width, int mode,
                                 int n_sections, const double *sos, int64_t max_chunk, int cuda_device,
                                 filark_view **out);
filark_status filark_view_push(filark_view *v, const float *d_in, int64_t ld_in, int64_t n_samples,
                               filark_stream_t stream);
filark_status filark_view_image(const filark_view *v, float *d_image, int64_t ld_image, filark_stream_t stream);
filark_status filark_view_get_info(const filark_view *v, int *rows, int64_t *columns, int *ring_offset);
filark_status filark_view_reset(filark_view *v, filark_stream_t stream);
filark_status filark_view_destroy(filark_view *v);   /* NULL ok */

/* Message for the last error returned to this thread ("" if none). */
const char *filark_last_error_string(void);

/* FILARK_ABI_VERSION of the loaded library. */
uint32_t filark_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FILARK_H */
