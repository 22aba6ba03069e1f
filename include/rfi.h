/*
 * rfi.h - C ABI of librfi: real-time broadband RFI excision by windowed median / MAD
 * thresholding on GB300 (sm_103a).
 *
 * The method (Buch et al., "Implementing and Characterizing Real-time Broadband RFI Excision
 * for the GMRT Wideband Backend", Section II-D): every input time series (one antenna
 * polarisation, Section II-C) is cut into non-overlapping data windows of W samples. For each
 * window the library computes the median M and the median absolute deviation D, the
 * thresholds tau_U,L = M +- k*(1.4826*D) (Eq. 1, the paper's multiple n is called k here),
 * and replaces every sample with x >= tau_U or x <= tau_L by a replacement value (Eq. 2):
 * zero, a constant, the threshold, or digital noise.
 *
 * Exact integer semantics (identical on every call and every device):
 *   - M and D are lower medians: element (n-1)/2 of the sorted window (of |x - M| for D).
 *   - Kq = floor(k*1.4826*65536 + 0.5); a sample is flagged iff D > 0 and
 *     |x - M| >= ceil(Kq*D / 65536), which is Eq. 2 with inclusive comparisons for integer x.
 *     D = 0 flags nothing.
 *   - RFI_REPLACE_CLIP writes M + floor(Kq*D/65536) above and M - floor(Kq*D/65536) below.
 *   - RFI_REPLACE_NOISE writes M + round_half_away(S2 * 97164 * D / (107020 * 65536)), where
 *     S2 = 2*sum(u_j) - 8*65535 over the eight 16-bit halves u_j of
 *     Philox4x32-10(key = (seed_lo, seed_hi), counter = (i_lo, i_hi, stream_id, 0)) and i is
 *     the absolute sample index in the stream (Salmon et al., SC'11).
 *   - every replacement is saturated to the sample range.
 *   - windows start at absolute sample 0; a stream whose length is not a multiple of W ends
 *     with a shorter window processed by the same rules.
 *
 * Data layout (all device pointers unless stated):
 *   in/out  stream s: stream_len[s] samples, int8 (sample_bits 8) or int16 holding values in
 *           [-2048, 2047] (sample_bits 12). out may equal in (in-place excision). Any alignment
 *           is accepted; 16-byte aligned streams with W*bytes_per_sample a multiple of 16 take
 *           the fast path (bulk copies and vector stores).
 *   mask    stream s: nwin(s) * ceil(W_s/32) uint32 words; window w owns words
 *           [w*ceil(W_s/32), (w+1)*ceil(W_s/32)); bit j (LSB first) of that block is sample j
 *           of the window; bits past the window's end are written as 0. 4-byte aligned.
 *   counts  stream s: nwin(s) uint32 values, the flagged samples per window. 4-byte aligned.
 *   median, mad (rfi_stats): stream s: nwin(s) int32 values.
 *   where nwin(s) = ceil(stream_len[s] / W_s).
 *
 * Ownership: the caller owns every sample, mask, count, median and mad buffer. The plan owns
 * its device workspace (work list, per-window M and D of the last call, counters, status
 * word) and its CUDA graph. Arrays in rfi_plan_desc are copied by rfi_plan_create.
 *
 * Errors: argument errors are returned synchronously and leave no side effects. Errors found
 * by the device (a 12-bit sample out of range, a bounded wait that timed out) are latched into
 * the plan's status word for that call and returned by rfi_stats; the outputs of that call are
 * then undefined. No entry point aborts, traps or waits without a bound.
 *
 * Threading: a plan may be used from one host thread at a time. Calls on one plan are ordered
 * on the CUDA stream they are given; two calls on one plan must not overlap on the device.
 */
#ifndef RFI_H
#define RFI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RFI_API __attribute__((visibility("default")))
#else
#define RFI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rfi_status {
    RFI_OK = 0,
    RFI_ERR_INVALID_ARG = 1,   /* a NULL, out-of-range or inconsistent argument */
    RFI_ERR_UNSUPPORTED = 2,   /* a valid request this build does not serve */
    RFI_ERR_ALIGNMENT = 3,     /* a mask or counts pointer that is not 4-byte aligned */
    RFI_ERR_OOM = 4,           /* device or host allocation failed, or a budget was exceeded */
    RFI_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    RFI_ERR_SAMPLE_RANGE = 6,  /* device: a 12-bit sample outside [-2048, 2047] */
    RFI_ERR_TIMEOUT = 7,       /* device: a bounded wait ran out */
    RFI_ERR_BUSY = 8           /* serving: no free slot for the request right now */
} rfi_status;

typedef enum rfi_mode {
    RFI_REPLACE_ZERO = 0,      /* blanking (Section II-D: "replaced by zeros") */
    RFI_REPLACE_CONST = 1,     /* constant value const_value */
    RFI_REPLACE_CLIP = 2,      /* held at the threshold */
    RFI_REPLACE_NOISE = 3      /* digital noise, see above */
} rfi_mode;

/* rfi_plan_desc.flags */
/* Output sample type (Section II-C: the excised stream feeds the correlator and beamformer,
 * whose channeliser FFT reads real values): the input's own type, or fp16 / bf16. */
typedef enum { RFI_OUT_SAME = 0, RFI_OUT_F16 = 1, RFI_OUT_BF16 = 2 } rfi_out_format;

#define RFI_PLAN_PER_STREAM 0x1u  /* one launch per stream, one CTA per window */
#define RFI_PLAN_BATCHED 0x2u     /* one persistent launch over all windows (default) */
#define RFI_PLAN_GRAPH 0x4u       /* batched launch replayed from a CUDA graph */
#define RFI_PLAN_AUTOTUNE 0x8u    /* time candidate launch shapes at create, keep the fastest */
#define RFI_PLAN_NO_SPLIT 0x20u   /* keep one work list even when window sizes differ widely (see
                                     rfi_plan_create) */
#define RFI_PLAN_POWER 0x10u      /* also sum x^2 and z^2 over every window (the detected power of
                                     the unfiltered and filtered signal, rfi_stats_power), for
                                     the improvement metric of Section III-A. Batched form and
                                     per-window MAD only (RFI_ERR_UNSUPPORTED otherwise); fixed
                                     launch shape as for mom_windows >= 2 */
#define RFI_PLAN_NOISE_PASS 0x40u /* batched noise plans: write the digital noise in a second kernel
                                     over the flag masks instead of inside the excision kernel
                                     (same bits; one more launch per call). Faster for windows of
                                     a few thousand samples, slower for densely flagged data. The
                                     first rfi_excise with a NULL mask for some stream allocates a
                                     plan-owned mask array (ceil(W/32) words per window) that
                                     rfi_plan_destroy frees. Ignored with RFI_PLAN_PER_STREAM,
                                     RFI_PLAN_POWER, fp16/bf16 output, by rfi_excise_host, and in
                                     plans with a stream of 2^31 samples or more */
#define RFI_PLAN_WRITE_FLAGGED 0x80u /* in-place excision that writes back only what changes:
                                        rfi_excise requires out[i] == in[i] for every stream
                                        (RFI_ERR_INVALID_ARG otherwise) and stores only the
                                        16-byte chunks that hold a flagged sample (zero, constant,
                                        threshold) or only the flagged samples themselves (digital
                                        noise); masks and counts are written in full. About 1 + f
                                        bytes of sample traffic per sample (f the fraction of
                                        chunks with a flag) instead of 2. 8-bit batched plans with
                                        per-window MAD only, without RFI_PLAN_POWER, fp16/bf16
                                        output or digital copies (RFI_ERR_UNSUPPORTED otherwise);
                                        RFI_PLAN_NOISE_PASS is ignored; rfi_excise_host writes
                                        every sample as usual */
#define RFI_PLAN_INJECT_TIMEOUT 0x100u /* test hook: CTA 0 waits on a barrier nothing arrives
                                          on (bounded by 1 ms), latching RFI_ERR_TIMEOUT */

/* Launch shape of the persistent kernel; a zero field means "choose". */
typedef struct rfi_launch_shape {
    int32_t consumer_warps;  /* 4, 8 or 16 warps processing windows (plus 1 copy warp) */
    int32_t stages;          /* shared-memory window buffers per CTA, 1..8 */
    int32_t ctas_per_sm;     /* resident CTAs per SM, 1..4 */
    int32_t stage_bytes;     /* bytes per buffer (>= the largest window); 0 = choose */
    int32_t dynamic_tiles;   /* 1: tiles taken from an atomic counter; 2: static round robin */
    int32_t hist_copies;     /* 12-bit histogram copies (1, 2, 4); ignored for 8-bit */
    int32_t groups;          /* consumer groups per CTA, 1 or 2 (each with its own copy warp;
                                2 needs consumer_warps <= 8) */
    int32_t warp_split;      /* 1: every consumer warp runs every phase of a window; 2: four
                                warps histogram, reduce and search each window while the other
                                four replace the window before it (int8 zero, constant and
                                threshold plans with 8 consumer warps in one group, also
                                write-flagged, but neither power-metered, nor digital copies, nor
                                another output format; RFI_ERR_UNSUPPORTED otherwise). 0 = choose: the
                                autotuner tries both where the split form runs, otherwise 1 */
} rfi_launch_shape;

typedef struct rfi_plan_desc {
    int32_t sample_bits;          /* 8 (int8) or 12 (int16 container, [-2048, 2047]) */
    int32_t num_streams;          /* S >= 1 */
    const int64_t *stream_len;    /* [S] samples, >= 1 */
    const int32_t *window_len;    /* [S] W_s in [1, 65536] */
    const uint32_t *stream_id;    /* [S] Philox stream key; NULL means 0..S-1 */
    double k;                     /* threshold multiple (the paper's n), > 0, Kq >= 1 */
    int32_t mode;                 /* rfi_mode */
    int32_t const_value;          /* RFI_REPLACE_CONST value, saturated to the sample range */
    uint64_t seed;                /* RFI_REPLACE_NOISE Philox key */
    uint32_t flags;               /* RFI_PLAN_* */
    const rfi_launch_shape *shape;/* NULL: autotuned or default shape */
    int32_t mom_windows;          /* Median of MAD (Section II-D, Eq. 3): 0 or 1 = each window's
                                     own MAD sets its thresholds; k >= 2 (<= 2^20) = the lower
                                     median of the MADs of the k windows ending at the window
                                     (fewer at a stream's start) does, around the window's own
                                     median. k >= 2 needs the batched form: RFI_PLAN_PER_STREAM
                                     and rfi_excise_host return RFI_ERR_UNSUPPORTED; the launch
                                     shape is fixed (one group of 4 or 8 consumer warps) and
                                     RFI_PLAN_AUTOTUNE has no effect. */
    int32_t out_format;           /* rfi_out_format: the type of the excised samples written to
                                     out (2 bytes per sample for fp16 / bf16); the samples'
                                     values are exact in both. fp16 and bf16 need the batched
                                     form (RFI_ERR_UNSUPPORTED with RFI_PLAN_PER_STREAM,
                                     rfi_excise_host, mom_windows >= 2, RFI_PLAN_POWER, and bf16
                                     with 12-bit samples); out must be 2-byte aligned; fixed
                                     launch shape. */
} rfi_plan_desc;

typedef struct rfi_plan_s *rfi_plan_t;

typedef struct rfi_totals {
    uint64_t windows;        /* windows processed by the last rfi_excise */
    uint64_t flagged;        /* samples flagged by the last rfi_excise */
    int32_t device_status;   /* rfi_status latched on the device during that call */
} rfi_totals;

typedef struct rfi_plan_info {
    int64_t k_q16;           /* Kq */
    uint64_t total_windows;
    uint64_t total_samples;
    uint64_t workspace_bytes;
    int32_t tiles;           /* work-list entries of the persistent kernel */
    int32_t grid;            /* persistent CTAs */
    rfi_launch_shape shape;  /* the shape in use */
    int32_t sm_count;
    int32_t kernels_per_call;/* kernel launches one rfi_excise makes (memsets excluded) */
} rfi_plan_info;

/* Validate desc, copy its arrays, allocate the workspace, build the work list and (with
 * RFI_PLAN_AUTOTUNE) time the candidate launch shapes on scratch buffers. Uses the current
 * CUDA device. Synchronous.
 * A batched plan whose window sizes span more than one stage class (windows of at most 16 KiB,
 * at most 32 KiB, and larger) is split into one internal plan per class, each with its own
 * launch shape, work list and graph, run one after the other on the caller's stream; results
 * are the same bits (RFI_PLAN_NO_SPLIT keeps one work list). rfi_plan_get_info then reports the
 * sum of tiles and kernels, the largest grid and the shape of the class with the most samples. */
RFI_API rfi_status rfi_plan_create(const rfi_plan_desc *desc, rfi_plan_t *plan);

/* Excise every stream of the plan: in[s] -> out[s], optional mask[s] and counts[s] (an array
 * pointer or an element may be NULL to skip that output). Asynchronous on `stream` (a
 * cudaStream_t; NULL = legacy default stream). Host arrays in/out/mask/counts hold device
 * pointers, are read during the call and may be reused at once. */
RFI_API rfi_status rfi_excise(rfi_plan_t plan, const void *const *in, void *const *out,
                      uint32_t *const *mask, uint32_t *const *counts, void *stream);

/* Same computation with HOST buffers (pinned or pageable): input is copied to the device in
 * chunks on `stream` and a second internal stream, excised, and copied back, overlapping the
 * three. Synchronous: returns when every output is in host memory. The first call allocates
 * the plan's staging area: three chunk slots of up to 128 MiB of input each (less when the
 * streams are shorter), with as much output and their masks and counts; rfi_plan_destroy
 * frees it. */
RFI_API rfi_status rfi_excise_host(rfi_plan_t plan, const void *const *in, void *const *out,
                           uint32_t *const *mask, uint32_t *const *counts, void *stream);

/* Results of the last rfi_excise: per-window median and mad into caller device arrays
 * (array pointer or element may be NULL), and totals into *totals (nullable). Synchronises
 * `stream`. Returns the device status of that call (RFI_OK, RFI_ERR_SAMPLE_RANGE,
 * RFI_ERR_TIMEOUT) or a call error. */
RFI_API rfi_status rfi_stats(rfi_plan_t plan, int32_t *const *median, int32_t *const *mad,
                     rfi_totals *totals, void *stream);

/* Digital copy (Section III-A: one input filtered with several threshold multiples and
 * replacement options at once, the FPGA's 1:4 copy mode). A plan for up to RFI_MAX_COPIES
 * variants of (k, mode, const_value, seed); desc gives the streams, windows, stream ids and
 * flags (its k, mode, const_value and seed are not used). One pass stages each window once,
 * estimates its median and MAD once and writes every variant's outputs; each variant's output
 * equals a plain plan's with its parameters. Batched form only (RFI_PLAN_PER_STREAM,
 * RFI_PLAN_POWER and mom_windows >= 2 return RFI_ERR_UNSUPPORTED); fixed launch shape;
 * rfi_excise on such a plan returns RFI_ERR_INVALID_ARG. rfi_stats gives the shared median
 * and MAD and, in totals, the flagged samples of all variants. */
#define RFI_MAX_COPIES 8
typedef struct rfi_variant {
    double k;
    int32_t mode;
    int32_t const_value;
    uint64_t seed;
} rfi_variant;
RFI_API rfi_status rfi_plan_create_copies(const rfi_plan_desc *desc, int32_t nvariants, const rfi_variant *variants,
                                          rfi_plan_t *plan);
/* in: [S] as rfi_excise; out, mask, counts: [nvariants * S], variant-major (entry v * S + s is
 * variant v of stream s); mask and counts (and their elements) may be NULL. Asynchronous. */
RFI_API rfi_status rfi_excise_copies(rfi_plan_t plan, const void *const *in, void *const *out,
                                     uint32_t *const *mask, uint32_t *const *counts, void *stream);

/* Median-of-MAD plans (mom_windows >= 2): the dispersion each window of the last rfi_excise
 * used, the lower median of the MADs of the mom_windows windows ending at it (Eq. 3), into
 * caller device arrays of nwin(s) int32 (array pointer or element may be NULL). Asynchronous
 * on `stream`. RFI_ERR_UNSUPPORTED for other plans. */
RFI_API rfi_status rfi_stats_mom(rfi_plan_t plan, int32_t *const *mom, void *stream);

/* RFI_PLAN_POWER plans: the detected power of every window of the last rfi_excise, two uint64
 * per window {sum of x^2 over its input samples, sum of z^2 over its output samples}, into
 * caller device arrays of 2 * nwin(s) (array pointer or element may be NULL). Asynchronous on
 * `stream`. RFI_ERR_UNSUPPORTED for other plans. */
RFI_API rfi_status rfi_stats_power(rfi_plan_t plan, uint64_t *const *power, void *stream);

/* The improvement metric of Section III-A, on the host, from one stream's per-window power as
 * rfi_stats_power writes it (host copy, 2 * nwin uint64): the power of windows_per_point
 * consecutive windows makes one point of the detected-power series; the points are cut into
 * blocks of points_per_block (a partial block is dropped); each block gives mean / RMS
 * deviation about its mean (blocks with zero deviation are left out), averaged over the blocks
 * into S_U (input) and S_F (output); *db = 10 log10(S_F / S_U), positive when excision improves
 * the series. RFI_ERR_INVALID_ARG without a complete block on both sides. */
RFI_API rfi_status rfi_improvement_db(const uint64_t *power, int64_t nwin, int32_t windows_per_point,
                                      int32_t points_per_block, double *db, double *s_unfiltered,
                                      double *s_filtered);

/* Describe the plan (Kq, sizes, launch shape). */
RFI_API rfi_status rfi_plan_get_info(rfi_plan_t plan, rfi_plan_info *info);

/* Release the plan and everything it owns. NULL-safe; safe after a device error. */
RFI_API rfi_status rfi_plan_destroy(rfi_plan_t plan);

/* Allocation-free excision. The paper has no counterpart: this entry point exists for callers
 * that must not allocate device memory while they excise, such as a real-time receiver loop
 * whose device memory is set aside once at start-up (an allocation can synchronise the device
 * and stall the sample stream) or a host whose memory budget is owned by another allocator.
 *
 * Same computation and layouts as rfi_plan_create + rfi_excise + rfi_stats with the batched
 * form, but with no plan: desc describes the call (flags 0 or RFI_PLAN_BATCHED; desc->shape is
 * ignored, a fixed launch shape is used), and the persistent kernel's work list, segment table
 * and counters live in one fixed device array inside the library of RFI_NOALLOC_SCRATCH_BYTES
 * (1,054,976 bytes: 256 of counters, a 96-byte record per stream and a 16-byte entry per tile,
 * at the limits below), reserved on every GPU that loads the library until the process exits.
 * Nothing is allocated, on the device or the host. median/mad (nullable) receive the
 * per-window M and D directly.
 *
 * Limits: at most RFI_NOALLOC_MAX_STREAMS streams and RFI_NOALLOC_MAX_TILES work-list entries
 * (a tile holds as many whole windows as fit in a stage of up to 227 KiB); beyond them the call
 * returns RFI_ERR_UNSUPPORTED before enqueueing anything.
 *
 * The first call on a device looks up the device address of the fixed array (once per device,
 * with that device current); make it before any stream capture. All calls share the array and
 * it keeps the last call's contents (the counters are cleared at the start of each call), so
 * calls that overlap on the GPU race: serialise them. Asynchronous on `stream` unless totals is
 * non-NULL, in which case the call synchronises `stream`, fills *totals and returns the device
 * status (RFI_OK, RFI_ERR_SAMPLE_RANGE, RFI_ERR_TIMEOUT). Device-detected errors (a 12-bit
 * sample out of range, a bounded wait that timed out) are reported ONLY that way: with totals
 * NULL nothing reads the status word, and the next call clears it.
 *
 * A CUDA error that an earlier call of the caller's left pending (cudaPeekAtLastError) makes
 * the call return RFI_ERR_CUDA before it enqueues anything; the error is left in place for the
 * caller to read. */
#define RFI_NOALLOC_MAX_STREAMS 64
#define RFI_NOALLOC_MAX_TILES 65536
#define RFI_NOALLOC_SCRATCH_BYTES (256 + 96 * RFI_NOALLOC_MAX_STREAMS + 16 * RFI_NOALLOC_MAX_TILES)
RFI_API rfi_status rfi_excise_noalloc(const rfi_plan_desc *desc, const void *const *in, void *const *out,
                                      uint32_t *const *mask, uint32_t *const *counts,
                                      int32_t *const *median, int32_t *const *mad, rfi_totals *totals,
                                      void *stream);

/* ---------------------------------------------------------------------------------------------
 * Serving: real-time excision of sample streams fed in chunks, plus backfill requests, with
 * continuous batching on one GPU (the GWB feeds 60 inputs at 800 Msps each, Section II-C).
 *
 * A server owns one device arena of memory_budget bytes. Each stream s has device rings of
 * ring_samples samples (rounded up to a multiple of W_s) for its input, output, mask, counts,
 * median and MAD. rfi_server_push appends a chunk (host or device memory) at the stream's
 * produced position, or returns RFI_ERR_BUSY when the ring has no room (samples whose output was
 * not yet read and released). rfi_server_submit admits a backfill request (an independent
 * buffer excised like a stream slice starting at absolute index abs0) into a free request slot;
 * a host request also needs room in the arena for its device copies; otherwise RFI_ERR_BUSY (or
 * RFI_ERR_OOM if it can never fit). rfi_server_step launches one persistent-kernel pass over
 * every complete window that has arrived on every ring plus a bounded slice of every admitted
 * request, as long as fewer than two passes are in flight; work that arrives while a pass runs
 * joins the next one. rfi_server_poll reports whether a chunk or request is done and its latency
 * on the device clock, from the push or submit call to the end of the pass that excised its last
 * window; a host request's also covers the copy of its results back. A chunk is done when every
 * window that ends inside it is excised (a trailing partial window is completed by the next
 * chunk of the stream, or by the flush, and is counted with that one). rfi_server_read copies
 * excised output of a stream out of the ring and may release it. Output equals the plan path on
 * the whole stream: windows are aligned to absolute multiples of W_s and the digital noise is
 * keyed by the absolute sample index, so chunking, batching and the mix of concurrent work do
 * not change any result.
 *
 * Checkpoint and resume: rfi_server_position returns, per stream, the absolute index up to which
 * output is complete (a window boundary). A new server created with stream_start = that index,
 * fed from that index on, continues bit for bit.
 *
 * Memory and ordering: the server's copies run on its own non-blocking streams, so device
 * samples passed to push or submit must be complete (their producer synchronised) before the
 * call, and a pushed device buffer may be reused once its chunk's ticket is done. Host chunks and host requests
 * are copied from the caller's memory (pinned memory keeps those copies asynchronous; pageable
 * memory makes them synchronous). A device request's in/out/mask/counts must stay valid until
 * its ticket is done. Reads return after their copy completed.
 *
 * A server is used from one host thread; all calls are synchronous with respect to the host
 * except the device work itself. Errors: RFI_ERR_INVALID_ARG for out-of-range arguments (checked
 * before any CUDA call), RFI_ERR_BUSY for back-pressure (retry after step/read), RFI_ERR_OOM
 * when the budget cannot hold the rings (create) or a host request (submit), RFI_ERR_CUDA when
 * a CUDA call fails; device-side errors (a 12-bit sample out of range, a timed-out wait) latch
 * into rfi_server_stats.device_status. */
typedef struct rfi_server_s *rfi_server_t;

typedef struct rfi_server_desc {
    int32_t sample_bits;             /* 8 or 12 */
    int32_t num_streams;             /* S >= 1 */
    const int32_t *window_len;       /* [S] W_s in [1, 65536] */
    const uint32_t *stream_id;       /* [S] Philox stream key; NULL means 0..S-1 */
    const int64_t *stream_start;     /* [S] absolute index of the first sample, a multiple of
                                        W_s (resume point); NULL means 0 */
    int64_t ring_samples;            /* per-stream ring capacity, >= W_s */
    double k;                        /* threshold multiple, as rfi_plan_desc */
    int32_t mode;                    /* rfi_mode */
    int32_t const_value;
    uint64_t seed;
    uint64_t memory_budget;          /* device bytes for rings, per-pass buffers and requests */
    int32_t max_requests;            /* request slots, >= 1 */
    int32_t request_windows_per_step;/* windows of one request per pass; 0 means 1024 */
} rfi_server_desc;

typedef struct rfi_request_desc {
    const void *in;                  /* samples, host or device (on_device) */
    void *out;                       /* output, same memory kind; may equal in */
    uint32_t *mask;                  /* nullable; layout as rfi_excise */
    uint32_t *counts;                /* nullable */
    int64_t len;                     /* samples, >= 1 */
    int32_t window_len;              /* W in [1, 65536] */
    uint32_t stream_id;              /* Philox stream key */
    int64_t abs0;                    /* absolute index of in[0], a multiple of W */
    int32_t on_device;               /* 1: device pointers; 0: host pointers (copied by the server) */
} rfi_request_desc;

typedef struct rfi_server_stats {
    uint64_t passes;                 /* kernel passes launched */
    uint64_t chunks_done, requests_done;
    uint64_t samples_done;           /* ring samples excised */
    uint64_t request_samples_done;
    uint64_t flagged;
    double chunk_latency_p50_us, chunk_latency_p99_us, chunk_latency_max_us;
    double request_latency_p50_us, request_latency_p99_us;
    double wall_seconds;             /* first push or submit to the last completion */
    uint64_t arena_bytes, arena_peak_bytes;
    int32_t device_status;           /* rfi_status latched by any pass */
    double gpu_busy_seconds;         /* sum of pass durations on the device clock */
} rfi_server_stats;

RFI_API rfi_status rfi_server_create(const rfi_server_desc *desc, rfi_server_t *server);
RFI_API rfi_status rfi_server_push(rfi_server_t server, int32_t stream, const void *samples, int64_t n,
                                   int32_t on_device, uint64_t *ticket);
RFI_API rfi_status rfi_server_submit(rfi_server_t server, const rfi_request_desc *req, uint64_t *ticket);
RFI_API rfi_status rfi_server_step(rfi_server_t server, int32_t *launched);
RFI_API rfi_status rfi_server_poll(rfi_server_t server, uint64_t ticket, int32_t *done, double *latency_us);
/* Copy output samples [start, start+n) of a stream (start, n whole windows except at a flushed
 * end; start >= the released position; start+n <= the completed position) to dst and, if
 * mask_dst != NULL, their mask words; release != 0 frees that ring space (start must then equal
 * the released position). */
RFI_API rfi_status rfi_server_read(rfi_server_t server, int32_t stream, int64_t start, int64_t n, void *dst,
                                   uint32_t *mask_dst, int32_t on_device, int32_t release);
/* Zero-copy consumer: device pointers to the ring's output (and mask words) from `start` (a
 * window boundary in [released, completed]) and the number n of samples readable there before
 * the completed position or the ring's wrap. They stay valid until the range is released. */
RFI_API rfi_status rfi_server_view(rfi_server_t server, int32_t stream, int64_t start, const void **out,
                                   const uint32_t **mask, int64_t *n);
/* Release a stream's output up to `upto` (a window boundary, or the completed end of a flushed
 * stream, in [released, completed]) without copying it. */
RFI_API rfi_status rfi_server_release(rfi_server_t server, int32_t stream, int64_t upto);
/* Move up to cap latency records (ticket, microseconds) of finished chunks and requests out of
 * the server, oldest first; *n gets the number moved. A taken ticket no longer polls as done;
 * the stats percentiles keep every record. */
RFI_API rfi_status rfi_server_take_latencies(rfi_server_t server, uint64_t *tickets, double *latency_us,
                                             int64_t cap, int64_t *n);
/* End of stream: the next pass also excises the last, partial window; no more pushes after. */
RFI_API rfi_status rfi_server_flush(rfi_server_t server, int32_t stream);
RFI_API rfi_status rfi_server_position(rfi_server_t server, int32_t stream, int64_t *produced, int64_t *completed,
                                       int64_t *released);
/* Step and poll until all admitted work is done (bounded by timeout_seconds). */
RFI_API rfi_status rfi_server_drain(rfi_server_t server, double timeout_seconds);
RFI_API rfi_status rfi_server_get_stats(rfi_server_t server, rfi_server_stats *stats);
RFI_API rfi_status rfi_server_destroy(rfi_server_t server);

/* Static description of a status code. */
RFI_API const char *rfi_status_string(rfi_status status);

/* Library version string. */
RFI_API const char *rfi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RFI_H */
