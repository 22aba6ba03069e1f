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
#define RFI_PLAN_PER_STREAM 0x1u  /* one launch per stream, one CTA per window */
#define RFI_PLAN_BATCHED 0x2u     /* one persistent launch over all windows (default) */
#define RFI_PLAN_GRAPH 0x4u       /* batched launch replayed from a CUDA graph */
#define RFI_PLAN_AUTOTUNE 0x8u    /* time candidate launch shapes at create, keep the fastest */
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
 * CUDA device. Synchronous. */
RFI_API rfi_status rfi_plan_create(const rfi_plan_desc *desc, rfi_plan_t *plan);

/* Excise every stream of the plan: in[s] -> out[s], optional mask[s] and counts[s] (an array
 * pointer or an element may be NULL to skip that output). Asynchronous on `stream` (a
 * cudaStream_t; NULL = legacy default stream). Host arrays in/out/mask/counts hold device
 * pointers, are read during the call and may be reused at once. */
RFI_API rfi_status rfi_excise(rfi_plan_t plan, const void *const *in, void *const *out,
                      uint32_t *const *mask, uint32_t *const *counts, void *stream);

/* Same computation with HOST buffers (pinned or pageable): input is copied to the device in
 * chunks on `stream` and a second internal stream, excised, and copied back, overlapping the
 * three. Synchronous: returns when every output is in host memory. */
RFI_API rfi_status rfi_excise_host(rfi_plan_t plan, const void *const *in, void *const *out,
                           uint32_t *const *mask, uint32_t *const *counts, void *stream);

/* Results of the last rfi_excise: per-window median and mad into caller device arrays
 * (array pointer or element may be NULL), and totals into *totals (nullable). Synchronises
 * `stream`. Returns the device status of that call (RFI_OK, RFI_ERR_SAMPLE_RANGE,
 * RFI_ERR_TIMEOUT) or a call error. */
RFI_API rfi_status rfi_stats(rfi_plan_t plan, int32_t *const *median, int32_t *const *mad,
                     rfi_totals *totals, void *stream);

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
 * and counters live in one fixed device array inside the library (about 1.1 MiB, reserved on
 * every GPU that loads the library until the process exits). Nothing is allocated, on the
 * device or the host. median/mad (nullable) receive the per-window M and D directly.
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
 * status (RFI_OK, RFI_ERR_SAMPLE_RANGE, RFI_ERR_TIMEOUT). */
#define RFI_NOALLOC_MAX_STREAMS 64
#define RFI_NOALLOC_MAX_TILES 65536
RFI_API rfi_status rfi_excise_noalloc(const rfi_plan_desc *desc, const void *const *in, void *const *out,
                                      uint32_t *const *mask, uint32_t *const *counts,
                                      int32_t *const *median, int32_t *const *mad, rfi_totals *totals,
                                      void *stream);

/* Static description of a status code. */
RFI_API const char *rfi_status_string(rfi_status status);

/* Library version string. */
RFI_API const char *rfi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RFI_H */
