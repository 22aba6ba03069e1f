// Internal interface between the plan (host C++) and the excision kernels (CUDA).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rfi {

// Bits that kernels OR into the plan's device status word.
constexpr uint32_t kStatusSampleRange = 1u;  // reported as RFI_ERR_SAMPLE_RANGE
constexpr uint32_t kStatusTimeout = 2u;      // reported as RFI_ERR_TIMEOUT
constexpr uint32_t kStatusLayout = 4u;       // unexpected shared-memory window: RFI_ERR_UNSUPPORTED

// Kernel modes beyond the four replacement modes (rfi_mode 0..3), for the Median-of-MAD
// variant (Eq. 3): a pass that only estimates M and D per window, and passes that apply Eq. 1
// and Eq. 2 with a per-window centre and dispersion read from memory (kModeApply + rfi_mode).
constexpr int kModeStats = 4;
constexpr int kModeApply = 8;
constexpr int kApplyTileWindows = 32;  // at most this many windows per tile in apply passes
// Flag bit of the power-metered excision: the kernel also sums x^2 and z^2 over every window
// (the detected power of the unfiltered and filtered signal, for the improvement metric of
// Section III-A) and writes them to Seg::power.
constexpr int kModePower = 16;
// Flag bit of the digital-copy pass (Section III-A): one histogram, median and MAD per window and
// up to kMaxCopies (k, replacement) variants written to their own outputs. The variants come
// from Params::var; variant v of segment s is segment v * Params::seg_stride + s.
constexpr int kModeCopies = 32;
// Flag bits of the fused output format: write the excised samples as fp16 (int8 and 12-bit
// input) or bf16 (int8 input), the real-valued input a channeliser FFT reads. Both are exact.
constexpr int kModeF16 = 64;
constexpr int kModeBF16 = 128;
constexpr int kMaxCopies = 8;
// Flag bit of the multi-window form (8-bit, one consumer group; plain excision or the estimation
// pass): tiles of several small windows of 2^l samples (512..8192) are histogrammed together and
// share one reduce and one set of barriers. A separate instantiation, so that plans without such
// windows keep the plain kernel's shared-memory layout and code.
constexpr int kModeMulti = 256;
// Flag bit of the in-place form that writes back only what changes (RFI_PLAN_WRITE_FLAGGED):
// chunks without a flagged sample are not stored, and with digital noise no chunk is (the noise
// pass writes every flagged sample). Its own instantiation, like kModeMulti.
constexpr int kModeFlaggedOnly = 512;
// Flag bit of the split-warp form (8-bit zero, constant and threshold modes, also write-flagged,
// one group of 8 consumer warps): warps 0-3 histogram, reduce and search window n + 1 while
// warps 4-7 replace window n, handing each window's thresholds over through a ring of slots with
// mbarriers. Its own instantiation, chosen by the launch shape (Shape::warp_split == 2).
constexpr int kModeWarpSplit = 1024;

// One variant of a digital-copy pass.
struct Variant {
    int64_t kq;     // round(k * 1.4826 * 2^16)
    uint64_t seed;  // noise key
    int32_t cval;   // constant replacement, already saturated
    int32_t mode;   // rfi_mode
};

// Device counters of one kernel pass, reset before it.
struct DevCounters {
    unsigned tile_counter;       // dynamic work-list cursor
    uint32_t status;             // kStatus* bits
    unsigned long long flagged;  // flagged samples of the pass
};

// One contiguous run of windows of one stream, starting on a window boundary.
struct Seg {
    const uint8_t *in;    // sample 0 of the run
    uint8_t *out;         // output sample 0
    uint32_t *mask;       // mask block of window 0 (nullable)
    uint32_t *counts;     // flagged count of window 0 (nullable)
    int32_t *med;         // median of window 0 (nullable)
    int32_t *mad;         // MAD of window 0 (nullable)
    int64_t len;          // samples in the run
    int64_t abs0;         // absolute stream index of sample 0 (multiple of W)
    int32_t W;            // window length
    uint32_t stream_id;   // Philox stream key
    int32_t mask_words;   // ceil(W / 32)
    int32_t vec;          // in/out 16-byte aligned and W * bytes_per_sample % 16 == 0
    uint64_t *power;      // detected power of window 0: {sum x^2, sum z^2} (nullable)
    uint32_t pad[2];
};

// Work-list entry of the persistent kernel: windows [w0, w0 + nw) of segment seg.
struct Tile {
    uint32_t seg;
    uint32_t w0;
    uint32_t nw;
    uint32_t bytes;       // input bytes covered by the tile
};

// Method parameters shared by every window of a call.
struct Params {
    int64_t kq;                   // round(k * 1.4826 * 2^16)
    uint64_t seed;                // noise key
    int32_t cval;                 // constant replacement, already saturated
    int32_t ncopies;              // 12-bit histogram copies (1, 2 or 4)
    uint32_t *status;             // device status word (atomicOr of kStatus*)
    unsigned long long *flagged;  // device total of flagged samples
    uint32_t rk0[10], rk1[10];    // Philox4x32-10 round keys of `seed` (see set_round_keys)
    // Digital copy: the number of variants (bits 0-3) and the distance between one variant's
    // segment table and the next (bits 4-31), and the byte offset of the variant table from the
    // status word (both live in the plan's workspace). Packed into 8 bytes: a larger parameter
    // block changes the register allocation of every excision kernel for the worse.
    int32_t copies;
    int32_t var_off;
};

__host__ __device__ inline int params_nvar(const Params &p) { return p.copies & 15; }
__host__ __device__ inline int params_seg_stride(const Params &p) { return p.copies >> 4; }
__host__ __device__ inline const Variant *params_var(const Params &p) {
    return reinterpret_cast<const Variant *>(reinterpret_cast<const char *>(p.status) + p.var_off);
}

// Philox4x32-10 key schedule: round r uses (seed_lo + r * 0x9E3779B9, seed_hi + r * 0xBB67AE85)
// (the Weyl increments of Salmon et al., SC'11), precomputed so kernels read them as constants.
inline void set_round_keys(Params &p) {
    uint32_t k0 = static_cast<uint32_t>(p.seed), k1 = static_cast<uint32_t>(p.seed >> 32);
    for (int r = 0; r < 10; ++r) {
        p.rk0[r] = k0;
        p.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

struct Shape {
    int consumer_warps;   // 4, 8 or 16
    int stages;           // 1..8
    int ctas_per_sm;      // 1..4
    int stage_bytes;      // multiple of 128, >= the largest tile
    int dynamic_tiles;    // 1: atomic counter, 2: static round robin
    int hist_copies;      // 12-bit histogram copies
    int groups;           // consumer groups per CTA (1 or 2)
    int warp_split;       // 2: the split-warp form (kModeWarpSplit) where it runs; 0 or 1: joint
};

// The mode a persistent launch of this shape runs: mode | kModeWarpSplit when the shape asks for
// the split-warp form and the mode and shape allow it.
inline bool warp_split_runs(int bits, int mode, const Shape &s) {
    const int base = mode & ~kModeFlaggedOnly;  // the write-flagged form splits too
    return bits == 8 && base >= 0 && base <= 2 && s.consumer_warps == 8 && s.groups == 1;
}
inline int shape_mode(int bits, int mode, const Shape &s) {
    return s.warp_split == 2 && warp_split_runs(bits, mode, s) ? (mode | kModeWarpSplit) : mode;
}

// Bytes of dynamic shared memory the kernels need.
size_t persistent_smem_bytes(int bits, int mode, const Shape &s);
size_t stream_smem_bytes(int bits, int mode, int consumer_warps, int ncopies, int window_bytes);

// Maximum resident CTAs per SM of the persistent kernel for this shape (0 if it cannot run).
int persistent_occupancy(int bits, int mode, const Shape &s);

// Persistent batched kernel over a device work list. counter: one zeroed uint32 (dynamic tiles).
cudaError_t launch_persistent(int bits, int mode, const Shape &s, int grid, const Seg *segs,
                              const Tile *tiles, int ntiles, const Params &p, unsigned *counter,
                              int inject_timeout, cudaStream_t st);

// Plain kernel: one CTA per window of one segment (windows [w_begin, w_begin + nw)).
cudaError_t launch_stream(int bits, int mode, int consumer_warps, const Seg &seg, int64_t w_begin,
                          int64_t nw, const Params &p, cudaStream_t st);

// Median of MAD (Eq. 3): windows [a, b) of the stream whose window 0 is entry `base` of the
// per-window MAD and MoM arrays. Mm[base + j] = lower median of D[base + max(0, j-kmom+1) .. j].
constexpr int kMomChunk = 128;
struct MomChunk {
    int64_t base;
    int32_t a, b;
};
cudaError_t launch_mom(int bits, const MomChunk *chunks, int nchunks, const int32_t *D, int32_t *Mm, int kmom,
                       cudaStream_t st);

// Digital noise as a second pass over segments whose excision pass wrote 0 at the flagged
// samples, the flag mask, every window's count and every window's M and D (segments of fewer
// than 2^31 samples). The pass's units are 256 mask words: of the whole segment's mask when
// fill_packs(W) (ceil(ceil(len / 32) / 256) units), else of each window (ceil(ceil(W / 32) / 256)
// a window); segment s holds units [fwin[s], fwin[s + 1]), nunits = fwin[nseg]. packed: some
// segment of the launch has fill_packs(W).
constexpr int kFillPackMax = 2048;
__host__ __device__ inline bool fill_packs(int32_t W) { return W % 128 == 0 && W <= kFillPackMax; }
int noise_fill_grid(int sm_count, bool packed);
cudaError_t launch_noise_fill(int bits, bool packed, const Seg *segs, int nseg, const uint32_t *fwin, uint32_t nunits,
                              const Params &p, int grid, cudaStream_t st);

// Write n (<= kSegBatch) segment descriptors to dst (device) from kernel parameters.
constexpr int kSegBatch = 32;
cudaError_t launch_write_segs(Seg *dst, const Seg *src_host, int n, cudaStream_t st);

}  // namespace rfi
