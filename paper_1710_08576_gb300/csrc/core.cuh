// Device building blocks of windowed median / MAD excision (Section II-D, Eq. 1 and Eq. 2).
//
// One data window of n samples lies in shared memory (sample 0 at a 16-byte aligned address).
// A thread group of T threads (the consumer warps of a CTA) processes it in five phases:
//   1. histogram   h[v] = #{i : x_i = v}, exact u32 counts in shared memory
//   2. reduce      fold the privatised histogram copies into one count per bin
//   3. scan        C[v] = sum_{u <= v} h[u] (block-wide prefix sum)
//   4. search      M = smallest v with C[v] >= ceil(n/2)                       (lower median)
//                  D = smallest d with C[M+d] - C[M-d-1] >= ceil(n/2)           (lower MAD)
//                  The second line is the cumulative histogram of |x - M| written through C:
//                  #{|x_i - M| <= d} = C[M+d] - C[M-d-1], so the |x - M| histogram is never
//                  materialised.
//   5. replace     t = ceil(Kq*D / 2^16); x is flagged iff D > 0 and |x - M| >= t, which is
//                  Eq. 2 (x >= tau_U or x <= tau_L) for integer x with Kq = round(k*1.4826*2^16);
//                  flagged samples get the replacement value, the mask bit and the count.
//
// 8-bit samples use a lane-striped histogram: the count of raw byte value u (the int8 sample
// read as unsigned) for lane l is word u*32 + l, so the 32 lanes of a warp always hit 32
// different banks and 32 different words; warps share the table through shared-memory
// atomics, and the reduce phase reads row u into logical bin u ^ 128 = x + 128. 12-bit
// samples use 1, 2 or 4 plain copies of a 4096-bin table selected by lane, which spreads
// same-bin collisions within a warp. One warp searches the cumulative counts for M and D and
// broadcasts the threshold and replacement values through shared memory.
//
// The int8 replace pass works on four samples per 32-bit word: a native byte absolute
// difference, a three-operation byte compare against t, a byte permute that replicates each
// byte's flag bit into 0x00/0xFF, and a byte dot product that packs the flags into mask bits.
//
// Digital-noise replacement is deferred and shared out over the group, in one of two ways
// chosen by sample width for the flag densities each one serves best. int8 (sparse, bursty
// flags): the replace pass lists the chunks that hold a flagged sample with their flag masks;
// after a group barrier the warps share out the list two chunks at a time, expand each mask
// over a half-warp into a per-warp queue of positions, and evaluate Philox whenever 32 are
// queued, so every lane of a batch has a sample. 12-bit (dense flags): the replace pass writes
// the flagged samples' positions into a per-group list, and after one more group barrier all
// threads evaluate Philox for the list; a window whose list would overflow hands the rest of
// its flagged samples to a per-warp path that numbers them across the warp.
//
// Small int8 windows (2^l = 512..8192 samples) can go several to a table (process_tile_multi8):
// window slot g of a tile is counted by its own group of lanes, so up to eight windows share one
// reduce, one set of barriers and searches on separate warps. The in-place form that writes
// back only what changes skips the stores of chunks without a flagged sample (phase_replace's
// FO parameter).

#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace rfi {
namespace dev {

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void red_add_shared(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also returns whether any participating thread passed v = true.
__device__ __forceinline__ bool named_bar_or(int id, int nthreads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(v)), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t tx) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
        "r"(tx)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// try_wait that lets the hardware suspend the thread for up to ~2 us while the phase is open,
// so a waiting warp does not take issue slots from the warps doing work.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(2000u)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity, giving up after timeout_ns of wall time (and after
// a fixed number of polls in any case). Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1; it < (1u << 24); ++it) {
        if (mbar_try_wait_sleep(bar, parity)) return true;
        if ((it & 7u) == 0 && global_timer_ns() - t0 > timeout_ns) return false;
    }
    return false;
}

// Bulk (non-tensor) asynchronous copy global -> shared, completing on an mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// ------------------------------------------------------------------ Philox4x32-10 noise
// Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw (SC'11): ten rounds; in each the
// words 0 and 2 are multiplied by the two round multipliers, the high product halves are
// xor-ed with words 1 and 3 and with the round key. Round r uses the key advanced by r Weyl
// increments, which a key source gives: precomputed in the kernel parameters (KeysPre), or
// derived from the seed on the fly (KeysSeed, for the per-variant seeds of a digital copy).
struct KeysPre {
    const Params &p;  // the kernel's own parameters: indexed with constants, read in place
    __device__ __forceinline__ uint32_t a(int r) const { return p.rk0[r]; }
    __device__ __forceinline__ uint32_t b(int r) const { return p.rk1[r]; }
};
struct KeysSeed {
    uint32_t s0, s1;
    __device__ __forceinline__ uint32_t a(int r) const { return s0 + static_cast<uint32_t>(r) * 0x9E3779B9u; }
    __device__ __forceinline__ uint32_t b(int r) const { return s1 + static_cast<uint32_t>(r) * 0xBB67AE85u; }
};

template <class K>
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const K &key) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit product per multiplier gives both halves
        const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
        const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
        const uint32_t lo0 = static_cast<uint32_t>(p0), hi0 = static_cast<uint32_t>(p0 >> 32);
        const uint32_t lo1 = static_cast<uint32_t>(p1), hi1 = static_cast<uint32_t>(p1 >> 32);
        c = make_uint4(hi1 ^ c.y ^ key.a(r), lo1, hi0 ^ c.w ^ key.b(r), lo0);
    }
    return c;
}

// Digital-noise replacement: M + round_half_away(S2 * sigq / (107020 * 2^16)), sigq = 97164*D,
// S2 = 2 * (sum of the eight 16-bit halves of the Philox output) - 8 * 65535.
// |S2| <= 524280 and sigq < 2^29, so |S2| * sigq < 2^48; dividing by 2^16 first and then by
// 107020 equals one floor division by their product.
template <class K>
__device__ __forceinline__ int32_t noise_value(int32_t M, uint32_t sigq, const K &key, uint32_t sid,
                                               int64_t idx, int32_t lo, int32_t hi) {
    const uint4 r = philox4x32_10(
        make_uint4(static_cast<uint32_t>(idx), static_cast<uint32_t>(static_cast<uint64_t>(idx) >> 32),
                   sid, 0u),
        key);
    // sum of the eight 16-bit halves: each dp2a adds both halves of one word (weights 1, 1)
    const uint32_t s = __dp2a_lo(r.x, 0x0101u, __dp2a_lo(r.y, 0x0101u, __dp2a_lo(r.z, 0x0101u,
                                                                              __dp2a_lo(r.w, 0x0101u, 0u))));
    const int32_t S2 = 2 * static_cast<int32_t>(s) - 8 * 65535;
    const uint32_t mag_s2 = static_cast<uint32_t>(S2 < 0 ? -S2 : S2);
    const uint64_t a = static_cast<uint64_t>(mag_s2) * sigq + 3506831360ull;  // + 107020 * 2^15
    const uint32_t q = static_cast<uint32_t>(a >> 16) / 107020u;
    const int32_t v = M + (S2 < 0 ? -static_cast<int32_t>(q) : static_cast<int32_t>(q));
    return v < lo ? lo : (v > hi ? hi : v);
}

// ------------------------------------------------------------------ shared-memory layout
template <int BITS>
struct Geo {
    static constexpr int kBins = BITS == 8 ? 256 : 4096;
    static constexpr int kOffset = BITS == 8 ? 128 : 2048;  // logical bin = x + kOffset
    static constexpr int kBps = BITS == 8 ? 1 : 2;          // bytes per sample
    static constexpr int kLo = BITS == 8 ? -128 : -2048;
    static constexpr int kHi = BITS == 8 ? 127 : 2047;
    // cumulative counts, laid out against bank conflicts: 8-bit padded, b + b/32; 12-bit
    // swizzled in place: within each row of 16 bins the 16-byte group q sits at q ^ (row/2 mod 4),
    // so that both a warp's consecutive 16-byte writes and its threads' reads of their own rows
    // touch 8 distinct bank groups per 8 lanes
    static constexpr int kCumWords = BITS == 8 ? kBins + kBins / 32 : kBins;
    __host__ __device__ static constexpr int cum_index(int b) {
        return BITS == 8 ? b + (b >> 5) : (b & ~15) | ((((b >> 2) ^ (b >> 5)) & 3) << 2) | (b & 3);
    }
    static constexpr int kChunkSamples = 16 / kBps;          // samples per 16-byte chunk
    // 8-bit, one consumer group: a 32 KiB table of 128-byte rows (raw byte u -> row u, lane l
    // -> word l). 8-bit, two groups: one 64 KiB table of 256-byte rows shared by both (group g
    // owns bytes [128g, 128g + 128) of every row). 12-bit: ncopies tables of 4096 words per group.
    __host__ __device__ static constexpr int hist_bytes(int ncopies, int groups) {
        return BITS == 8 ? (groups == 2 ? 65536 : 32768) : kBins * 4 * ncopies * groups;
    }
    __host__ __device__ static constexpr int row_bytes(int groups) { return groups == 2 ? 256 : 128; }
};

// Shared-window address of the first byte of dynamic shared memory. The 8-bit histogram sits
// there and its atomics use it as an immediate offset; kernels check it at entry.
constexpr uint32_t kDynSmemShared = 1024;

__device__ __forceinline__ int pad32(int b) { return b + (b >> 5); }

struct __align__(16) RepShared {
    int32_t M, D, t, hiv, lov;
    uint32_t sigq, active, pad;
    // int8 replace constants (see Rep8)
    uint32_t mb4, tlo7, tsmall, c4, hi4, lo4, ulo7, usmall;
    uint32_t unone;
    int32_t cval;  // constant replacement (saturated)
    uint32_t pad2[2];
};

// Digital copy only (its own region, so that other kernels keep their shared-memory size).
struct CopyShared {
    RepShared vrep[kMaxCopies];        // threshold and replacement values per variant
    uint32_t vcount[kMaxCopies][2];    // flagged samples, by variant and window parity
    uint32_t ncount[2 * kMaxCopies];   // 12-bit digital-noise list entries, by variant and parity
};

// Apply passes over whole tiles: the thresholds and flag counts of the tile's windows.
struct ApplyTile {
    RepShared rep[kApplyTileWindows];
    uint32_t count[kApplyTileWindows];
};

// Multi-window tiles (8-bit, one consumer group): up to K (4 or 8) small windows are
// histogrammed at once, window slot g in lanes (32/K)g .. (32/K)(g+1)-1 of the lane-striped
// table, so that one reduce, one set of barriers and parallel searches serve them all. Their
// cumulative counts (at most 8192, the largest window of this form) are 16-bit: slot g's
// kCumWords entries at (uint16_t *)cum + g * kCumWords.
constexpr int kMultiMax = 8;
struct MultiTile {
    RepShared rep[kMultiMax];
    uint32_t count[kMultiMax];
};

struct Ctl {
    uint32_t warp_tot[32];
    RepShared rep;       // threshold and replacement values of the current window
    uint32_t count[2];   // flagged samples, by window parity
    uint32_t done[2];    // warps finished with the window, by window parity
    uint32_t err[2];     // 12-bit range error seen in the window, by window parity
    uint32_t ncount[2];  // 12-bit digital-noise list entries, by window parity
    unsigned long long pw[2][2];  // power-metered excision: {sum x^2, sum z^2}, by window parity
    uint32_t abort;      // set when any warp gave up on a bounded wait
    int32_t mb;          // median bin of the current window (written by its owner thread)
    unsigned long long flagged;  // group total
};

// Per-thread running row sums of the 8-bit histogram (the table is never cleared: a window's
// count of a bin is the difference of two consecutive sums, exact modulo 2^32).
struct RowSums {
    uint32_t s[2];
};

// Per-CTA view of the shared-memory regions used by window processing.
struct Shm {
    uint8_t *hist;       // histogram (generic pointer; 8-bit: the 64 KiB table)
    uint32_t hist_s;     // histogram (shared address)
    uint32_t grp;        // 8-bit: byte offset of this group's half row (0 or 128)
    uint32_t *cum;       // padded cumulative counts
    Ctl *ctl;
    int ncopies;         // 12-bit only
    int bar_id;          // named barrier of this consumer group
    CopyShared *cp;      // digital copy: per-variant state (or null)
    uint16_t *nlist;     // digital noise work area (or null): int8, the entries of the chunks that
                         // hold flagged samples (32-bit); 12-bit, the positions of flagged samples
    uint32_t *nring;     // int8 digital noise: kNoiseRing positions per consumer warp (or null)
    ApplyTile *at;       // apply passes: the current tile's thresholds and counts (or null)
    struct MultiTile *mt;  // 8-bit, one group: state of a multi-window tile (or null)
};

// Capacity of the digital-noise work area (16-bit entries: int8 chunk masks of windows up to
// 65536 samples, or 12-bit flagged positions) and the mark of a list entry that was handed to
// the per-warp path.
constexpr int kNoiseList = 4096;
constexpr uint16_t kNoiseSkip = 0xFFFFu;
// Positions a warp's ring holds: fewer than 32 wait between two batches, and one expansion step
// adds at most 32.
constexpr int kNoiseRing = 64;

// Per-thread sums of x^2 and z^2 of the power-metered excision. A thread sees at most
// 65536 / 128 samples of a window, each below 2^22, so 32 bits hold its sums.
struct Pow {
    uint32_t x, z;
};

// One window to process.
struct Win {
    const uint8_t *data;  // shared memory, sample 0, 16-byte aligned
    int32_t n;            // samples
    uint8_t *out;         // global output of sample 0
    uint32_t *mask;       // global mask block (nullable)
    int32_t mask_words;   // ceil(W / 32)
    int64_t abs_idx;      // absolute stream index of sample 0
    uint32_t sid;
    bool vec;             // out is 16-byte aligned: vector stores
};

// ------------------------------------------------------------------ phase 1: histogram
// Shared atomic at histogram address kDynSmemShared + a.
__device__ __forceinline__ void red_hist8(uint32_t a) {
    asm volatile("red.shared.add.u32 [%0+1024], %1;" ::"r"(a), "r"(1u));
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Four int8 samples.
// 256-byte rows: lp = 128*group + 4*lane; the table offset of raw byte u is u*256 + lp, which one
// byte permute assembles (byte 0 from lp, byte 1 = sample byte j, bytes 2-3 zero).
// 128-byte rows: lp = shared address of the table + 4*lane; the address is lp + u*128.
template <int ROWB>
__device__ __forceinline__ void hist8_word(uint32_t lp, uint32_t w) {
    static_assert(kDynSmemShared == 1024, "immediate offset of red_hist8");
    if (ROWB == 256) {
        red_hist8(prmt(w, lp, 0x5504u));
        red_hist8(prmt(w, lp, 0x5514u));
        red_hist8(prmt(w, lp, 0x5524u));
        red_hist8(prmt(w, lp, 0x5534u));
    } else {
        red_add_shared(lp + ((w & 0xFFu) << 7), 1u);
        red_add_shared(lp + (prmt(w, 0u, 0x4441u) << 7), 1u);
        red_add_shared(lp + (prmt(w, 0u, 0x4442u) << 7), 1u);
        red_add_shared(lp + ((w >> 24) << 7), 1u);
    }
}

// Two 12-bit samples in int16 halves. The bin x + 2048 of an in-range sample is its low 12 bits
// with bit 11 flipped; a half is in range iff its bits 15..11 are all equal, which the caller
// accumulates as (w ^ (w << 1)) & 0xF000F000.
__device__ __forceinline__ void hist12_word(uint32_t copy_base, uint32_t w) {
    red_add_shared(copy_base + (((w & 0xFFFu) ^ 0x800u) << 2), 1u);
    red_add_shared(copy_base + ((((w >> 16) & 0xFFFu) ^ 0x800u) << 2), 1u);
}

__device__ __forceinline__ uint32_t range12_bits(uint32_t w) { return (w ^ (w << 1)) & 0xF000F000u; }

template <int BITS, int T, int ROWB>
__device__ __forceinline__ void phase_histogram(const Shm &sm, const Win &w, int tid, int par) {
    const int lane = tid & 31;
    const int nbytes = w.n * Geo<BITS>::kBps;
    const int nfull = nbytes >> 4;
    const uint4 *d4 = reinterpret_cast<const uint4 *>(w.data);
    if (BITS == 8) {
        const uint32_t lb = (ROWB == 256 ? sm.grp : sm.hist_s) + 4u * lane;
        int c = tid;
        for (; c + T < nfull; c += 2 * T) {
            const uint4 a = d4[c], b = d4[c + T];
            hist8_word<ROWB>(lb, a.x); hist8_word<ROWB>(lb, a.y); hist8_word<ROWB>(lb, a.z); hist8_word<ROWB>(lb, a.w);
            hist8_word<ROWB>(lb, b.x); hist8_word<ROWB>(lb, b.y); hist8_word<ROWB>(lb, b.z); hist8_word<ROWB>(lb, b.w);
        }
        if (c < nfull) {
            const uint4 a = d4[c];
            hist8_word<ROWB>(lb, a.x); hist8_word<ROWB>(lb, a.y); hist8_word<ROWB>(lb, a.z); hist8_word<ROWB>(lb, a.w);
        }
        const int rem = nbytes & 15;
        if (tid < rem) {
            const uint32_t u = static_cast<uint32_t>(w.data[nfull * 16 + tid]);
            if (ROWB == 256) red_hist8(lb + (u << 8));
            else red_add_shared(lb + (u << 7), 1u);
        }
    } else {
        const uint32_t cb = sm.hist_s + static_cast<uint32_t>(lane & (sm.ncopies - 1)) * 16384u;
        uint32_t bad = 0;
        for (int c = tid; c < nfull; c += T) {
            const uint4 a = d4[c];
            hist12_word(cb, a.x); hist12_word(cb, a.y); hist12_word(cb, a.z); hist12_word(cb, a.w);
            bad |= range12_bits(a.x) | range12_bits(a.y) | range12_bits(a.z) | range12_bits(a.w);
        }
        const int rem = (nbytes & 15) >> 1;
        if (tid < rem) {
            const uint32_t x = reinterpret_cast<const uint16_t *>(w.data)[nfull * 8 + tid];
            red_add_shared(cb + (((x & 0xFFFu) ^ 0x800u) << 2), 1u);
            bad |= range12_bits(x) & 0xF000u;
        }
        if (bad) atomicOr(&sm.ctl->err[par], 1u);
    }
}

// ------------------------------------------------------------------ phases 2-3: reduce + scan
// Block exclusive offsets of per-thread totals `run` (named barrier inside).
template <int T>
__device__ __forceinline__ uint32_t block_offsets(const Shm &sm, uint32_t run, int tid) {
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sm.ctl->warp_tot[warp] = inc;
    named_bar(sm.bar_id, T);
    const uint32_t pre = __reduce_add_sync(0xFFFFFFFFu, lane < warp ? sm.ctl->warp_tot[lane] : 0u);
    return pre + inc - run;
}

// 8-bit estimation pass: each thread's bins' counts for this window (the differences of its
// running row sums) into the cumulative-count array, for one warp to scan.
template <int T, int ROWB>
__device__ __forceinline__ void phase_reduce8_counts(const Shm &sm, int tid, RowSums &rs) {
    constexpr int TE = T < 256 ? T : 256;
    constexpr int BPT = 256 / TE;
    static_assert(BPT <= 2, "RowSums holds two rows");
    const int lane = tid & 31;
    if (tid < TE) {
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const uint4 *row = reinterpret_cast<const uint4 *>(sm.hist + ((tid * BPT + i) ^ 128) * ROWB + sm.grp);
            uint32_t s = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {  // this group's 32 lane counters (128 bytes of the row)
                const uint4 a = row[(q + lane) & 7];
                s += a.x + a.y + a.z + a.w;
            }
            sm.cum[pad32(tid * BPT + i)] = s - rs.s[i];
            rs.s[i] = s;
        }
    }
}

// One warp, after phase_reduce8_counts and a group barrier: the inclusive scan of the 256 counts
// in place (8 consecutive bins per lane) and the median bin, the lowest whose cumulative count
// reaches ceil(n/2), into the control block.
__device__ __forceinline__ void phase_scan8_warp(const Shm &sm, int n, int lane) {
    uint32_t *cum = sm.cum;
    uint32_t c[8];
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        run += cum[pad32(lane * 8 + j)];
        c[j] = run;
    }
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t excl = inc - run;
    const uint32_t half = static_cast<uint32_t>((n + 1) >> 1);
    int found = -1;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t v = c[j] + excl;
        const uint32_t before = (j ? c[j - 1] : 0u) + excl;
        cum[pad32(lane * 8 + j)] = v;
        if (v >= half && before < half) found = lane * 8 + j;
    }
    if (found >= 0) sm.ctl->mb = found;
    __syncwarp();
}

// 12-bit: fold the copies into padded totals (conflict-free strided pass), then scan
// contiguous bins per thread.
template <int T>
__device__ __forceinline__ void phase_reduce_scan12(const Shm &sm, int tid, int n) {
    constexpr int B = 4096;
    constexpr int BPT = B / T;  // consecutive bins per thread in the scan
    static_assert(BPT % 4 == 0, "whole 16-byte groups of bins per thread");
    uint4 *h4 = reinterpret_cast<uint4 *>(sm.hist);
    uint32_t *cum = sm.cum;
    const int nc = sm.ncopies;
    // fold the copies (and clear them) four bins at a time, coalesced
    for (int i4 = tid; i4 < B / 4; i4 += T) {
        uint4 s = h4[i4];
        h4[i4] = make_uint4(0u, 0u, 0u, 0u);
        for (int c = 1; c < nc; ++c) {
            const uint4 a = h4[c * (B / 4) + i4];
            h4[c * (B / 4) + i4] = make_uint4(0u, 0u, 0u, 0u);
            s.x += a.x;
            s.y += a.y;
            s.z += a.z;
            s.w += a.w;
        }
        *reinterpret_cast<uint4 *>(cum + Geo<12>::cum_index(4 * i4)) = s;
    }
    named_bar(sm.bar_id, T);
    uint32_t v[BPT];
    uint32_t run = 0;
#pragma unroll
    for (int q = 0; q < BPT / 4; ++q) {
        const uint4 a = *reinterpret_cast<const uint4 *>(cum + Geo<12>::cum_index(tid * BPT + 4 * q));
        run += a.x;
        v[4 * q] = run;
        run += a.y;
        v[4 * q + 1] = run;
        run += a.z;
        v[4 * q + 2] = run;
        run += a.w;
        v[4 * q + 3] = run;
    }
    const uint32_t excl = block_offsets<T>(sm, run, tid);
    const uint32_t half = static_cast<uint32_t>((n + 1) >> 1);
    uint32_t prev = excl;
#pragma unroll
    for (int q = 0; q < BPT / 4; ++q) {
        uint32_t c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            c[k] = v[4 * q + k] + excl;
            if (c[k] >= half && prev < half) sm.ctl->mb = tid * BPT + 4 * q + k;
            prev = c[k];
        }
        *reinterpret_cast<uint4 *>(cum + Geo<12>::cum_index(tid * BPT + 4 * q)) = make_uint4(c[0], c[1], c[2], c[3]);
    }
}

// ------------------------------------------------------------------ phase 4: search
// Smallest v in [0, B) with pred(v), for a monotone pred with pred(B-1) true; one warp.
template <int B, typename Pred>
__device__ __forceinline__ int warp_search(int lane, Pred pred) {
    int base = 0, span = B;
    while (span > 32) {
        const int st = span >> 5;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, pred(base + (lane + 1) * st - 1));
        base += (__ffs(bal) - 1) * st;
        span = st;
    }
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, lane < span && pred(base + lane));
    return base + __ffs(bal) - 1;
}

struct Rep {
    int32_t M, D;
    int32_t cval;     // constant replacement (saturated)
    int32_t t;        // min(ceil(Kq*D / 2^16), sample span + 1)
    int32_t hiv, lov; // threshold replacement above / below (saturated)
    uint32_t sigq;    // 97164 * D
    bool active;      // some sample can be flagged
};

__device__ __forceinline__ int32_t sat_to(int64_t v, int32_t lo, int32_t hi) {
    return v < lo ? lo : (v > hi ? hi : static_cast<int32_t>(v));
}

// Threshold and replacement values of a window with median M and dispersion D (Eq. 1; D is the
// window's MAD, or the median of MADs of Eq. 3).
template <int BITS>
__device__ __forceinline__ RepShared make_rep(int32_t M, int32_t d, int64_t kq, int32_t cval) {
    constexpr int SPAN = Geo<BITS>::kHi - Geo<BITS>::kLo;
    RepShared r;
    r.M = M;
    r.D = d;
    const int64_t kd = kq * static_cast<int64_t>(d);
    const int64_t t = (kd + 65535) >> 16;
    const int64_t c = kd >> 16;
    r.t = static_cast<int32_t>(t < SPAN + 1 ? t : SPAN + 1);
    r.hiv = sat_to(static_cast<int64_t>(r.M) + c, Geo<BITS>::kLo, Geo<BITS>::kHi);
    r.lov = sat_to(static_cast<int64_t>(r.M) - c, Geo<BITS>::kLo, Geo<BITS>::kHi);
    r.sigq = 97164u * static_cast<uint32_t>(d);
    r.active = (d > 0 && t <= SPAN) ? 1u : 0u;  // |x - M| never exceeds the sample span
    r.pad = 0u;
    r.cval = cval;
    if (BITS == 8) {
        const uint32_t tt = static_cast<uint32_t>(r.t > 255 ? 255 : r.t);
        const uint32_t ub = static_cast<uint32_t>(r.M + 129);  // smallest biased value above M
        r.mb4 = static_cast<uint32_t>(r.M + 128) * 0x01010101u;
        r.tlo7 = (tt & 0x7Fu) * 0x01010101u;
        r.tsmall = tt < 128u ? ~0u : 0u;
        r.c4 = (static_cast<uint32_t>(cval) & 0xFFu) * 0x01010101u;
        r.hi4 = (static_cast<uint32_t>(r.hiv) & 0xFFu) * 0x01010101u;
        r.lo4 = (static_cast<uint32_t>(r.lov) & 0xFFu) * 0x01010101u;
        r.ulo7 = (ub & 0x7Fu) * 0x01010101u;
        r.usmall = ub < 128u ? ~0u : 0u;
        r.unone = ub > 255u ? 1u : 0u;
    } else {
        // 12-bit, two samples per word (see rep12_word): u = x + 2048 per 16-bit half
        const uint32_t mb = static_cast<uint32_t>(r.M + 2048);
        const uint32_t tt = static_cast<uint32_t>(r.t);  // <= 4096
        r.mb4 = (mb + tt) * 0x00010001u;                  // upper bound, u >= it flags
        r.tlo7 = (0x8000u + mb - tt) * 0x00010001u;       // 0x8000 + lower bound, u <= it flags
        r.c4 = (static_cast<uint32_t>(cval) & 0xFFFFu) * 0x00010001u;
        r.hi4 = (static_cast<uint32_t>(r.hiv) & 0xFFFFu) * 0x00010001u;
        r.lo4 = (static_cast<uint32_t>(r.lov) & 0xFFFFu) * 0x00010001u;
        r.tsmall = r.ulo7 = r.usmall = r.unone = 0u;
    }
    return r;
}

// One warp: lower median bin, then the MAD, then the threshold and replacement values, written
// to the shared control block.
template <int BITS>
__device__ __forceinline__ void phase_search(const Shm &sm, int n, int lane, int64_t kq, int32_t cval) {
    constexpr int B = Geo<BITS>::kBins;
    const uint32_t *cum = sm.cum;
    const uint32_t half = static_cast<uint32_t>((n + 1) >> 1);
    const int mb = sm.ctl->mb;  // found by its owner thread during the scan
    const int d = warp_search<B>(lane, [&](int dd) {
        const int hi = mb + dd < B - 1 ? mb + dd : B - 1;
        const int lo = mb - dd - 1;
        const uint32_t f = cum[Geo<BITS>::cum_index(hi)] - (lo >= 0 ? cum[Geo<BITS>::cum_index(lo)] : 0u);
        return f >= half;
    });
    if (lane == 0) sm.ctl->rep = make_rep<BITS>(mb - Geo<BITS>::kOffset, d, kq, cval);
}

__device__ __forceinline__ Rep load_rep(const RepShared &s) {
    Rep r;
    r.M = s.M;
    r.D = s.D;
    r.cval = s.cval;
    r.t = s.t;
    r.hiv = s.hiv;
    r.lov = s.lov;
    r.sigq = s.sigq;
    r.active = s.active != 0u;
    return r;
}

// ------------------------------------------------------------------ phase 5: replace
// Bit 7 of byte j of the result is [a_j >= c_j] for unsigned bytes, given clo7 = c & 0x7F7F7F7F
// and csmall = all ones when every c_j < 128 (zero when every c_j >= 128). The subtraction
// cannot borrow across bytes because (a | 0x80) >= 0x80 > (c & 0x7F).
__device__ __forceinline__ uint32_t ge_bytes_msb(uint32_t a, uint32_t clo7, uint32_t csmall) {
    const uint32_t d = (a | 0x80808080u) - clo7;  // bit 7: low 7 bits of a >= low 7 bits of c
    return (a & d) | ((a | d) & csmall);
}

// Per-window constants of the int8 replace pass.
struct Rep8 {
    uint32_t mb4;      // (M + 128) in every byte
    uint32_t tlo7;     // t & 0x7F in every byte
    uint32_t tsmall;   // t < 128 ? ~0 : 0
    uint32_t c4;       // constant replacement in every byte
    uint32_t hi4, lo4; // threshold replacement above / below in every byte
    uint32_t ulo7;     // (M + 129) & 0x7F in every byte (x > M test)
    uint32_t usmall;   // M + 129 < 128 ? ~0 : 0
    uint32_t unone;    // M == 127: nothing lies above the median
};

// 4 int8 samples: returns the output word and sets f to 0xFF in flagged bytes. Noise bytes are
// left 0 here and written by the compacted noise pass.
template <int MODE>
__device__ __forceinline__ uint32_t rep8_word(uint32_t w, const Rep8 &k, uint32_t &f) {
    const uint32_t wb = w ^ 0x80808080u;                  // x + 128 in every byte
    const uint32_t ad = __vabsdiffu4(wb, k.mb4);         // |x - M|
    f = prmt(ge_bytes_msb(ad, k.tlo7, k.tsmall), 0u, 0xBA98u);
    uint32_t rep = 0u;
    if (MODE == 1) rep = k.c4;
    if (MODE == 2) {
        const uint32_t up = k.unone ? 0u : prmt(ge_bytes_msb(wb, k.ulo7, k.usmall), 0u, 0xBA98u);
        rep = (k.hi4 & up) | (k.lo4 & ~up);
    }
    return (w & ~f) | (rep & f);
}

// Two 12-bit samples (int16 halves of w, in range): returns the output word and sets fm to the
// flag bits (bit 15 / bit 31). With u = x + 2048 (12 bits) per half and bounds lo = M + 2048 - t,
// hi = M + 2048 + t: x is flagged iff u >= hi or u <= lo (Eq. 2 with |x - M| >= t). Per half,
// (u | 0x8000) - hi has bit 15 set iff u >= hi, and (0x8000 + lo) - u iff u <= lo; no borrow
// crosses the halves because every operand is below 2^13. A flag moved down to bit 0 / 16 and
// multiplied by 0xFFFF gives the half's select mask.
template <int MODE>
__device__ __forceinline__ uint32_t rep12_word(uint32_t w, uint32_t hi2, uint32_t lo2x, uint32_t c2, uint32_t h2,
                                               uint32_t l2, uint32_t &fm) {
    const uint32_t u = (w ^ 0x08000800u) & 0x0FFF0FFFu;
    const uint32_t up = (u | 0x80008000u) - hi2;   // bit 15 / 31: u >= hi
    const uint32_t dn = lo2x - u;                   // bit 15 / 31: u <= lo
    fm = (up | dn) & 0x80008000u;
    const uint32_t m = (fm >> 15) * 0xFFFFu;  // 0xFFFF in a flagged half
    uint32_t z = 0u;
    if (MODE == 1) z = c2;
    if (MODE == 2) {
        const uint32_t ma = ((up >> 15) & 0x00010001u) * 0xFFFFu;
        z = (h2 & ma) | (l2 & ~ma);
    }
    return (w & ~m) | (z & m);
}

// Mask bits of a 16-sample chunk from its four flag words (0x00/0xFF bytes), sample j -> bit j.
// A flag byte read as signed is -1, so a signed byte dot product with negated powers of two
// (-1, -2, -4, -8 for the first word of a half, -16 .. -128 for the second) packs 8 flags.
__device__ __forceinline__ uint32_t chunk_bits(uint32_t f0, uint32_t f1, uint32_t f2, uint32_t f3) {
    const int lo = __dp4a(static_cast<int>(f1), static_cast<int>(0x80C0E0F0u),
                          __dp4a(static_cast<int>(f0), static_cast<int>(0xF8FCFEFFu), 0));
    const int hi = __dp4a(static_cast<int>(f3), static_cast<int>(0x80C0E0F0u),
                          __dp4a(static_cast<int>(f2), static_cast<int>(0xF8FCFEFFu), 0));
    return static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 8);
}

// Position of the j-th (0-based) set bit of m (j < popc(m)), by halving popcount search.
__device__ __forceinline__ int nth_set_bit(uint32_t m, int j) {
    int pos = 0;
    int c = __popc(m & 0xFFFFu);
    if (j >= c) { j -= c; pos += 16; m >>= 16; }
    c = __popc(m & 0xFFu);
    if (j >= c) { j -= c; pos += 8; m >>= 8; }
    c = __popc(m & 0xFu);
    if (j >= c) { j -= c; pos += 4; m >>= 4; }
    c = __popc(m & 0x3u);
    if (j >= c) { j -= c; pos += 2; m >>= 2; }
    return pos + ((j >= static_cast<int>(m & 1u)) ? 1 : 0);
}

// ------------------------------------------------------------------ output formats
// OUTF 0 writes the input's type; 1 writes fp16 and 2 bf16 (int8 input only). Every sample value
// is exact in either: |x| <= 2048 needs 12 significant bits (fp16 has 11 + 1) and int8 needs 8
// (bf16 has 7 + 1).
template <int BITS, int OUTF>
__device__ __forceinline__ void store_sample(uint8_t *out, int pos, int32_t z) {
    if (OUTF == 1) reinterpret_cast<__half *>(out)[pos] = __int2half_rn(z);
    else if (OUTF == 2) reinterpret_cast<__nv_bfloat16 *>(out)[pos] = __int2bfloat16_rn(z);
    else if (BITS == 8) out[pos] = static_cast<uint8_t>(z);
    else reinterpret_cast<int16_t *>(out)[pos] = static_cast<int16_t>(z);
}

// The 16 int8 output samples of chunk c (v holds them as bytes) in format OUTF: 16-byte stores
// when vec, else one sample at a time. fp16: a biased byte u = x + 128 placed under 0x64 is the
// fp16 1024 + u, and subtracting 1152 leaves x. bf16: u placed in the fp32 2^23 + u, minus
// 2^23 + 128, leaves x as fp32; its bf16 rounding is exact.
template <int OUTF>
__device__ __forceinline__ void store_chunk8(uint8_t *out, int c, const uint4 &v, bool vec) {
    const uint32_t ww[4] = {v.x, v.y, v.z, v.w};
    if constexpr (OUTF == 0) {
        if (vec) {
            __stcs(reinterpret_cast<uint4 *>(out) + c, v);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) out[c * 16 + j] = static_cast<uint8_t>(ww[j >> 2] >> ((j & 3) * 8));
        }
    } else {
        uint32_t h[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t u = ww[q] ^ 0x80808080u;
            if (OUTF == 1) {
                const __half2 off = __half2half2(__ushort_as_half(static_cast<unsigned short>(0x6480u)));  // 1152
                __half2 lo, hi;
                *reinterpret_cast<uint32_t *>(&lo) = __byte_perm(u, 0x64646464u, 0x5140u);
                *reinterpret_cast<uint32_t *>(&hi) = __byte_perm(u, 0x64646464u, 0x7362u);
                lo = __hsub2(lo, off);
                hi = __hsub2(hi, off);
                h[2 * q] = *reinterpret_cast<uint32_t *>(&lo);
                h[2 * q + 1] = *reinterpret_cast<uint32_t *>(&hi);
            } else {
                float f[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    f[k] = __uint_as_float(__byte_perm(u, 0x4B000000u, 0x7540u | k)) - 8388736.0f;
                const __nv_bfloat162 a = __floats2bfloat162_rn(f[0], f[1]);
                const __nv_bfloat162 b = __floats2bfloat162_rn(f[2], f[3]);
                h[2 * q] = *reinterpret_cast<const uint32_t *>(&a);
                h[2 * q + 1] = *reinterpret_cast<const uint32_t *>(&b);
            }
        }
        if (vec) {
            uint4 *o = reinterpret_cast<uint4 *>(out) + 2 * c;
            __stcs(o, make_uint4(h[0], h[1], h[2], h[3]));
            __stcs(o + 1, make_uint4(h[4], h[5], h[6], h[7]));
        } else {
            uint16_t *o = reinterpret_cast<uint16_t *>(out) + 16 * c;
#pragma unroll
            for (int j = 0; j < 16; ++j) o[j] = static_cast<uint16_t>(h[j >> 1] >> ((j & 1) * 16));
        }
    }
}

// Digital noise for the flagged samples of up to four rounds of the warp. Lane l holds in nb
// the 16-bit flag masks of its chunks c0 + k*T (k = 0..3, mask k in bits [16k, 16k+16)). The
// flagged samples are numbered across the warp (an exclusive prefix sum of the per-lane
// counts); in each pass lane q takes sample q, found by a shuffle binary search for the lane
// that owns it and a popcount search for its bit, and all 32 lanes evaluate Philox together.
// The stores go straight to the output; they follow the chunks' own stores in warp order
// (__syncwarp before the call).
template <int BITS, int T, bool PW, class K, int OUTF = 0>
__device__ __forceinline__ void noise_batch(const Win &w, const Rep &r, const K &p, int lane, int c0,
                                            uint64_t nb, Pow &pw) {
    constexpr int CS = Geo<BITS>::kChunkSamples;
    const uint32_t lo = static_cast<uint32_t>(nb), hi = static_cast<uint32_t>(nb >> 32);
    const uint32_t cnt = __popc(lo) + __popc(hi);
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
    const uint32_t excl = inc - cnt;
    for (uint32_t q0 = 0; q0 < total; q0 += 32) {
        const uint32_t q = q0 + lane;
        // owner: the last lane whose first index is <= q (lanes without flags share the next
        // lane's first index, so the search passes over them)
        int L = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const uint32_t e = __shfl_sync(0xFFFFFFFFu, excl, L + step);
            if (e <= q) L += step;
        }
        const uint32_t eL = __shfl_sync(0xFFFFFFFFu, excl, L);
        const uint32_t loL = __shfl_sync(0xFFFFFFFFu, lo, L);
        const uint32_t hiL = __shfl_sync(0xFFFFFFFFu, hi, L);
        const int cL = __shfl_sync(0xFFFFFFFFu, c0, L);
        if (q < total) {
            const int j = static_cast<int>(q - eL);
            const int clo = __popc(loL);
            const bool inlo = j < clo;
            const int bp = (inlo ? 0 : 32) + nth_set_bit(inlo ? loL : hiL, inlo ? j : j - clo);
            const int pos = (cL + (bp >> 4) * T) * CS + (bp & 15);
            const int32_t z = noise_value(r.M, r.sigq, p, w.sid, w.abs_idx + pos, Geo<BITS>::kLo, Geo<BITS>::kHi);
            store_sample<BITS, OUTF>(w.out, pos, z);
            if (PW) pw.z += static_cast<uint32_t>(z * z);
        }
    }
}

// Digital noise, replace pass: the warp numbers its flagged samples of this round, reserves that
// many list entries with one shared atomic, and each lane writes its positions. Windows of
// 65536 samples (position 65535 would equal the skip mark) and rounds that do not fit in the
// list take the per-warp path at once; list entries reserved beyond the written ones are
// marked skipped. Called by all lanes of the warp with the round's chunk c and flag bits.
template <int BITS, int T, bool PW, class K, int OUTF = 0>
__device__ __forceinline__ void noise_append(const Shm &sm, const Win &w, const Rep &r, const K &p, int lane,
                                             int c, uint32_t bits, uint32_t *nlc, Pow &pw) {
    constexpr int CS = Geo<BITS>::kChunkSamples;
    if (!__any_sync(0xFFFFFFFFu, bits != 0u)) return;
    const uint32_t cnt = __popc(bits);
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
    const bool listed = sm.nlist != nullptr && w.n < 65536;
    uint32_t base = kNoiseList;
    if (listed && lane == 31) base = atomicAdd(nlc, total);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    if (base + total <= static_cast<uint32_t>(kNoiseList)) {
        uint32_t off = base + inc - cnt;
        for (uint32_t m = bits; m; m &= m - 1u) sm.nlist[off++] = static_cast<uint16_t>(c * CS + __ffs(m) - 1);
        return;
    }
    for (uint32_t i = base + lane; i < static_cast<uint32_t>(kNoiseList); i += 32) sm.nlist[i] = kNoiseSkip;
    __syncwarp();  // the round's chunk stores come first
    noise_batch<BITS, T, PW, K, OUTF>(w, r, p, lane, c, static_cast<uint64_t>(bits), pw);
}

// Digital noise, after the group barrier that follows the replace pass: every thread of the
// group evaluates Philox for a share of the list and stores the value over the chunk's output.
template <int BITS, int T, bool PW, class K, int OUTF = 0>
__device__ __forceinline__ void noise_list(const Shm &sm, const Win &w, const Rep &r, const K &p, int tid,
                                           uint32_t *nlc, Pow &pw) {
    if (sm.nlist == nullptr) return;
    const uint32_t n = min(*nlc, static_cast<uint32_t>(kNoiseList));
    uint32_t i = static_cast<uint32_t>(tid);
    // two entries at a time: the two Philox chains are independent, so their rounds interleave
    // and fill each other's dependency stalls (60 streams of 2^25 12-bit samples in 8192-sample
    // windows, a quarter of them flagged: 4.60 -> 4.53 ms per call)
    for (; i + T < n; i += 2 * T) {
        const uint32_t pa = sm.nlist[i], pb = sm.nlist[i + T];
        const int32_t za = noise_value(r.M, r.sigq, p, w.sid, w.abs_idx + pa, Geo<BITS>::kLo, Geo<BITS>::kHi);
        const int32_t zb = noise_value(r.M, r.sigq, p, w.sid, w.abs_idx + pb, Geo<BITS>::kLo, Geo<BITS>::kHi);
        if (pa != kNoiseSkip) {
            store_sample<BITS, OUTF>(w.out, pa, za);
            if (PW) pw.z += static_cast<uint32_t>(za * za);
        }
        if (pb != kNoiseSkip) {
            store_sample<BITS, OUTF>(w.out, pb, zb);
            if (PW) pw.z += static_cast<uint32_t>(zb * zb);
        }
    }
    for (; i < n; i += T) {
        const uint32_t pos = sm.nlist[i];
        if (pos == kNoiseSkip) continue;
        const int32_t z = noise_value(r.M, r.sigq, p, w.sid, w.abs_idx + pos, Geo<BITS>::kLo, Geo<BITS>::kHi);
        store_sample<BITS, OUTF>(w.out, pos, z);
        if (PW) pw.z += static_cast<uint32_t>(z * z);
    }
}

// Digital noise (int8), replace pass: the warp appends one list entry per chunk of its round
// that holds a flagged sample, (chunk << 16) | the chunk's 16 flag bits, at places reserved
// with one shared atomic on the entry count *nlc. The list has room for every chunk of a stage.
// Called by all lanes of the warp (bits = 0 for a lane without a chunk).
__device__ __forceinline__ void noise_note8(const Shm &sm, int lane, int c, uint32_t bits, uint32_t *nlc) {
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, bits != 0u);
    if (bal == 0u) return;
    uint32_t base = 0u;
    if (lane == 0) base = atomicAdd(nlc, static_cast<uint32_t>(__popc(bal)));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (bits)
        reinterpret_cast<uint32_t *>(sm.nlist)[base + __popc(bal & ((1u << lane) - 1u))] =
            (static_cast<uint32_t>(c) << 16) | bits;
}

// Digital noise (int8), after the replace pass and a group barrier: the n entries noted by
// noise_note8, in any order (a sample's noise depends only on its absolute index). Warp w
// expands entries 2w and 2w + 1, then 2w + 2NW and 2w + 2NW + 1, and so on: each half-warp
// takes one entry and its lane j tests flag bit j. The flagged positions go into the warp's
// ring, compacted by a ballot and a prefix popcount, and whenever 32 are waiting every lane
// takes one and emit(pos) evaluates and stores its noise. Fewer than 32 are left for the end.
// Every lane does Philox work in every batch but the last, however the flags are spread over
// the chunks, and the chunks are shared out evenly between the warps.
template <int T, class Emit>
__device__ __forceinline__ void noise_expand8(const Shm &sm, uint32_t n, int tid, Emit &&emit) {
    constexpr uint32_t NW = T / 32;
    constexpr uint32_t RM = kNoiseRing - 1;
    const int lane = tid & 31;
    const uint32_t warp = static_cast<uint32_t>(tid >> 5);
    const uint32_t *list = reinterpret_cast<const uint32_t *>(sm.nlist);
    uint32_t *ring = sm.nring + warp * kNoiseRing;
    const uint32_t j = static_cast<uint32_t>(lane & 15);
    const uint32_t below = (1u << lane) - 1u;
    uint32_t head = 0u, tail = 0u;  // positions taken / queued so far (tail - head < 32 between steps)
    for (uint32_t e0 = 2u * warp; e0 < n; e0 += 2u * NW) {
        const uint32_t e = e0 + static_cast<uint32_t>(lane >> 4);
        const uint32_t ent = e < n ? list[e] : 0u;
        const bool fl = ((ent >> j) & 1u) != 0u;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, fl);
        if (fl) ring[(tail + static_cast<uint32_t>(__popc(bal & below))) & RM] = (ent >> 16) * 16u + j;
        tail += static_cast<uint32_t>(__popc(bal));
        if (tail - head >= 32u) {
            __syncwarp();
            const uint32_t pos = ring[(head + static_cast<uint32_t>(lane)) & RM];
            __syncwarp();  // read before the next step refills the slot
            head += 32u;
            emit(pos);
        }
    }
    if (tail != head) {
        __syncwarp();
        if (static_cast<uint32_t>(lane) < tail - head) emit(ring[(head + static_cast<uint32_t>(lane)) & RM]);
    }
}

// Digital noise (int8) of one window, after its replace pass noted its chunks in the list (*nlc
// entries): one group barrier, then noise_expand8. Every store is checked against the window's
// length.
template <int T, bool PW, class K, int OUTF = 0>
__device__ __forceinline__ void noise_deferred8(const Shm &sm, const Win &w, const Rep &r, const K &p, int tid,
                                                const uint32_t *nlc, Pow &pw) {
    named_bar(sm.bar_id, T);  // every entry of the window is in the list
    noise_expand8<T>(sm, *nlc, tid, [&](uint32_t pos) {
        if (pos >= static_cast<uint32_t>(w.n)) return;
        const int32_t z = noise_value(r.M, r.sigq, p, w.sid, w.abs_idx + pos, Geo<8>::kLo, Geo<8>::kHi);
        store_sample<8, OUTF>(w.out, static_cast<int>(pos), z);
        if (PW) pw.z += static_cast<uint32_t>(z * z);
    });
}

// Sum of squares of the bytes of w kept by keep (0xFF per kept byte), as signed int8 samples.
__device__ __forceinline__ uint32_t sq4(uint32_t w, uint32_t keep) {
    const int32_t v = static_cast<int32_t>(w & keep);
    return static_cast<uint32_t>(__dp4a(v, v, 0));
}

// rsrc: the shared record r was loaded from (its int8 constants are read from there). FO (8-bit
// in-place form): chunks without a flagged sample are not stored, and in noise mode no chunk is
// (the noise pass writes every flagged sample). PAIR (the split-warp form's replace warps):
// full rounds go two at a time.
template <int BITS, int MODE, int T, bool PW, class K, int OUTF = 0, bool FO = false, bool PAIR = false>
__device__ __forceinline__ uint32_t phase_replace(const Shm &sm, const Win &w, const Rep &r, const K &p,
                                                  int tid, uint32_t *nlc, Pow &pw, const RepShared *rsrc) {
    constexpr int BPS = Geo<BITS>::kBps;
    const int lane = tid & 31, warp = tid >> 5;
    const int nbytes = w.n * BPS;
    const int nfull = nbytes >> 4;
    const int nchunks = (nbytes + 15) >> 4;
    const uint4 *d4 = reinterpret_cast<const uint4 *>(w.data);
    uint32_t flagged = 0;
    if (BITS == 8) {
        const uint4 *rq = reinterpret_cast<const uint4 *>(rsrc);
        const uint4 q2 = rq[2], q3 = rq[3], q4 = rq[4];
        Rep8 k;
        k.mb4 = q2.x;
        k.tlo7 = q2.y;
        k.tsmall = q2.z;
        k.c4 = q2.w;
        k.hi4 = q3.x;
        k.lo4 = q3.y;
        k.ulo7 = q3.z;
        k.usmall = q3.w;
        k.unone = q4.x;
        uint16_t *mk = reinterpret_cast<uint16_t *>(w.mask);
        int base = warp * 32;
        if (r.active && w.vec && mk) {
            // rounds in which all 32 chunks of the warp are full: no bounds checks
            auto full_round = [&](int c, uint4 v) {
                if (PW) pw.x += sq4(v.x, ~0u) + sq4(v.y, ~0u) + sq4(v.z, ~0u) + sq4(v.w, ~0u);
                uint32_t f0, f1, f2, f3;
                v.x = rep8_word<MODE>(v.x, k, f0);
                v.y = rep8_word<MODE>(v.y, k, f1);
                v.z = rep8_word<MODE>(v.z, k, f2);
                v.w = rep8_word<MODE>(v.w, k, f3);
                const uint32_t bits = chunk_bits(f0, f1, f2, f3);
                if (!FO || (MODE != 3 && bits)) store_chunk8<OUTF>(w.out, c, v, true);
                if (PW) pw.z += sq4(v.x, ~0u) + sq4(v.y, ~0u) + sq4(v.z, ~0u) + sq4(v.w, ~0u);
                mk[c] = static_cast<uint16_t>(bits);
                flagged += __popc(bits);
                if (MODE == 3) noise_note8(sm, lane, c, bits, nlc);
            };
            // two rounds at a time, both chunks loaded before either is replaced (the loads of the
            // second overlap the first's arithmetic): zero, constant and threshold in the split-warp
            // form (1.618 -> 1.607 ms for a zero-mode call over 60 streams of 2^26 int8 samples in
            // 16384-sample windows; in the joint form the fp16 output lost 6 % and the digital copy
            // and the Median-of-MAD apply pass 1 %)
            if (PAIR && MODE != 3) {
                for (; base + T + 32 <= nfull; base += 2 * T) {
                    const uint4 va = d4[base + lane];
                    const uint4 vb = d4[base + T + lane];
                    full_round(base + lane, va);
                    full_round(base + T + lane, vb);
                }
            }
            for (; base + 32 <= nfull; base += T) full_round(base + lane, d4[base + lane]);
        }
        // warp-uniform rounds: lane handles chunk base + lane
        for (; base < nchunks; base += T) {
            const int c = base + lane;
            uint32_t bits = 0;
            if (c < nchunks) {
                uint4 v = d4[c];
                const uint4 vin = v;
                if (r.active) {
                    uint32_t f0, f1, f2, f3;
                    v.x = rep8_word<MODE>(v.x, k, f0);
                    v.y = rep8_word<MODE>(v.y, k, f1);
                    v.z = rep8_word<MODE>(v.z, k, f2);
                    v.w = rep8_word<MODE>(v.w, k, f3);
                    bits = chunk_bits(f0, f1, f2, f3);
                }
                if (c < nfull) {
                    if (!FO || (MODE != 3 && bits)) store_chunk8<OUTF>(w.out, c, v, w.vec);
                } else {  // ragged last chunk of the window
                    const int valid = nbytes - c * 16;
                    bits &= (1u << valid) - 1u;
                    const uint32_t ww[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (j < valid && (!FO || (MODE != 3 && ((bits >> j) & 1u))))
                            store_sample<8, OUTF>(w.out, c * 16 + j, static_cast<int8_t>(ww[j >> 2] >> ((j & 3) * 8)));
                }
                if (PW) {
                    // the samples of the window only: the ragged chunk's tail bytes are not its own
                    const int valid = c < nfull ? 16 : nbytes - c * 16;
                    uint32_t kp[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int nv = valid - 4 * q;
                        kp[q] = nv >= 4 ? ~0u : (nv <= 0 ? 0u : (1u << (8 * nv)) - 1u);
                    }
                    pw.x += sq4(vin.x, kp[0]) + sq4(vin.y, kp[1]) + sq4(vin.z, kp[2]) + sq4(vin.w, kp[3]);
                    pw.z += sq4(v.x, kp[0]) + sq4(v.y, kp[1]) + sq4(v.z, kp[2]) + sq4(v.w, kp[3]);
                }
                flagged += __popc(bits);
                if (mk) mk[c] = static_cast<uint16_t>(bits);
            }
            if (MODE == 3) noise_note8(sm, lane, c, bits, nlc);
        }
        if (mk) {
            for (int c = nchunks + tid; c < 2 * w.mask_words; c += T) mk[c] = 0;
        }
    } else {
        uint8_t *mk = reinterpret_cast<uint8_t *>(w.mask);
        const int32_t t = r.t;
        const RepShared k12 = *rsrc;
        for (int base = warp * 32; base < nchunks; base += T) {
            const int c = base + lane;
            uint32_t bits = 0;
            if (c < nchunks) {
                const uint4 v = d4[c];
                uint32_t ww[4] = {v.x, v.y, v.z, v.w};
                const int valid = c < nfull ? 8 : ((nbytes - c * 16) >> 1);  // samples in the window
                if (!PW) {
                    if (r.active) {
                        uint32_t f[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) ww[q] = rep12_word<MODE>(ww[q], k12.mb4, k12.tlo7, k12.c4, k12.hi4,
                                                                             k12.lo4, f[q]);
                        // flag bits 15 / 31 of the four words -> bits 0..7 (sample order)
                        const uint32_t g0 = __byte_perm(f[0], f[1], 0x7531u) & 0x80808080u;
                        const uint32_t g1 = __byte_perm(f[2], f[3], 0x7531u) & 0x80808080u;
                        bits = ((g0 * 0x00204081u) >> 28) | (((g1 * 0x00204081u) >> 28) << 4);
                        // samples past the window (a ragged last chunk) are neither flagged nor stored
                        if (valid < 8) bits &= (1u << valid) - 1u;
                    }
                } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int sh = (j & 1) * 16;
                    const int32_t x = static_cast<int16_t>((ww[j >> 1] >> sh) & 0xFFFFu);
                    const int32_t ad = x > r.M ? x - r.M : r.M - x;
                    const bool fl = r.active && ad >= t && j < valid;
                    int32_t zo = x;
                    if (fl) {
                        int32_t z = 0;
                        if (MODE == 1) z = r.cval;
                        else if (MODE == 2) z = x > r.M ? r.hiv : r.lov;
                        ww[j >> 1] = (ww[j >> 1] & ~(0xFFFFu << sh)) | ((static_cast<uint32_t>(z) & 0xFFFFu) << sh);
                        bits |= 1u << j;
                        zo = z;
                    }
                    if (PW && j < valid) {
                        pw.x += static_cast<uint32_t>(x * x);
                        pw.z += static_cast<uint32_t>(zo * zo);
                    }
                }
                }
                flagged += __popc(bits);
                if (OUTF == 1) {  // fp16: each int16 pair converted in place, same bytes per chunk
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const __half2 hv = __halves2half2(__short2half_rn(static_cast<short>(ww[q] & 0xFFFFu)),
                                                          __short2half_rn(static_cast<short>(ww[q] >> 16)));
                        ww[q] = *reinterpret_cast<const uint32_t *>(&hv);
                    }
                }
                if (w.vec && c < nfull) {
                    __stcs(reinterpret_cast<uint4 *>(w.out + c * 16), make_uint4(ww[0], ww[1], ww[2], ww[3]));
                } else {
                    uint16_t *o = reinterpret_cast<uint16_t *>(w.out);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j < valid) o[c * 8 + j] = static_cast<uint16_t>((ww[j >> 1] >> ((j & 1) * 16)) & 0xFFFFu);
                }
                if (mk) mk[c] = static_cast<uint8_t>(bits);
            }
            if (MODE == 3) noise_append<12, T, PW, K, OUTF>(sm, w, r, p, lane, c, bits, nlc, pw);
        }
        if (mk) {
            for (int c = nchunks + tid; c < 4 * w.mask_words; c += T) mk[c] = 0;
        }
    }
    return flagged;
}

// ------------------------------------------------------------------ one window
// All T threads of the group call this; the histogram must be zero on entry and is zero again
// when the first warp leaves the reduce phase. Uses the group's named barrier three times
// (after the histogram, inside the scan, after the cumulative counts) plus once after the
// search. There is no barrier at the end: each warp adds its flag count and marks itself done,
// and the last warp of the window (window parity `par`) writes the count, median and MAD to
// slot `widx` of the segment and, when release_bar != 0, releases the stage through it.
// `stage_ok` is this thread's result of waiting for the stage (false: timed out); the first
// barrier combines it, and the function returns false if any thread of the group timed out.
//
// MODE & 3 is the replacement mode (rfi_mode); the other bits select a form of the pass. For
// the Median-of-MAD variant (Eq. 3), kModeStats runs phases 1-4 only and writes M and D, and
// kModeApply skips phases 1-4, reads the window's M from sg.med and its dispersion from sg.mad
// and runs phase 5 (amd, when given, holds the window's {M, dispersion} in shared memory).
// kModePower also sums x^2 and z^2 over the window into sg.power.
template <int BITS, int MODE, int T, int ROWB>
__device__ bool process_window(const Shm &sm, const Win &w, const Seg &sg, int64_t widx, const Params &p,
                               int tid, int par, uint32_t release_bar, bool stage_ok, RowSums &rs,
                               const int2 *amd = nullptr, const Seg *vsegs = nullptr) {
    constexpr int NW = T / 32;
    constexpr bool STATS = (MODE & kModeStats) != 0;
    constexpr bool APPLY = (MODE & kModeApply) != 0;
    constexpr bool PW = (MODE & kModePower) != 0;
    constexpr bool COPIES = (MODE & kModeCopies) != 0;
    constexpr int OUTF = (MODE & kModeF16) ? 1 : ((MODE & kModeBF16) ? 2 : 0);
    constexpr int RMODE = MODE & 3;
    const int lane = tid & 31;
    if (STATS) {
        // Estimation only (the first pass of Eq. 3): M and D of the window. Nothing reads the
        // stage after the histogram, so the tile's last window releases it there; the search
        // warp writes M and D itself while the other warps go on to the next window. sg lives in
        // the stage's descriptor, which the copy warp rewrites once the stage is released: its
        // output pointers are taken first.
        int32_t *const med = sg.med, *const mad = sg.mad;
        if (stage_ok) phase_histogram<BITS, T, ROWB>(sm, w, tid, par);
        if (named_bar_or(sm.bar_id, T, !stage_ok)) return false;
        if (tid == 0 && release_bar) mbar_arrive(release_bar);
        // int8: the counts go to one warp, which scans them and searches while the other warps
        // start the next window (one group barrier fewer than a block-wide scan)
        if (BITS == 8) phase_reduce8_counts<T, ROWB>(sm, tid, rs);
        else phase_reduce_scan12<T>(sm, tid, w.n);
        named_bar(sm.bar_id, T);
        if (tid < 32) {
            if (BITS == 8) phase_scan8_warp(sm, w.n, lane);
            phase_search<BITS>(sm, w.n, lane, p.kq, p.cval);
            if (lane == 0) {  // the lane that wrote the record
                if (med) med[widx] = sm.ctl->rep.M;
                if (mad) mad[widx] = sm.ctl->rep.D;
                if (BITS == 12 && atomicExch(&sm.ctl->err[par], 0u)) atomicOr(p.status, kStatusSampleRange);
            }
        }
        return true;
    }
    if (!APPLY) {
        if (stage_ok) phase_histogram<BITS, T, ROWB>(sm, w, tid, par);
        if (named_bar_or(sm.bar_id, T, !stage_ok)) return false;
        if (BITS == 8) phase_reduce8_counts<T, ROWB>(sm, tid, rs);
        else phase_reduce_scan12<T>(sm, tid, w.n);
        named_bar(sm.bar_id, T);
        if (tid < 32) {
            if (BITS == 8) phase_scan8_warp(sm, w.n, lane);
            phase_search<BITS>(sm, w.n, lane, p.kq, p.cval);
        }
    } else {
        // every thread has read the previous window's values before this barrier
        if (named_bar_or(sm.bar_id, T, !stage_ok)) return false;
        if (tid == 0) {  // from the stage's copy (amd) when the copy warp brought it along
            const int2 md = amd ? *amd : make_int2(sg.med[widx], sg.mad[widx]);
            sm.ctl->rep = make_rep<BITS>(md.x, md.y, p.kq, p.cval);
        }
    }
    named_bar(sm.bar_id, T);
    const Rep r = load_rep(sm.ctl->rep);
    uint32_t f = 0;
    Pow pw = {0u, 0u};
    const KeysPre key{p};
    if (!STATS && !COPIES)
        f = phase_replace<BITS, RMODE, T, PW, KeysPre, OUTF, (MODE & kModeFlaggedOnly) != 0>(
            sm, w, r, key, tid, &sm.ctl->ncount[par], pw, &sm.ctl->rep);
    if (!STATS && !COPIES && RMODE == 3) {
        if (BITS == 8) {
            noise_deferred8<T, PW, KeysPre, OUTF>(sm, w, r, key, tid, &sm.ctl->ncount[par], pw);
        } else {
            named_bar(sm.bar_id, T);  // every flagged position of the window is in the list
            noise_list<BITS, T, PW, KeysPre, OUTF>(sm, w, r, key, tid, &sm.ctl->ncount[par], pw);
        }
    }
    if (COPIES) {
        // every variant's values from the window's M and D, then its replace pass
        if (tid < params_nvar(p)) {
            const Variant vr = params_var(p)[tid];
            sm.cp->vrep[tid] = make_rep<BITS>(r.M, r.D, vr.kq, vr.cval);
        }
        named_bar(sm.bar_id, T);
        for (int v = 0; v < params_nvar(p); ++v) {
            const Variant vr = params_var(p)[v];
            const Seg &sv = vsegs[static_cast<int64_t>(v) * params_seg_stride(p)];
            Win wv = w;
            wv.out = sv.out + widx * sv.W * Geo<BITS>::kBps;
            wv.mask = sv.mask ? sv.mask + widx * sv.mask_words : nullptr;
            wv.vec = sv.vec != 0;
            const Rep rv = load_rep(sm.cp->vrep[v]);
            const KeysSeed vkey{static_cast<uint32_t>(vr.seed), static_cast<uint32_t>(vr.seed >> 32)};
            uint32_t *nc = &sm.cp->ncount[2 * v + par];
            uint32_t fv;
            switch (vr.mode) {
                case 0: fv = phase_replace<BITS, 0, T, false>(sm, wv, rv, vkey, tid, nc, pw, &sm.cp->vrep[v]); break;
                case 1: fv = phase_replace<BITS, 1, T, false>(sm, wv, rv, vkey, tid, nc, pw, &sm.cp->vrep[v]); break;
                case 2: fv = phase_replace<BITS, 2, T, false>(sm, wv, rv, vkey, tid, nc, pw, &sm.cp->vrep[v]); break;
                default:
                    fv = phase_replace<BITS, 3, T, false>(sm, wv, rv, vkey, tid, nc, pw, &sm.cp->vrep[v]);
                    if (BITS == 8) {
                        noise_deferred8<T, false>(sm, wv, rv, vkey, tid, nc, pw);
                    } else {
                        named_bar(sm.bar_id, T);
                        noise_list<BITS, T, false>(sm, wv, rv, vkey, tid, nc, pw);
                    }
                    // the noise work area and the first indices are reused by the next variant
                    if (v + 1 < params_nvar(p)) named_bar(sm.bar_id, T);
                    break;
            }
            fv = __reduce_add_sync(0xFFFFFFFFu, fv);
            if (lane == 0 && fv) atomicAdd(&sm.cp->vcount[v][par], fv);
        }
    }
    f = __reduce_add_sync(0xFFFFFFFFu, f);
    unsigned long long px = 0ull, pz = 0ull;
    if (PW) {  // warp sums in two 16-bit halves, so that no partial sum overflows 32 bits
        px = (static_cast<unsigned long long>(__reduce_add_sync(0xFFFFFFFFu, pw.x >> 16)) << 16) +
             __reduce_add_sync(0xFFFFFFFFu, pw.x & 0xFFFFu);
        pz = (static_cast<unsigned long long>(__reduce_add_sync(0xFFFFFFFFu, pw.z >> 16)) << 16) +
             __reduce_add_sync(0xFFFFFFFFu, pw.z & 0xFFFFu);
    }
    if (lane == 0) {
        if (f) atomicAdd(&sm.ctl->count[par], f);
        if (PW) {
            atomicAdd(&sm.ctl->pw[par][0], px);
            atomicAdd(&sm.ctl->pw[par][1], pz);
        }
        __threadfence_block();
        if (atomicAdd(&sm.ctl->done[par], 1u) == NW - 1) {
            // last warp of this window: every count is in and every read of the stage is done
            __threadfence_block();
            const uint32_t cnt = atomicExch(&sm.ctl->count[par], 0u);
            sm.ctl->done[par] = 0u;
            if (RMODE == 3 && !COPIES) sm.ctl->ncount[par] = 0u;  // every warp has read it
            if (COPIES) {
                for (int v = 0; v < params_nvar(p); ++v) {
                    const uint32_t cv = atomicExch(&sm.cp->vcount[v][par], 0u);
                    sm.cp->ncount[2 * v + par] = 0u;
                    const Seg &sv = vsegs[static_cast<int64_t>(v) * params_seg_stride(p)];
                    if (sv.counts) sv.counts[widx] = cv;
                    sm.ctl->flagged += cv;
                }
            }
            if (PW) {
                const unsigned long long sx = atomicExch(&sm.ctl->pw[par][0], 0ull);
                const unsigned long long sz = atomicExch(&sm.ctl->pw[par][1], 0ull);
                if (sg.power) {
                    sg.power[2 * widx] = sx;
                    sg.power[2 * widx + 1] = sz;
                }
            }
            if (!COPIES && sg.counts) sg.counts[widx] = cnt;
            if (!APPLY && sg.med) sg.med[widx] = r.M;
            if (!APPLY && sg.mad) sg.mad[widx] = r.D;
            sm.ctl->flagged += cnt;
            if (BITS == 12 && atomicExch(&sm.ctl->err[par], 0u)) atomicOr(p.status, kStatusSampleRange);
            if (release_bar) mbar_arrive(release_bar);
        }
    }
    return true;
}

// ------------------------------------------------------------------ replace pass over a tile
// Eq. 1 and Eq. 2 over a whole tile of nw full int8 windows of one segment, W = 2^lw samples
// each, 16-byte aligned, window k (of the tile) with the thresholds reps[k] already in shared
// memory: the replace pass over all of the tile's chunks (a warp's round of 32 chunks lies in
// one window, whose flag count takes one shared atomic), then the digital noise of the listed
// chunks as in noise_deferred8, each sample taking its window's M and spread. The last warp
// writes the windows' counts from cnt (and zeroes them) and, when release_bar != 0, releases
// the stage. Windows start at window w0 of the segment.
template <int RMODE, int T>
__device__ void replace_tile8(const Shm &sm, const uint8_t *stage, const Seg &sg, uint32_t w0, int nw, int lw,
                              const RepShared *reps, uint32_t *cnt, const Params &p, int tid, int par,
                              uint32_t release_bar) {
    constexpr int NW = T / 32;
    const int lane = tid & 31, warp = tid >> 5;
    const int lcw = lw - 4;  // log2 of the chunks per window
    const int nchunks = nw << lcw;
    const uint4 *d4 = reinterpret_cast<const uint4 *>(stage);
    uint8_t *out = sg.out + (static_cast<int64_t>(w0) << lw);
    uint16_t *mk = sg.mask ? reinterpret_cast<uint16_t *>(sg.mask + static_cast<int64_t>(w0) * sg.mask_words)
                           : nullptr;
    for (int c0 = warp * 32; c0 < nchunks; c0 += T) {
        const int k = c0 >> lcw;
        const RepShared &rk = reps[k];
        const uint4 *rq = reinterpret_cast<const uint4 *>(&rk);
        const uint4 q2 = rq[2], q3 = rq[3], q4 = rq[4];
        Rep8 k8;
        k8.mb4 = q2.x;
        k8.tlo7 = q2.y;
        k8.tsmall = q2.z;
        k8.c4 = q2.w;
        k8.hi4 = q3.x;
        k8.lo4 = q3.y;
        k8.ulo7 = q3.z;
        k8.usmall = q3.w;
        k8.unone = q4.x;
        const int c = c0 + lane;
        uint4 v = d4[c];
        uint32_t bits = 0;
        if (rk.active) {
            uint32_t f0, f1, f2, f3;
            v.x = rep8_word<RMODE>(v.x, k8, f0);
            v.y = rep8_word<RMODE>(v.y, k8, f1);
            v.z = rep8_word<RMODE>(v.z, k8, f2);
            v.w = rep8_word<RMODE>(v.w, k8, f3);
            bits = chunk_bits(f0, f1, f2, f3);
        }
        store_chunk8<0>(out, c, v, true);
        if (mk) mk[c] = static_cast<uint16_t>(bits);
        if (RMODE == 3) noise_note8(sm, lane, c, bits, &sm.ctl->ncount[par]);
        const uint32_t wf = __reduce_add_sync(0xFFFFFFFFu, __popc(bits));
        if (lane == 0 && wf) atomicAdd(&cnt[k], wf);
    }

    if (RMODE == 3) {
        named_bar(sm.bar_id, T);  // every entry of the tile is in the list
        const KeysPre key{p};
        const int64_t abs0 = sg.abs0 + (static_cast<int64_t>(w0) << lw);
        noise_expand8<T>(sm, sm.ctl->ncount[par], tid, [&](uint32_t pos) {
            const RepShared &rk = reps[pos >> lw];
            const int32_t z = noise_value(rk.M, rk.sigq, key, sg.stream_id, abs0 + pos, Geo<8>::kLo, Geo<8>::kHi);
            out[pos] = static_cast<uint8_t>(z);
        });
    }

    if (lane == 0) {
        __threadfence_block();
        if (atomicAdd(&sm.ctl->done[par], 1u) == NW - 1) {
            // last warp of the tile: every count is in and every read of the stage is done
            __threadfence_block();
            sm.ctl->done[par] = 0u;
            if (RMODE == 3) sm.ctl->ncount[par] = 0u;  // every warp has read it
            unsigned long long tot = 0ull;
            for (int k = 0; k < nw; ++k) {
                const uint32_t ck = cnt[k];
                cnt[k] = 0u;
                if (sg.counts) sg.counts[w0 + k] = ck;
                tot += ck;
            }
            sm.ctl->flagged += tot;
            if (release_bar) mbar_arrive(release_bar);
        }
    }
}

// ------------------------------------------------------------------ apply pass over a tile
// The apply pass (Eq. 1 and Eq. 2 around each window's given M with its given dispersion, as
// for the median of MADs of Eq. 3) over a whole tile of nw full int8 windows of one segment,
// W = 2^lw >= 512 samples each, 16-byte aligned: one barrier for the tile's thresholds (thread
// k builds window k's), then replace_tile8. Against one window at a time this saves three
// barriers per window and keeps every thread busy on windows of 4096 samples, which give 256
// threads one chunk each.
template <int MODE, int T>
__device__ bool process_tile_apply8(const Shm &sm, const uint8_t *stage, const Tile &tl, const Seg &sg,
                                    const int2 *amd, const Params &p, int tid, int par, int lw,
                                    uint32_t release_bar, bool stage_ok) {
    const int nw = static_cast<int>(tl.nw);
    // every thread has finished the previous tile or window (its thresholds, counts, noise
    // work area) before this barrier
    if (named_bar_or(sm.bar_id, T, !stage_ok)) return false;
    RepShared *reps = sm.at->rep;
    if (tid < nw) reps[tid] = make_rep<8>(amd[tid].x, amd[tid].y, p.kq, p.cval);
    named_bar(sm.bar_id, T);
    replace_tile8<MODE & 3, T>(sm, stage, sg, tl.w0, nw, lw, reps, sm.at->count, p, tid, par, release_bar);
    return true;
}

// ------------------------------------------------------------------ multi-window tiles
// Histogram of up to K windows of 2^lw samples at once: window slot g (< nw) is counted by the
// 32/K lanes (32/K)g .. of every warp into their own columns of the lane-striped table, so the
// atomics stay conflict-free and the slots never mix.
template <int T, int K>
__device__ __forceinline__ void hist8_multi(const Shm &sm, const uint8_t *stage, int lw, int nw, int tid) {
    constexpr int LPS = 32 / K;  // lanes per slot
    constexpr int TS = T / K;    // threads per slot
    const int lane = tid & 31, warp = tid >> 5;
    const int g = lane / LPS;
    if (g >= nw) return;
    const int i = warp * LPS + (lane % LPS);
    const uint32_t lb = sm.hist_s + 4u * lane;
    const uint4 *d4 = reinterpret_cast<const uint4 *>(stage + (g << lw));
    const int nch = 1 << (lw - 4);
    int c = i;
    for (; c + TS < nch; c += 2 * TS) {
        const uint4 a = d4[c], b = d4[c + TS];
        hist8_word<128>(lb, a.x); hist8_word<128>(lb, a.y); hist8_word<128>(lb, a.z); hist8_word<128>(lb, a.w);
        hist8_word<128>(lb, b.x); hist8_word<128>(lb, b.y); hist8_word<128>(lb, b.z); hist8_word<128>(lb, b.w);
    }
    if (c < nch) {
        const uint4 a = d4[c];
        hist8_word<128>(lb, a.x); hist8_word<128>(lb, a.y); hist8_word<128>(lb, a.z); hist8_word<128>(lb, a.w);
    }
}

// Counts of every slot from the table, which is zeroed as it is read (the 128-byte row of raw
// byte u holds lane l's count at word l; a slot's lanes are 8/K of the row's eight 16-byte
// groups). The eight threads tid & ~7 .. tid | 7 read the eight groups of the same row, so the
// reads and clears are free of bank conflicts; with four slots, thread pairs combine their
// groups by a shuffle. Counts go to 16-bit arrays, 264 entries per slot (slot g's array starts
// on bank 4g, so the stores of one row's slots do not collide either).
template <int T, int K>
__device__ __forceinline__ void reduce8_multi(const Shm &sm, int tid) {
    static_assert(K == 4 || K == 8, "four or eight window slots");
    constexpr int RPT = 256 / (T / 8);  // rows per thread
    const int p = tid & 7;
    const int r0 = (tid >> 3) * RPT;
    uint4 *tab = reinterpret_cast<uint4 *>(sm.hist);
    uint16_t *cumg = reinterpret_cast<uint16_t *>(sm.cum) + (K == 8 ? p : (p >> 1)) * Geo<8>::kCumWords;
#pragma unroll 4
    for (int k = 0; k < RPT; ++k) {
        const int row = r0 + k;
        uint4 *a = tab + row * 8 + p;
        const uint4 v = *a;
        *a = make_uint4(0u, 0u, 0u, 0u);
        uint32_t sum = v.x + v.y + v.z + v.w;
        if (K == 4) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, 1);
        if (K == 8 || (p & 1) == 0) cumg[pad32(row ^ 128)] = static_cast<uint16_t>(sum);
    }
}

// One warp: the inclusive scan of a slot's 256 counts in place (8 consecutive bins per lane),
// then its lower median bin and MAD (the searches of phase_scan8_warp and phase_search), and the
// threshold and replacement values into *rep (lane 0). The counts and cumulative counts are
// 16-bit (a window of this form has at most 8192 samples).
__device__ __forceinline__ void scan_search8(uint16_t *cum, int n, int lane, int64_t kq, int32_t cval,
                                             RepShared *rep) {
    uint32_t c[8];
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        run += cum[pad32(lane * 8 + j)];
        c[j] = run;
    }
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t excl = inc - run;
    const uint32_t half = static_cast<uint32_t>((n + 1) >> 1);
    int found = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t v = c[j] + excl;
        const uint32_t before = (j ? c[j - 1] : 0u) + excl;
        cum[pad32(lane * 8 + j)] = static_cast<uint16_t>(v);
        if (v >= half && before < half) found = lane * 8 + j + 1;
    }
    // the median bin is the one lane that found it; the others hold 0
    const int mb = static_cast<int>(__reduce_max_sync(0xFFFFFFFFu, static_cast<uint32_t>(found))) - 1;
    __syncwarp();
    const int d = warp_search<256>(lane, [&](int dd) {
        const int hi = mb + dd < 255 ? mb + dd : 255;
        const int lo = mb - dd - 1;
        const uint32_t f = static_cast<uint32_t>(cum[pad32(hi)]) - (lo >= 0 ? static_cast<uint32_t>(cum[pad32(lo)]) : 0u);
        return f >= half;
    });
    if (lane == 0) *rep = make_rep<8>(mb - Geo<8>::kOffset, d, kq, cval);
}

// A tile of nw (1 <= nw <= K) full int8 windows of 2^lw samples, 16-byte aligned, in shared
// memory at stage, for the plain excision modes (MODE 0..3) or the estimation pass of the
// Median of MAD (kModeStats). The histogram table must be zero on entry and is zero again
// after the reduce. Barriers: after the histogram (a bar.red.or that also agrees on a timeout),
// after the reduce, and, for excision, after the searches; warp w searches windows w, w + NW,
// ... M and D go straight to the segment's arrays. release_bar (nonzero for the tile's last
// windows) releases the stage: after the histogram for kModeStats, else after the replace pass.
template <int MODE, int T, int K>
__device__ bool process_tile_multi8(const Shm &sm, const uint8_t *stage, const Seg &sg, uint32_t w0, int nw, int lw,
                                    const Params &p, int tid, int par, uint32_t release_bar, bool stage_ok) {
    constexpr bool STATS = (MODE & kModeStats) != 0;
    constexpr int NW = T / 32;
    const int lane = tid & 31, warp = tid >> 5;
    int32_t *const med = sg.med, *const mad = sg.mad;  // sg lives in the stage descriptor
    if (stage_ok) hist8_multi<T, K>(sm, stage, lw, nw, tid);
    if (named_bar_or(sm.bar_id, T, !stage_ok)) return false;
    if (STATS && tid == 0 && release_bar) mbar_arrive(release_bar);
    reduce8_multi<T, K>(sm, tid);
    named_bar(sm.bar_id, T);
    for (int g = warp; g < nw; g += NW) {
        RepShared *rep = &sm.mt->rep[g];
        scan_search8(reinterpret_cast<uint16_t *>(sm.cum) + g * Geo<8>::kCumWords, 1 << lw, lane, p.kq, p.cval, rep);
        __syncwarp();
        if (lane == 0) {
            if (med) med[w0 + g] = rep->M;
            if (mad) mad[w0 + g] = rep->D;
        }
    }
    if (STATS) return true;
    named_bar(sm.bar_id, T);
    replace_tile8<MODE & 3, T>(sm, stage, sg, w0, nw, lw, sm.mt->rep, sm.mt->count, p, tid, par, release_bar);
    return true;
}

}  // namespace dev
}  // namespace rfi
