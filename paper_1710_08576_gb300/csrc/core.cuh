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
// 8-bit samples use a lane-striped histogram: bin v of lane l is word v*32 + l, so the 32
// lanes of a warp always hit 32 different banks and 32 different words; warps share the table
// through shared-memory atomics. 12-bit samples use 1, 2 or 4 plain copies of a 4096-bin
// table selected by lane, which spreads same-bin collisions within a warp.

#pragma once

#include <cstdint>
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

// Wait for the phase of the given parity, giving up after timeout_ns of wall time (and after
// a fixed number of polls in any case). Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31u) == 0 && global_timer_ns() - t0 > timeout_ns) return false;
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
// xor-ed with words 1 and 3 and with the round key, and the key advances by two Weyl
// increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Digital-noise replacement: M + round_half_away(S2 * sigq / (107020 * 2^16)), sigq = 97164*D,
// S2 = 2 * (sum of the eight 16-bit halves of the Philox output) - 8 * 65535.
// |S2| <= 524280 and sigq < 2^29, so |S2| * sigq < 2^48; dividing by 2^16 first and then by
// 107020 equals one floor division by their product.
__device__ __forceinline__ int32_t noise_value(int32_t M, uint32_t sigq, uint64_t seed, uint32_t sid,
                                               int64_t idx, int32_t lo, int32_t hi) {
    const uint4 r = philox4x32_10(
        make_uint4(static_cast<uint32_t>(idx), static_cast<uint32_t>(static_cast<uint64_t>(idx) >> 32),
                   sid, 0u),
        static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    const uint32_t s = (r.x & 0xFFFFu) + (r.x >> 16) + (r.y & 0xFFFFu) + (r.y >> 16) + (r.z & 0xFFFFu) +
                       (r.z >> 16) + (r.w & 0xFFFFu) + (r.w >> 16);
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
    static constexpr int kOffset = BITS == 8 ? 128 : 2048;  // bin = x + kOffset
    static constexpr int kBps = BITS == 8 ? 1 : 2;          // bytes per sample
    static constexpr int kLo = BITS == 8 ? -128 : -2048;
    static constexpr int kHi = BITS == 8 ? 127 : 2047;
    static constexpr int kCumWords = kBins + kBins / 32;     // padded: index b + b/32
    __host__ __device__ static constexpr int hist_bytes(int ncopies) {
        return BITS == 8 ? kBins * 32 * 4 : kBins * 4 * ncopies;
    }
};

__device__ __forceinline__ int pad32(int b) { return b + (b >> 5); }

struct Ctl {
    uint32_t warp_tot[32];
    int32_t mb;        // median bin
    int32_t d;         // MAD
    uint32_t count;    // flagged samples of the current window
    int32_t go;        // consumer broadcast: tile index, -1 end, -2 timeout
    uint32_t abort;    // set when any warp gave up on a bounded wait
    uint32_t err;      // 12-bit range error seen in the current window
    unsigned long long flagged;  // CTA total
};

// Per-CTA view of the shared-memory regions used by window processing.
struct Shm {
    uint8_t *hist;     // histogram (generic pointer)
    uint32_t hist_s;   // histogram (shared address)
    uint32_t *cum;     // padded cumulative counts
    Ctl *ctl;
    int ncopies;       // 12-bit only
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
    uint32_t *count_out;  // nullable
    int32_t *med_out;     // nullable
    int32_t *mad_out;     // nullable
};

// ------------------------------------------------------------------ phase 1: histogram
__device__ __forceinline__ void hist8_word(uint32_t lane_base, uint32_t w) {
    // lane_base = hist_s + 4 * lane; bin b of byte j: byte offset b * 128
    const uint32_t wb = w ^ 0x80808080u;  // int8 -> bin index x + 128 per byte
    red_add_shared(lane_base + ((wb << 7) & 0x7F80u), 1u);
    red_add_shared(lane_base + ((wb >> 1) & 0x7F80u), 1u);
    red_add_shared(lane_base + ((wb >> 9) & 0x7F80u), 1u);
    red_add_shared(lane_base + ((wb >> 17) & 0x7F80u), 1u);
}

__device__ __forceinline__ uint32_t hist12_sample(uint32_t copy_base, int32_t x) {
    const uint32_t b = static_cast<uint32_t>(x + 2048);
    red_add_shared(copy_base + ((b & 4095u) << 2), 1u);
    return b > 4095u ? 1u : 0u;
}

__device__ __forceinline__ uint32_t hist12_word(uint32_t copy_base, uint32_t w) {
    return hist12_sample(copy_base, static_cast<int16_t>(w & 0xFFFFu)) |
           hist12_sample(copy_base, static_cast<int16_t>(w >> 16));
}

template <int BITS, int T>
__device__ __forceinline__ void phase_histogram(const Shm &sm, const Win &w, int tid) {
    const int lane = tid & 31;
    const int nbytes = w.n * Geo<BITS>::kBps;
    const int nfull = nbytes >> 4;
    const uint4 *d4 = reinterpret_cast<const uint4 *>(w.data);
    if (BITS == 8) {
        const uint32_t lb = sm.hist_s + 4u * lane;
        int c = tid;
        for (; c + T < nfull; c += 2 * T) {
            const uint4 a = d4[c], b = d4[c + T];
            hist8_word(lb, a.x); hist8_word(lb, a.y); hist8_word(lb, a.z); hist8_word(lb, a.w);
            hist8_word(lb, b.x); hist8_word(lb, b.y); hist8_word(lb, b.z); hist8_word(lb, b.w);
        }
        if (c < nfull) {
            const uint4 a = d4[c];
            hist8_word(lb, a.x); hist8_word(lb, a.y); hist8_word(lb, a.z); hist8_word(lb, a.w);
        }
        const int rem = nbytes & 15;
        if (tid < rem) {
            const uint32_t b = static_cast<uint32_t>(static_cast<int8_t>(w.data[nfull * 16 + tid]) + 128);
            red_add_shared(lb + b * 128u, 1u);
        }
    } else {
        const uint32_t cb = sm.hist_s + static_cast<uint32_t>(lane & (sm.ncopies - 1)) * 16384u;
        uint32_t bad = 0;
        for (int c = tid; c < nfull; c += T) {
            const uint4 a = d4[c];
            bad |= hist12_word(cb, a.x) | hist12_word(cb, a.y) | hist12_word(cb, a.z) | hist12_word(cb, a.w);
        }
        const int rem = (nbytes & 15) >> 1;
        if (tid < rem) {
            const int16_t x = reinterpret_cast<const int16_t *>(w.data)[nfull * 8 + tid];
            bad |= hist12_sample(cb, x);
        }
        if (bad) atomicOr(&sm.ctl->err, 1u);
    }
}

// ------------------------------------------------------------------ phases 2-4
template <int BITS, int T>
__device__ __forceinline__ void phase_reduce(const Shm &sm, int tid) {
    const int lane = tid & 31;
    uint32_t *cum = sm.cum;
    if (BITS == 8) {
        // row r = bin r: 32 lane counters (128 bytes); read and clear in 8 rotated 16-byte pieces
        for (int r = tid; r < 256; r += T) {
            uint4 *row = reinterpret_cast<uint4 *>(sm.hist + r * 128);
            uint32_t s = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int qq = (q + lane) & 7;
                const uint4 v = row[qq];
                s += v.x + v.y + v.z + v.w;
                row[qq] = make_uint4(0u, 0u, 0u, 0u);
            }
            cum[pad32(r)] = s;
        }
    } else {
        uint32_t *h = reinterpret_cast<uint32_t *>(sm.hist);
        const int nc = sm.ncopies;
        for (int b = tid; b < 4096; b += T) {
            uint32_t s = 0;
            for (int c = 0; c < nc; ++c) {
                s += h[c * 4096 + b];
                h[c * 4096 + b] = 0u;
            }
            cum[pad32(b)] = s;
        }
    }
}

template <int BITS, int T>
__device__ __forceinline__ void phase_scan(const Shm &sm, int tid) {
    constexpr int B = Geo<BITS>::kBins;
    constexpr int TE = T < B ? T : B;
    constexpr int BPT = B / TE;
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t *cum = sm.cum;
    uint32_t v[BPT];
    uint32_t run = 0;
    if (tid < TE) {
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            run += cum[pad32(tid * BPT + i)];
            v[i] = run;
        }
    }
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sm.ctl->warp_tot[warp] = inc;
    named_bar(1, T);
    uint32_t pre = 0;
    for (int q = 0; q < warp; ++q) pre += sm.ctl->warp_tot[q];
    const uint32_t excl = pre + inc - run;
    if (tid < TE) {
#pragma unroll
        for (int i = 0; i < BPT; ++i) cum[pad32(tid * BPT + i)] = v[i] + excl;
    }
}

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

template <int BITS>
__device__ __forceinline__ void phase_search(const Shm &sm, int n, int lane) {
    constexpr int B = Geo<BITS>::kBins;
    const uint32_t *cum = sm.cum;
    const uint32_t half = static_cast<uint32_t>((n + 1) >> 1);
    const int mb = warp_search<B>(lane, [&](int v) { return cum[pad32(v)] >= half; });
    const int d = warp_search<B>(lane, [&](int dd) {
        const int hi = mb + dd < B - 1 ? mb + dd : B - 1;
        const int lo = mb - dd - 1;
        const uint32_t f = cum[pad32(hi)] - (lo >= 0 ? cum[pad32(lo)] : 0u);
        return f >= half;
    });
    if (lane == 0) {
        sm.ctl->mb = mb;
        sm.ctl->d = d;
        sm.ctl->count = 0u;
    }
}

// ------------------------------------------------------------------ phase 5: replace
struct Rep {
    int32_t M, D;
    int64_t t;        // ceil(Kq*D / 2^16)
    int32_t hiv, lov; // threshold replacement above / below (saturated)
    uint32_t sigq;    // 97164 * D
    bool active;      // some sample can be flagged
};

__device__ __forceinline__ int32_t sat_to(int64_t v, int32_t lo, int32_t hi) {
    return v < lo ? lo : (v > hi ? hi : static_cast<int32_t>(v));
}

template <int BITS>
__device__ __forceinline__ Rep make_rep(const Ctl *ctl, int64_t kq) {
    Rep r;
    r.M = ctl->mb - Geo<BITS>::kOffset;
    r.D = ctl->d;
    const int64_t kd = kq * static_cast<int64_t>(r.D);
    r.t = (kd + 65535) >> 16;
    const int64_t c = kd >> 16;
    r.hiv = sat_to(static_cast<int64_t>(r.M) + c, Geo<BITS>::kLo, Geo<BITS>::kHi);
    r.lov = sat_to(static_cast<int64_t>(r.M) - c, Geo<BITS>::kLo, Geo<BITS>::kHi);
    r.sigq = 97164u * static_cast<uint32_t>(r.D);
    // |x - M| never exceeds the sample span
    r.active = r.D > 0 && r.t <= (Geo<BITS>::kHi - Geo<BITS>::kLo);
    return r;
}

// 4 int8 samples: returns the output word and sets f to 0xFF in flagged bytes.
template <int MODE>
__device__ __forceinline__ uint32_t rep8_word(uint32_t w, uint32_t mb4, uint32_t t4, uint32_t c4,
                                              uint32_t hi4, uint32_t lo4, uint32_t &f) {
    const uint32_t wb = w ^ 0x80808080u;
    f = __vcmpgeu4(__vabsdiffu4(wb, mb4), t4);
    uint32_t rep = 0u;
    if (MODE == 1) rep = c4;
    if (MODE == 2) {
        const uint32_t up = __vcmpgtu4(wb, mb4);
        rep = (hi4 & up) | (lo4 & ~up);
    }
    return (w & ~f) | (rep & f);
}

// flag bytes (0x00/0xFF) -> 4 bits, byte j -> bit j
__device__ __forceinline__ uint32_t byte_flags_to_bits(uint32_t f) {
    return ((f & 0x80808080u) * 0x00204081u) >> 28;
}

__device__ __forceinline__ uint32_t set_byte(uint32_t w, int j, uint32_t v) {
    const int sh = j * 8;
    return (w & ~(0xFFu << sh)) | ((v & 0xFFu) << sh);
}

template <int BITS, int MODE, int T>
__device__ __forceinline__ uint32_t phase_replace(const Win &w, const Rep &r, const Params &p, int tid) {
    constexpr int BPS = Geo<BITS>::kBps;
    constexpr int LO = Geo<BITS>::kLo, HI = Geo<BITS>::kHi;
    const int nbytes = w.n * BPS;
    const int nchunks = (nbytes + 15) >> 4;
    const uint4 *d4 = reinterpret_cast<const uint4 *>(w.data);
    uint32_t flagged = 0;
    if (BITS == 8) {
        const uint32_t mb4 = static_cast<uint32_t>(r.M + 128) * 0x01010101u;
        const uint32_t t4 = static_cast<uint32_t>(r.t > 255 ? 255 : r.t) * 0x01010101u;
        const uint32_t c4 = (static_cast<uint32_t>(p.cval) & 0xFFu) * 0x01010101u;
        const uint32_t hi4 = (static_cast<uint32_t>(r.hiv) & 0xFFu) * 0x01010101u;
        const uint32_t lo4 = (static_cast<uint32_t>(r.lov) & 0xFFu) * 0x01010101u;
        uint16_t *mk = reinterpret_cast<uint16_t *>(w.mask);
        for (int c = tid; c < nchunks; c += T) {
            uint4 v = d4[c];
            uint32_t bits = 0;
            if (r.active) {
                uint32_t f0, f1, f2, f3;
                v.x = rep8_word<MODE>(v.x, mb4, t4, c4, hi4, lo4, f0);
                v.y = rep8_word<MODE>(v.y, mb4, t4, c4, hi4, lo4, f1);
                v.z = rep8_word<MODE>(v.z, mb4, t4, c4, hi4, lo4, f2);
                v.w = rep8_word<MODE>(v.w, mb4, t4, c4, hi4, lo4, f3);
                bits = byte_flags_to_bits(f0) | (byte_flags_to_bits(f1) << 4) |
                       (byte_flags_to_bits(f2) << 8) | (byte_flags_to_bits(f3) << 12);
            }
            const int valid = nbytes - c * 16;  // bytes of this chunk inside the window
            if (valid < 16) bits &= (1u << valid) - 1u;
            if (MODE == 3) {
                uint32_t m = bits;
                while (m) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1u;
                    const uint32_t z = static_cast<uint32_t>(
                        noise_value(r.M, r.sigq, p.seed, w.sid, w.abs_idx + c * 16 + j, LO, HI));
                    if (j < 4) v.x = set_byte(v.x, j, z);
                    else if (j < 8) v.y = set_byte(v.y, j - 4, z);
                    else if (j < 12) v.z = set_byte(v.z, j - 8, z);
                    else v.w = set_byte(v.w, j - 12, z);
                }
            }
            flagged += __popc(bits);
            if (w.vec && valid >= 16) {
                __stcs(reinterpret_cast<uint4 *>(w.out + c * 16), v);
            } else {
                const uint32_t ww[4] = {v.x, v.y, v.z, v.w};
                const int lim = valid < 16 ? valid : 16;
                for (int j = 0; j < lim; ++j) w.out[c * 16 + j] = static_cast<uint8_t>(ww[j >> 2] >> ((j & 3) * 8));
            }
            if (mk) mk[c] = static_cast<uint16_t>(bits);
        }
        if (mk) {
            for (int c = nchunks + tid; c < 2 * w.mask_words; c += T) mk[c] = 0;
        }
    } else {
        uint8_t *mk = reinterpret_cast<uint8_t *>(w.mask);
        const int64_t t = r.t;
        for (int c = tid; c < nchunks; c += T) {
            const uint4 v = d4[c];
            uint32_t ww[4] = {v.x, v.y, v.z, v.w};
            const int valid = (nbytes - c * 16) >> 1;  // samples of this chunk in the window
            uint32_t bits = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int32_t x = static_cast<int16_t>((ww[j >> 1] >> ((j & 1) * 16)) & 0xFFFFu);
                const int32_t ad = x > r.M ? x - r.M : r.M - x;
                const bool fl = r.active && ad >= t && j < valid;
                if (fl) {
                    int32_t z;
                    if (MODE == 0) z = 0;
                    else if (MODE == 1) z = p.cval;
                    else if (MODE == 2) z = x > r.M ? r.hiv : r.lov;
                    else z = noise_value(r.M, r.sigq, p.seed, w.sid, w.abs_idx + c * 8 + j, LO, HI);
                    const int sh = (j & 1) * 16;
                    ww[j >> 1] = (ww[j >> 1] & ~(0xFFFFu << sh)) | ((static_cast<uint32_t>(z) & 0xFFFFu) << sh);
                    bits |= 1u << j;
                }
            }
            flagged += __popc(bits);
            if (w.vec && valid >= 8) {
                __stcs(reinterpret_cast<uint4 *>(w.out + c * 16), make_uint4(ww[0], ww[1], ww[2], ww[3]));
            } else {
                int16_t *o = reinterpret_cast<int16_t *>(w.out);
                const int lim = valid < 8 ? valid : 8;
                for (int j = 0; j < lim; ++j)
                    o[c * 8 + j] = static_cast<int16_t>((ww[j >> 1] >> ((j & 1) * 16)) & 0xFFFFu);
            }
            if (mk) mk[c] = static_cast<uint8_t>(bits);
        }
        if (mk) {
            for (int c = nchunks + tid; c < 4 * w.mask_words; c += T) mk[c] = 0;
        }
    }
    return flagged;
}

// ------------------------------------------------------------------ one window
// All T threads of the group call this; the histogram must be zero on entry and is zero again
// on exit. Uses named barrier 1 over T threads.
template <int BITS, int MODE, int T>
__device__ void process_window(const Shm &sm, const Win &w, const Params &p, int tid) {
    const int lane = tid & 31, warp = tid >> 5;
    phase_histogram<BITS, T>(sm, w, tid);
    named_bar(1, T);
    phase_reduce<BITS, T>(sm, tid);
    named_bar(1, T);
    phase_scan<BITS, T>(sm, tid);
    named_bar(1, T);
    if (warp == 0) phase_search<BITS>(sm, w.n, lane);
    named_bar(1, T);
    const Rep r = make_rep<BITS>(sm.ctl, p.kq);
    uint32_t f = phase_replace<BITS, MODE, T>(w, r, p, tid);
    f = __reduce_add_sync(0xFFFFFFFFu, f);
    if (lane == 0 && f) atomicAdd(&sm.ctl->count, f);
    named_bar(1, T);
    if (tid == 0) {
        const uint32_t cnt = sm.ctl->count;
        if (w.count_out) *w.count_out = cnt;
        if (w.med_out) *w.med_out = r.M;
        if (w.mad_out) *w.mad_out = r.D;
        sm.ctl->flagged += cnt;
        if (BITS == 12 && sm.ctl->err) {
            atomicOr(p.status, kStatusSampleRange);
            sm.ctl->err = 0u;
        }
    }
}

}  // namespace dev
}  // namespace rfi
