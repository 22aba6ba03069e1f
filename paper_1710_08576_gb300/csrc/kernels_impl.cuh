// Excision kernels: the persistent batched kernel (bulk-copy pipeline, work list) and the plain
// one-CTA-per-window kernel. Instantiated per sample width in kernels8.cu / kernels12.cu.
#pragma once

#include <cstddef>
#include <mutex>

#include "core.cuh"

namespace rfi {
namespace dev {

constexpr int kMaxStages = 8;
constexpr uint64_t kWaitTimeoutNs = 4000000000ull;   // 4 s: no healthy wait comes close
constexpr uint64_t kInjectTimeoutNs = 1000000ull;    // 1 ms for the test hook

__host__ __device__ constexpr int align_up(int v, int a) { return (v + a - 1) / a * a; }

// Per-stage descriptor written by the copy warp: the tile, its segment and the tile index.
struct StageMeta {
    Tile tile;
    Seg seg;
    int32_t tidx;   // tile index, -1: no more tiles
    int32_t pad[3];
};

// Split-warp form: a window handed from the histogram warps to the replace warps. Slot j is
// filled by histogram warp 0 (lane 0) after waiting for its empty mbarrier, announced through its
// full mbarrier, and released by the last replace warp to finish the window.
constexpr int kSplitSlots = 4;
struct __align__(16) SplitSlot {
    RepShared rep;    // the window's M, D, threshold and replacement values
    int64_t widx;     // window of the segment
    int32_t stage;    // stage buffer holding it
    int32_t k;        // window of the stage's tile
    int32_t last;     // the tile's last window: its replace releases the stage
    int32_t end;      // no more windows
    int32_t upar;     // parity of the stage's fill
    int32_t pad;
};

// Dynamic shared memory: the histogram at offset 0 (8-bit: one table for all groups; 12-bit:
// per group; none for the apply passes of Eq. 3), then one block per consumer group
// (cumulative counts, control block, mbarriers, stage descriptors), then the stage buffers of
// every group.
struct Layout {
    int grp;        // first group block
    int grp_size;   // bytes per group block
    int cum, ctl, bar, meta;  // offsets inside a group block
    int nlist;                // digital-noise work area inside a group block (0: none)
    int nring;                // int8 digital noise: the warps' position rings (0: none)
    int amd;                  // apply passes: per stage, {M, dispersion} of its windows (0: none)
    int atile;                // apply passes: thresholds and counts of the current tile (0: none)
    int cps;                  // digital copy: per-variant state inside a group block (0: none)
    int mt;                   // 8-bit plain excision and estimation: multi-window tile state (0: none)
    int split;                // split-warp form: the hand-over slots (0: none)
    int stage;      // first stage buffer; group g stage s at stage + (g * stages + s) * stage_bytes
    int total;
};

template <int BITS>
__host__ __device__ inline Layout layout(int ncopies, int stages, int stage_bytes, int cw, int groups, int mode) {
    Layout L;
    L.grp = (mode & kModeApply) ? 0 : align_up(Geo<BITS>::hist_bytes(ncopies, groups), 128);
    // multi-window tiles: 8-bit, one group, plain excision or the estimation pass
    const bool multi = BITS == 8 && groups == 1 && (mode & kModeMulti) != 0;
    L.cum = 0;
    // (multi-window tiles: up to kMultiMax slots of 16-bit counts)
    L.ctl = align_up(multi ? Geo<BITS>::kCumWords * 2 * kMultiMax : Geo<BITS>::kCumWords * 4, 128);
    const bool split = (mode & kModeWarpSplit) != 0;
    L.bar = align_up(L.ctl + static_cast<int>(sizeof(Ctl)), 128);
    // full and empty barriers per stage, the test hook's barrier, and for the split-warp form a
    // full and an empty barrier per hand-over slot
    L.meta = align_up(L.bar + (2 * kMaxStages + 1 + (split ? 2 * kSplitSlots : 0)) * 8, 128);
    const int meta_end = align_up(L.meta + kMaxStages * static_cast<int>(sizeof(StageMeta)), 128);
    const bool noise = ((mode & 3) == 3 || (mode & kModeCopies) != 0) && (mode & kModeStats) == 0;
    L.nlist = noise ? meta_end : 0;
    // int8: a 32-bit entry for every 16-byte chunk of a stage that may hold a flagged sample,
    // then each consumer warp's ring of kNoiseRing 32-bit positions (multi-window tiles keep the
    // rings in their cumulative-count area, which is idle by then and large enough); 12-bit: the
    // position list
    const int list_bytes = align_up(stage_bytes / 4 > 128 ? stage_bytes / 4 : 128, 128);
    const int ring_bytes = multi ? 0 : cw * kNoiseRing * 4;
    static_assert(kNoiseRing * 4 * 16 <= Geo<8>::kCumWords * 2 * kMultiMax, "rings of 16 warps fit the multi-window counts");
    const int noise_bytes = BITS == 8 ? list_bytes + ring_bytes : kNoiseList * 2;
    L.nring = (noise && BITS == 8) ? (multi ? L.cum : meta_end + list_bytes) : 0;
    const int list_end = noise ? align_up(meta_end + noise_bytes, 128) : meta_end;
    const bool apply = (mode & kModeApply) != 0;
    L.amd = apply ? list_end : 0;
    L.atile = apply ? align_up(list_end + kMaxStages * kApplyTileWindows * 8, 128) : 0;
    const int amd_end = apply ? align_up(L.atile + static_cast<int>(sizeof(ApplyTile)), 128) : list_end;
    const bool copies = (mode & kModeCopies) != 0;
    L.cps = copies ? amd_end : 0;
    const int cps_end = copies ? align_up(amd_end + static_cast<int>(sizeof(CopyShared)), 128) : amd_end;
    L.mt = multi ? cps_end : 0;
    L.grp_size = multi ? align_up(cps_end + static_cast<int>(sizeof(MultiTile)), 128) : cps_end;
    L.split = split ? L.grp_size : 0;
    if (split) L.grp_size = align_up(L.grp_size + kSplitSlots * static_cast<int>(sizeof(SplitSlot)), 128);
    L.stage = L.grp + groups * L.grp_size;
    L.total = L.stage + groups * stages * stage_bytes;
    return L;
}

// The shared-memory view of consumer group g.
template <int BITS>
__device__ __forceinline__ Shm group_view(uint8_t *smem, const Layout &L, int g, int ncopies) {
    Shm sm;
    uint8_t *gb = smem + L.grp + g * L.grp_size;
    sm.hist = BITS == 8 ? smem : smem + g * Geo<12>::kBins * 4 * ncopies;  // 8-bit: one table
    sm.hist_s = smem_addr(sm.hist);
    sm.grp = BITS == 8 ? 128u * static_cast<uint32_t>(g) : 0u;
    sm.cum = reinterpret_cast<uint32_t *>(gb + L.cum);
    sm.ctl = reinterpret_cast<Ctl *>(gb + L.ctl);
    sm.ncopies = ncopies;
    sm.bar_id = 1 + g;
    sm.nlist = L.nlist ? reinterpret_cast<uint16_t *>(gb + L.nlist) : nullptr;
    sm.nring = L.nlist && BITS == 8 ? reinterpret_cast<uint32_t *>(gb + L.nring) : nullptr;
    sm.cp = L.cps ? reinterpret_cast<CopyShared *>(gb + L.cps) : nullptr;
    sm.at = L.atile ? reinterpret_cast<ApplyTile *>(gb + L.atile) : nullptr;
    sm.mt = L.mt ? reinterpret_cast<MultiTile *>(gb + L.mt) : nullptr;
    return sm;
}

__device__ __forceinline__ void zero_shared(uint8_t *smem, int bytes, int tid, int nthreads) {
    uint4 *h = reinterpret_cast<uint4 *>(smem);
    for (int i = tid; i < bytes / 16; i += nthreads) h[i] = make_uint4(0u, 0u, 0u, 0u);
}

__device__ __forceinline__ Win make_win(const Seg &sg, int64_t w, const uint8_t *data, int bps) {
    Win win;
    const int64_t s0 = w * sg.W;
    const int64_t left = sg.len - s0;
    win.data = data;
    win.n = static_cast<int32_t>(left < sg.W ? left : sg.W);
    win.out = sg.out + s0 * bps;
    win.mask = sg.mask ? sg.mask + w * sg.mask_words : nullptr;
    win.mask_words = sg.mask_words;
    win.abs_idx = sg.abs0 + s0;
    win.sid = sg.stream_id;
    win.vec = sg.vec != 0;
    return win;
}

// ------------------------------------------------------------------ persistent kernel
// G consumer groups per CTA, each with CW consumer warps and one copy warp. The copy warp of a
// group owns a ring of `stages` shared-memory buffers; for each tile it fills the stage
// descriptor, arms the stage's full barrier with the byte count and issues one bulk copy.
// The group's consumers wait on the full barrier, process the tile's windows, and release the
// stage through its empty barrier. All waits are bounded.
// Resident CTAs per SM that the register budget is sized for (0: left to the compiler). One
// group of 8 + 1 warps runs three CTAs per SM, which its shared memory allows and 72 registers
// a thread fit; the hint keeps the allocator from cutting registers for a fourth CTA that the
// shared memory never grants.
constexpr int min_ctas_per_sm(int cw, int g) { return g != 1 ? 0 : (cw == 8 ? 3 : (cw == 4 ? 4 : 0)); }

// ------------------------------------------------------------------ split-warp consumers
// The consumer warps of the split-warp form (int8, zero / constant / threshold, also
// write-flagged, one group of 8 consumer warps). Warps 0-3 (the histogram warps, named barrier 1) take the stages in order:
// per window the histogram, the reduce and, on warp 0, the scan and the searches, whose result
// warp 0 hands over in a slot; they go on to the next window's histogram at once, so warp 0's
// searches overlap the other histogram warps' work. Warps 4-7 (the replace warps, named barrier 2)
// take the slots in order and run the replace pass of each window (Eq. 1 and Eq. 2) from the
// stage, which the last of them to finish releases after the tile's last window; they write the
// counts, warp 0 of the histogram warps M and D. The histogram table keeps its running sums as in
// the joint form. Every wait is bounded; the first barrier after each wait agrees on a timeout
// among its warps, and a timeout or the end of the work list reaches the replace warps through
// a slot marked end (or, if the hand-over itself timed out, through their own bounded waits).
template <int MODE, int CW>
__device__ bool split_consumers(const Shm &sm, uint8_t *gb, const Layout &L, StageMeta *meta, uint8_t *stage0,
                                int stages, int stage_bytes, uint32_t bar0, const Params &p, int tid) {
    static_assert(CW == 8, "four histogram and four replace warps");
    constexpr int NH = 4, NR = CW - NH, TH = NH * 32, TR = NR * 32;
    constexpr int RMODE = MODE & 3;
    const int lane = tid & 31;
    SplitSlot *slots = reinterpret_cast<SplitSlot *>(gb + L.split);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (kMaxStages + s); };
    auto slot_full = [&](int j) { return bar0 + 8u * (2 * kMaxStages + 1 + j); };
    auto slot_empty = [&](int j) { return bar0 + 8u * (2 * kMaxStages + 1 + kSplitSlots + j); };
    bool tmo = false;
    if (tid < TH) {
        RowSums rs = {{0u, 0u}};
        int seq = 0;          // windows handed over so far
        bool stop = false;    // warp 0: a hand-over timed out
        for (int it = 0;; ++it) {
            const int s = it % stages;
            const int u = it / stages;
            const bool ok = mbar_wait_bounded(full_bar(s), u & 1, kWaitTimeoutNs);
            if (named_bar_or(1, TH, !ok || stop)) {
                tmo = true;
                break;
            }
            if (meta[s].tidx < 0) break;  // the end of the work list, seen alike by every thread
            const Tile tl = meta[s].tile;
            const Seg &sg = meta[s].seg;
            uint8_t *stage = stage0 + s * stage_bytes;
            if (!sg.vec) {
                const uint8_t *src = sg.in + static_cast<int64_t>(tl.w0) * sg.W;
                for (int i = tid; i < static_cast<int>(tl.bytes); i += TH) stage[i] = src[i];
                named_bar(1, TH);
            }
            bool brk = false;
            for (uint32_t k = 0; k < tl.nw; ++k) {
                const int64_t widx = static_cast<int64_t>(tl.w0) + k;
                const Win win = make_win(sg, widx, stage + k * sg.W, 1);
                phase_histogram<8, TH, 128>(sm, win, tid, 0);
                // warp 0 has finished the previous window's searches and hand-over
                if (named_bar_or(1, TH, stop)) {
                    brk = true;
                    break;
                }
                phase_reduce8_counts<TH, 128>(sm, tid, rs);
                named_bar(1, TH);
                if (tid < 32) {
                    phase_scan8_warp(sm, win.n, lane);
                    const int j = seq % kSplitSlots, use = seq / kSplitSlots;
                    int okj = 1;
                    if (use > 0 && lane == 0) okj = mbar_wait_bounded(slot_empty(j), (use - 1) & 1, kWaitTimeoutNs);
                    okj = __shfl_sync(0xFFFFFFFFu, okj, 0);
                    phase_search<8>(sm, win.n, lane, p.kq, p.cval);
                    __syncwarp();
                    if (lane == 0) {
                        if (okj) {
                            SplitSlot &sl = slots[j];
                            sl.rep = sm.ctl->rep;
                            sl.widx = widx;
                            sl.stage = s;
                            sl.k = static_cast<int32_t>(k);
                            sl.last = k + 1 == tl.nw ? 1 : 0;
                            sl.end = 0;
                            sl.upar = u & 1;
                            if (sg.med) sg.med[widx] = sm.ctl->rep.M;
                            if (sg.mad) sg.mad[widx] = sm.ctl->rep.D;
                            mbar_arrive(slot_full(j));
                        }
                    }
                    if (!okj) stop = true;
                }
                ++seq;
            }
            if (brk) {
                tmo = true;
                break;
            }
        }
        if (tid < 32 && !tmo) {  // the end mark for the replace warps
            const int j = seq % kSplitSlots, use = seq / kSplitSlots;
            int okj = 1;
            if (use > 0 && lane == 0) okj = mbar_wait_bounded(slot_empty(j), (use - 1) & 1, kWaitTimeoutNs);
            if (lane == 0 && okj) {
                slots[j].end = 1;
                mbar_arrive(slot_full(j));
            }
            if (!__shfl_sync(0xFFFFFFFFu, okj, 0)) tmo = true;
        }
    } else {
        const int rtid = tid - TH;
        Shm sr = sm;
        sr.bar_id = 2;
        int seq = 0, par = 0;
        const KeysPre key{p};
        for (;;) {
            const int j = seq % kSplitSlots, use = seq / kSplitSlots;
            const bool ok = mbar_wait_bounded(slot_full(j), use & 1, kWaitTimeoutNs);
            if (named_bar_or(2, TR, !ok)) {
                tmo = true;
                break;
            }
            const SplitSlot &sl = slots[j];
            if (sl.end) break;
            const int s = sl.stage;
            // the stage's fill has completed; waiting on it orders its bytes for these threads
            mbar_wait_bounded(full_bar(s), static_cast<uint32_t>(sl.upar), kWaitTimeoutNs);
            const Seg &sg = meta[s].seg;
            const int64_t widx = sl.widx;
            const Win win = make_win(sg, widx, stage0 + s * stage_bytes + sl.k * sg.W, 1);
            const Rep r = load_rep(sl.rep);
            Pow pw = {0u, 0u};
            uint32_t f = phase_replace<8, RMODE, TR, false, KeysPre, 0, (MODE & kModeFlaggedOnly) != 0, true>(
                sr, win, r, key, rtid, &sm.ctl->ncount[par], pw, &sl.rep);
            f = __reduce_add_sync(0xFFFFFFFFu, f);
            if (lane == 0) {
                if (f) atomicAdd(&sm.ctl->count[par], f);
                __threadfence_block();
                if (atomicAdd(&sm.ctl->done[par], 1u) == NR - 1) {
                    // the last replace warp of the window: every count is in, every read done
                    __threadfence_block();
                    const uint32_t cnt = atomicExch(&sm.ctl->count[par], 0u);
                    sm.ctl->done[par] = 0u;
                    if (sg.counts) sg.counts[widx] = cnt;
                    sm.ctl->flagged += cnt;
                    if (sl.last) mbar_arrive(empty_bar(s));
                    mbar_arrive(slot_empty(j));
                }
            }
            ++seq;
            par ^= 1;
        }
    }
    return !tmo;
}

template <int BITS, int MODE, int CW, int G>
__global__ void __launch_bounds__(G *(CW + 1) * 32, min_ctas_per_sm(CW, G))
persistent_kernel(const Seg *__restrict__ segs, const Tile *__restrict__ tiles, int ntiles, Params p,
                  int stages, int stage_bytes, int dynamic_tiles, unsigned *counter, int inject_timeout) {
    constexpr int T = CW * 32;          // consumer threads per group
    constexpr int GT = (CW + 1) * 32;   // threads per group
    constexpr int BPS = Geo<BITS>::kBps;
    extern __shared__ __align__(128) uint8_t smem[];
    if (BITS == 8 && smem_addr(smem) != kDynSmemShared) {
        if (threadIdx.x == 0) atomicOr(p.status, kStatusLayout);
        return;
    }
    const Layout L = layout<BITS>(p.ncopies, stages, stage_bytes, CW, G, MODE);
    const int g = threadIdx.x / GT;
    const int tid = threadIdx.x % GT;
    const int warp = tid >> 5, lane = tid & 31;
    const Shm sm = group_view<BITS>(smem, L, g, p.ncopies);
    uint8_t *gb = smem + L.grp + g * L.grp_size;
    const uint32_t bar0 = smem_addr(gb + L.bar);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (kMaxStages + s); };
    const uint32_t inj_bar = bar0 + 8u * (2 * kMaxStages);
    StageMeta *meta = reinterpret_cast<StageMeta *>(gb + L.meta);
    uint8_t *stage0 = smem + L.stage + g * stages * stage_bytes;

    zero_shared(smem, L.stage, threadIdx.x, blockDim.x);  // histogram and group blocks
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(inj_bar, 1);
        if (MODE & kModeWarpSplit)
            for (int j = 0; j < 2 * kSplitSlots; ++j) mbar_init(inj_bar + 8u * (1 + j), 1);
        fence_mbar_init();
    }
    __syncthreads();

    const unsigned qid = blockIdx.x * G + g;  // static tile queue of this group
    const unsigned nq = gridDim.x * G;
    if (warp == CW) {
        // ---------------- copy warp
        // The tile descriptors are fetched three iterations deep, one dependent step per
        // iteration: the tile index of iteration it + 3 (the atomic of the dynamic queue), the
        // tile words of it + 2 and the segment words of it + 1. Every value is used one
        // iteration after it was requested, so the refill of a stage waits on no global round
        // trip but its own bulk copy. Lane l < 4 holds word l of the tile, lanes 4..27 word
        // l - 4 of its segment: the stage descriptor as it is stored.
        constexpr unsigned kAll = 0xFFFFFFFFu;
        static_assert(sizeof(Tile) == 16 && sizeof(Seg) == 96, "descriptor copy layout");
        constexpr int kLaneW0 = offsetof(Tile, w0) / 4, kLaneNw = offsetof(Tile, nw) / 4;
        constexpr int kLaneBytes = offsetof(Tile, bytes) / 4;
        constexpr int kLaneIn = 4 + offsetof(Seg, in) / 4, kLaneMed = 4 + offsetof(Seg, med) / 4;
        constexpr int kLaneMad = 4 + offsetof(Seg, mad) / 4, kLaneW = 4 + offsetof(Seg, W) / 4;
        constexpr int kLaneVec = 4 + offsetof(Seg, vec) / 4;
        const uint32_t *tile_w = reinterpret_cast<const uint32_t *>(tiles);
        const uint32_t *seg_w = reinterpret_cast<const uint32_t *>(segs);
        auto grab = [&](int i) -> int {  // lane 0: the group's tile of iteration i
            return dynamic_tiles == 1 ? static_cast<int>(atomicAdd(counter, 1u))
                                      : static_cast<int>(qid + static_cast<unsigned>(i) * nq);
        };
        auto tile_word = [&](int t) -> uint32_t {
            return (t < ntiles && lane < 4) ? tile_w[4 * t + lane] : 0u;
        };
        auto desc_word = [&](int t, uint32_t tw) -> uint32_t {
            const uint32_t si = __shfl_sync(kAll, tw, 0);
            return lane < 4 ? tw : ((t < ntiles && lane < 28) ? seg_w[24 * si + (lane - 4)] : 0u);
        };
        auto ptr = [&](uint32_t dw, int l) -> uint64_t {
            return static_cast<uint64_t>(__shfl_sync(kAll, dw, l)) |
                   (static_cast<uint64_t>(__shfl_sync(kAll, dw, l + 1)) << 32);
        };
        int g0 = 0, g1 = 0;
        if (lane == 0) {
            g0 = grab(0);
            g1 = g0 < ntiles ? grab(1) : ntiles;
        }
        int t0 = __shfl_sync(kAll, g0, 0);
        int t1 = __shfl_sync(kAll, g1, 0);
        uint32_t dw = desc_word(t0, tile_word(t0));  // descriptor of iteration it
        uint32_t tw1 = tile_word(t1);                // tile words of iteration it + 1
        int pend = 0;                                // lane 0: tile index of iteration it + 2
        if (lane == 0) pend = t1 < ntiles ? grab(2) : ntiles;
        int issued = 0;  // iterations whose full barrier was armed
        for (int it = 0;; ++it) {
            const int s = it % stages;
            const int u = it / stages;
            if (u > 0) {
                int ok = 1;
                if (lane == 0) ok = mbar_wait_bounded(empty_bar(s), (u - 1) & 1, kWaitTimeoutNs);
                ok = __shfl_sync(kAll, ok, 0);
                if (!ok) {
                    if (lane == 0) {
                        atomicOr(p.status, kStatusTimeout);
                        atomicExch(&sm.ctl->abort, 1u);
                    }
                    break;
                }
            }
            if (*reinterpret_cast<volatile uint32_t *>(&sm.ctl->abort)) break;
            const int t = t0;
            issued = it + 1;
            if (t >= ntiles) {
                if (lane == 0) {
                    meta[s].tidx = -1;
                    mbar_arrive(full_bar(s));
                }
                break;
            }
            const uint32_t w0 = __shfl_sync(kAll, dw, kLaneW0), nw = __shfl_sync(kAll, dw, kLaneNw);
            const uint32_t tbytes = __shfl_sync(kAll, dw, kLaneBytes);
            const uint8_t *in = reinterpret_cast<const uint8_t *>(ptr(dw, kLaneIn));
            const int32_t W = static_cast<int32_t>(__shfl_sync(kAll, dw, kLaneW));
            const bool vec = __shfl_sync(kAll, dw, kLaneVec) != 0u;
            uint32_t *md = reinterpret_cast<uint32_t *>(&meta[s]);
            if (lane < 28) md[lane] = dw;
            uint8_t *stage = stage0 + s * stage_bytes;
            if (MODE & kModeApply) {
                // the centre and dispersion of the tile's windows ride along with the stage
                const int32_t *med = reinterpret_cast<const int32_t *>(ptr(dw, kLaneMed));
                const int32_t *mad = reinterpret_cast<const int32_t *>(ptr(dw, kLaneMad));
                if (static_cast<uint32_t>(lane) < nw && nw <= kApplyTileWindows) {
                    int2 *amd = reinterpret_cast<int2 *>(gb + L.amd) + s * kApplyTileWindows;
                    amd[lane] = make_int2(med[w0 + lane], mad[w0 + lane]);
                }
            }
            const uint8_t *src = in + static_cast<int64_t>(w0) * W * BPS;
            const uint32_t bulk = vec ? (tbytes & ~15u) : 0u, rem = tbytes & 15u;
            if (vec && static_cast<uint32_t>(lane) < rem) stage[bulk + lane] = src[bulk + lane];
            __syncwarp();
            if (lane == 0) {
                meta[s].tidx = t;
                mbar_arrive_tx(full_bar(s), bulk);
                if (bulk) bulk_g2s(smem_addr(stage), src, bulk, full_bar(s));
            }
            // advance the descriptor pipeline by one iteration
            dw = desc_word(t1, tw1);
            const int t2 = __shfl_sync(kAll, pend, 0);
            tw1 = tile_word(t2);
            if (lane == 0) pend = t2 < ntiles ? grab(it + 3) : ntiles;
            t0 = t1;
            t1 = t2;
        }
        // drain: every armed stage has landed before the copy warp leaves
        if (lane == 0) {
            for (int i = issued - stages < 0 ? 0 : issued - stages; i < issued; ++i)
                mbar_wait_bounded(full_bar(i % stages), (i / stages) & 1, kWaitTimeoutNs);
        }
        return;
    }

    // ---------------- consumer warps of group g
    if (inject_timeout && blockIdx.x == 0 && g == 0 && tid == 0) {
        if (!mbar_wait_bounded(inj_bar, 0, kInjectTimeoutNs)) atomicOr(p.status, kStatusTimeout);
    }
    if constexpr (BITS == 8 && G == 1 && (MODE & kModeWarpSplit) != 0) {
        if (!split_consumers<MODE & (3 | kModeFlaggedOnly), CW>(sm, gb, L, meta, stage0, stages, stage_bytes, bar0, p,
                                                              tid)) {
            atomicOr(p.status, kStatusTimeout);
            atomicExch(&sm.ctl->abort, 1u);
        }
        named_bar(3, T);  // every consumer thread of the CTA
        if (tid == 0 && sm.ctl->flagged) atomicAdd(p.flagged, sm.ctl->flagged);
        return;
    }
    int par = 0;  // window parity
    bool timed_out = false;
    RowSums rs = {{0u, 0u}};
    // the table holds the per-window path's running sums (multi-window tiles need it zero)
    bool dirty = false;
    for (int it = 0;; ++it) {
        const int s = it % stages;
        const int u = it / stages;
        // every consumer thread waits for the stage itself (bounded). The first named barrier
        // after the wait is always a bar.red.or, so a thread that timed out and the others
        // agree on leaving.
        const bool ok = mbar_wait_bounded(full_bar(s), u & 1, kWaitTimeoutNs);
        const int t = ok ? meta[s].tidx : -2;
        if (t < 0) {  // end of the work list (-1, seen alike by every thread) or a timeout (-2)
            timed_out = named_bar_or(sm.bar_id, T, t == -2);
            break;
        }
        const Tile tl = meta[s].tile;
        const Seg &sg = meta[s].seg;
        uint8_t *stage = stage0 + s * stage_bytes;
        if (!sg.vec) {
            const uint8_t *src = sg.in + static_cast<int64_t>(tl.w0) * sg.W * BPS;
            for (int i = tid; i < static_cast<int>(tl.bytes); i += T) stage[i] = src[i];
            if (named_bar_or(sm.bar_id, T, false)) {
                timed_out = true;
                break;
            }
        }
        bool alive = true;
        if constexpr (BITS == 8 && (MODE & kModeApply) != 0 && (MODE & ~(kModeApply | 3)) == 0) {
            // a tile of full windows of 2^lw >= 512 aligned samples goes through in one pass
            const uint32_t W = static_cast<uint32_t>(sg.W);
            if (sg.vec && tl.nw <= static_cast<uint32_t>(kApplyTileWindows) && W >= 512u && (W & (W - 1u)) == 0u &&
                tl.bytes == tl.nw * W) {
                const int2 *amd = reinterpret_cast<const int2 *>(gb + L.amd) + s * kApplyTileWindows;
                alive = process_tile_apply8<MODE, T>(sm, stage, tl, sg, amd, p, tid, par, 31 - __clz(static_cast<int>(W)),
                                                     empty_bar(s), true);
                par ^= 1;
                if (!alive) {
                    timed_out = true;
                    break;
                }
                continue;
            }
        }
        if constexpr (BITS == 8 && G == 1 && (MODE & kModeMulti) != 0) {
            // several small full windows of 2^lw samples: eight (W <= 2048, or a tile of eight or
            // more) or four at a time share the histogram table, the reduce, the barriers and the
            // searches
            const uint32_t W = static_cast<uint32_t>(sg.W);
            if (sg.vec && tl.nw >= 2u && W >= 512u && W <= 8192u && (W & (W - 1u)) == 0u && tl.bytes == tl.nw * W) {
                if (dirty) {
                    zero_shared(sm.hist, 32768, tid, T);
                    named_bar(sm.bar_id, T);
                    dirty = false;
                }
                const int lw = 31 - __clz(static_cast<int>(W));
                const uint32_t K = (W <= 2048u || tl.nw >= 8u) ? 8u : 4u;
                for (uint32_t k0 = 0; k0 < tl.nw && alive; k0 += K) {
                    const int nwk = static_cast<int>(tl.nw - k0 < K ? tl.nw - k0 : K);
                    const uint32_t rel = k0 + K >= tl.nw ? empty_bar(s) : 0u;
                    if (K == 8u)
                        alive = process_tile_multi8<MODE & ~kModeMulti, T, 8>(sm, stage + (k0 << lw), sg, tl.w0 + k0,
                                                                              nwk, lw, p, tid, par, rel, true);
                    else
                        alive = process_tile_multi8<MODE & ~kModeMulti, T, 4>(sm, stage + (k0 << lw), sg, tl.w0 + k0,
                                                                              nwk, lw, p, tid, par, rel, true);
                    par ^= 1;
                }
                rs = {{0u, 0u}};  // the reduce left the table zero
                if (!alive) {
                    timed_out = true;
                    break;
                }
                continue;
            }
            dirty = true;
        }
        for (uint32_t k = 0; k < tl.nw && alive; ++k) {
            const int64_t widx = static_cast<int64_t>(tl.w0) + k;
            const Win win = make_win(sg, widx, stage + k * sg.W * BPS, (MODE & (kModeF16 | kModeBF16)) ? 2 : BPS);
            const int2 *amd = ((MODE & kModeApply) && tl.nw <= kApplyTileWindows)
                                  ? reinterpret_cast<const int2 *>(gb + L.amd) + s * kApplyTileWindows + k
                                  : nullptr;
            alive = process_window<BITS, MODE, T, Geo<BITS>::row_bytes(G)>(
                sm, win, sg, widx, p, tid, par, k + 1 == tl.nw ? empty_bar(s) : 0u, true, rs, amd,
                (MODE & kModeCopies) ? segs + tl.seg : nullptr);
            par ^= 1;
        }
        if (!alive) {
            timed_out = true;
            break;
        }
    }
    if (timed_out && tid == 0) {
        atomicOr(p.status, kStatusTimeout);
        atomicExch(&sm.ctl->abort, 1u);
    }
    // the group's flagged total, once every warp of the group has finished
    named_bar(sm.bar_id, T);
    if (tid == 0 && sm.ctl->flagged) atomicAdd(p.flagged, sm.ctl->flagged);
}

// ------------------------------------------------------------------ plain kernel
template <int BITS, int MODE, int CW>
__global__ void __launch_bounds__(CW * 32) stream_kernel(Seg sg, int64_t w_begin, Params p) {
    constexpr int T = CW * 32;
    constexpr int BPS = Geo<BITS>::kBps;
    extern __shared__ __align__(128) uint8_t smem[];
    if (BITS == 8 && smem_addr(smem) != kDynSmemShared) {
        if (threadIdx.x == 0) atomicOr(p.status, kStatusLayout);
        return;
    }
    const Layout L = layout<BITS>(p.ncopies, 1, align_up(sg.W * Geo<BITS>::kBps, 128), CW, 1, MODE);  // as the host
    const Shm sm = group_view<BITS>(smem, L, 0, p.ncopies);
    const int tid = threadIdx.x;
    uint8_t *buf = smem + L.stage;
    zero_shared(smem, L.stage, tid, T);
    const int64_t w = w_begin + blockIdx.x;
    const int64_t s0 = w * sg.W;
    const int n = static_cast<int>(sg.len - s0 < sg.W ? sg.len - s0 : sg.W);
    const int nbytes = n * BPS;
    const uint8_t *src = sg.in + s0 * BPS;
    if (sg.vec) {
        const int nfull = nbytes >> 4;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *b4 = reinterpret_cast<uint4 *>(buf);
        for (int c = tid; c < nfull; c += T) b4[c] = __ldcs(s4 + c);
        for (int i = nfull * 16 + tid; i < nbytes; i += T) buf[i] = src[i];
    } else {
        for (int i = tid; i < nbytes; i += T) buf[i] = src[i];
    }
    __syncthreads();
    const Win win = make_win(sg, w, buf, BPS);
    RowSums rs = {{0u, 0u}};
    process_window<BITS, MODE, T, Geo<BITS>::row_bytes(1)>(sm, win, sg, w, p, tid, 0, 0u, true, rs);
    __syncthreads();
    if (tid == 0 && sm.ctl->flagged) atomicAdd(p.flagged, sm.ctl->flagged);
}

// ------------------------------------------------------------------ host-side dispatch
// Raise the dynamic shared-memory cap of one kernel instantiation, once per process. The tag
// parameters make the static once-flag distinct for every instantiation.
template <int KIND, int BITS, int MODE, int CW, int G, typename K>
inline cudaError_t allow_smem(K kernel) {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [&] {
        err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    return err;
}

template <int BITS, int MODE, int CW, int G>
cudaError_t persistent_launch_t(const Shape &s, int grid, const Seg *segs, const Tile *tiles, int ntiles,
                                const Params &p, unsigned *counter, int inject, cudaStream_t st) {
    auto k = persistent_kernel<BITS, MODE, CW, G>;
    cudaError_t e = allow_smem<0, BITS, MODE, CW, G>(k);
    if (e != cudaSuccess) return e;
    const Layout L = layout<BITS>(p.ncopies, s.stages, s.stage_bytes, CW, G, MODE);
    k<<<grid, G * (CW + 1) * 32, L.total, st>>>(segs, tiles, ntiles, p, s.stages, s.stage_bytes, s.dynamic_tiles,
                                                counter, inject);
    return cudaGetLastError();
}

template <int BITS, int MODE, int CW, int G>
int persistent_occ_t(const Shape &s) {
    auto k = persistent_kernel<BITS, MODE, CW, G>;
    if (allow_smem<0, BITS, MODE, CW, G>(k) != cudaSuccess) return 0;
    const Layout L = layout<BITS>(s.hist_copies, s.stages, s.stage_bytes, CW, G, MODE);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, G * (CW + 1) * 32, L.total) != cudaSuccess) return 0;
    return n;
}

template <int BITS, int MODE, int CW>
cudaError_t stream_launch_t(const Seg &sg, int64_t w_begin, int64_t nw, const Params &p, cudaStream_t st) {
    auto k = stream_kernel<BITS, MODE, CW>;
    cudaError_t e = allow_smem<1, BITS, MODE, CW, 1>(k);
    if (e != cudaSuccess) return e;
    const Layout L = layout<BITS>(p.ncopies, 1, align_up(sg.W * Geo<BITS>::kBps, 128), CW, 1, MODE);
    for (int64_t b = 0; b < nw; b += 0x7FFFFFFF) {
        const int64_t gsz = nw - b < 0x7FFFFFFF ? nw - b : 0x7FFFFFFF;
        k<<<static_cast<unsigned>(gsz), CW * 32, L.total, st>>>(sg, w_begin + b, p);
    }
    return cudaGetLastError();
}

// Template dispatch over (mode, consumer warps[, groups]).
#define RFI_CASE_MCG(BITS, FN, M, C, G, ...) \
    case (M * 1000 + C * 10 + G): return FN<BITS, M, C, G>(__VA_ARGS__);
#define RFI_CASES_CG(BITS, FN, M, ...)                                                       \
    RFI_CASE_MCG(BITS, FN, M, 4, 1, __VA_ARGS__) RFI_CASE_MCG(BITS, FN, M, 8, 1, __VA_ARGS__)  \
    RFI_CASE_MCG(BITS, FN, M, 16, 1, __VA_ARGS__) RFI_CASE_MCG(BITS, FN, M, 4, 2, __VA_ARGS__) \
    RFI_CASE_MCG(BITS, FN, M, 8, 2, __VA_ARGS__)
#define RFI_DISPATCH_PERSISTENT(BITS, FN, MODE, CW, G, ...)        \
    do {                                                           \
        switch (MODE * 1000 + CW * 10 + G) {                       \
            RFI_CASES_CG(BITS, FN, 0, __VA_ARGS__)                 \
            RFI_CASES_CG(BITS, FN, 1, __VA_ARGS__)                 \
            RFI_CASES_CG(BITS, FN, 2, __VA_ARGS__)                 \
            RFI_CASES_CG(BITS, FN, 3, __VA_ARGS__)                 \
            default: break;                                        \
        }                                                          \
    } while (0)

#define RFI_DISPATCH_MODE_CW(BITS, FN, MODE, CW, ...)                                          \
    do {                                                                                       \
        switch (MODE * 100 + CW) {                                                             \
            case 4: return FN<BITS, 0, 4>(__VA_ARGS__);                                        \
            case 8: return FN<BITS, 0, 8>(__VA_ARGS__);                                        \
            case 16: return FN<BITS, 0, 16>(__VA_ARGS__);                                      \
            case 104: return FN<BITS, 1, 4>(__VA_ARGS__);                                      \
            case 108: return FN<BITS, 1, 8>(__VA_ARGS__);                                      \
            case 116: return FN<BITS, 1, 16>(__VA_ARGS__);                                     \
            case 204: return FN<BITS, 2, 4>(__VA_ARGS__);                                      \
            case 208: return FN<BITS, 2, 8>(__VA_ARGS__);                                      \
            case 216: return FN<BITS, 2, 16>(__VA_ARGS__);                                     \
            case 304: return FN<BITS, 3, 4>(__VA_ARGS__);                                      \
            case 308: return FN<BITS, 3, 8>(__VA_ARGS__);                                      \
            case 316: return FN<BITS, 3, 16>(__VA_ARGS__);                                     \
            default: break;                                                                    \
        }                                                                                      \
    } while (0)

}  // namespace dev
}  // namespace rfi
