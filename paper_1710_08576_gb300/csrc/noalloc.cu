// rfi_excise_noalloc: the batched persistent excision without a plan and without any
// allocation. Some callers cannot allocate device memory when they excise: a real-time
// receiver loop whose device memory is carved out once at start-up (any cudaMalloc/cudaFree
// there can synchronise the device and stall the sample stream), or a host whose memory budget
// is owned by another allocator. For them the work list, the segment table and the counters of
// the persistent kernel live in one fixed device array of this file (kScratchBytes), reserved
// when the library is loaded and kept by every GPU that loads it until the process exits.
//
// Rules, for callers:
//   - the first call on a device looks up the array's device address (cudaGetSymbolAddress,
//     once per device, with that device current); make that first call before any stream
//     capture;
//   - every call uses the same array and leaves the last call's contents in it; the counters
//     are cleared at the start of each call. Calls whose work overlaps on the GPU (two streams,
//     two threads) race on the array and must be serialised by the caller;
//   - at most kMaxStreams streams and kMaxTiles work-list entries per call; larger requests are
//     rejected with RFI_ERR_UNSUPPORTED before anything is enqueued;
//   - device-detected errors are returned only when the caller asks for the totals (which
//     synchronises the stream); a CUDA error already pending on entry is left in place and the
//     call returns RFI_ERR_CUDA without enqueueing anything.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "rfi.h"
#include "internal.h"

namespace rfi {
namespace {

constexpr int kMaxStreams = RFI_NOALLOC_MAX_STREAMS;
constexpr int kMaxTiles = RFI_NOALLOC_MAX_TILES;
constexpr int kMaxDevices = 64;

struct Counters {
    unsigned tile_counter;
    uint32_t status;
    unsigned long long flagged;
};

constexpr size_t kCtrBytes = 256;
constexpr size_t kSegBytes = sizeof(Seg) * kMaxStreams;
constexpr size_t kTileBytes = sizeof(Tile) * kMaxTiles;
constexpr size_t kScratchBytes = kCtrBytes + kSegBytes + kTileBytes;
static_assert(kScratchBytes == RFI_NOALLOC_SCRATCH_BYTES, "the header states the array's size");

static __device__ __align__(256) uint8_t g_scratch[kScratchBytes];

std::mutex g_mu;
uint8_t *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
rfi_status scratch_address(uint8_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RFI_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return RFI_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<uint8_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return RFI_OK;
}

// Work-list layout of one call, passed by value to the tile writer.
struct TileSpec {
    int32_t nseg;
    int32_t ntiles;
    int32_t bps;
    int32_t tile_off[kMaxStreams + 1];  // first tile of each segment
    int32_t per[kMaxStreams];           // windows per tile
    int32_t nwin[kMaxStreams];
    int64_t len[kMaxStreams];
    int32_t W[kMaxStreams];
};

// One thread per work-list entry: stream-major order, `per` consecutive windows per tile.
__global__ void write_tiles_kernel(Tile *tiles, TileSpec spec) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= spec.ntiles) return;
    int s = 0;
    while (s + 1 < spec.nseg && spec.tile_off[s + 1] <= t) ++s;
    const int64_t w0 = static_cast<int64_t>(t - spec.tile_off[s]) * spec.per[s];
    const int64_t nw = min(static_cast<int64_t>(spec.per[s]), spec.nwin[s] - w0);
    const int64_t s0 = w0 * spec.W[s];
    const int64_t s1 = min(spec.len[s], (w0 + nw) * spec.W[s]);
    Tile tl;
    tl.seg = static_cast<uint32_t>(s);
    tl.w0 = static_cast<uint32_t>(w0);
    tl.nw = static_cast<uint32_t>(nw);
    tl.bytes = static_cast<uint32_t>((s1 - s0) * spec.bps);
    tiles[t] = tl;
}

}  // namespace
}  // namespace rfi

using namespace rfi;

extern "C" rfi_status rfi_excise_noalloc(const rfi_plan_desc *d, const void *const *in, void *const *out,
                                         uint32_t *const *mask, uint32_t *const *counts,
                                         int32_t *const *median, int32_t *const *mad, rfi_totals *totals,
                                         void *stream) {
    // ---- validation (the same rules as rfi_plan_create)
    if (!d || !in || !out) return RFI_ERR_INVALID_ARG;
    if (d->sample_bits != 8 && d->sample_bits != 12) return RFI_ERR_INVALID_ARG;
    if (d->num_streams < 1 || !d->stream_len || !d->window_len) return RFI_ERR_INVALID_ARG;
    if (!(d->k > 0.0) || !std::isfinite(d->k) || d->k > 1.0e6) return RFI_ERR_INVALID_ARG;
    if (d->mode < RFI_REPLACE_ZERO || d->mode > RFI_REPLACE_NOISE) return RFI_ERR_INVALID_ARG;
    if (d->flags & ~(RFI_PLAN_BATCHED)) return RFI_ERR_INVALID_ARG;
    if (d->num_streams > kMaxStreams) return RFI_ERR_UNSUPPORTED;
    if (d->mom_windows < 0 || d->mom_windows > (1 << 20)) return RFI_ERR_INVALID_ARG;
    if (d->mom_windows >= 2) return RFI_ERR_UNSUPPORTED;  // per-window MAD only
    if (d->out_format != RFI_OUT_SAME) return d->out_format < 0 || d->out_format > 2 ? RFI_ERR_INVALID_ARG
                                                                                    : RFI_ERR_UNSUPPORTED;
    const int64_t kq = static_cast<int64_t>(std::floor(d->k * 1.4826 * 65536.0 + 0.5));
    if (kq < 1) return RFI_ERR_INVALID_ARG;
    const int S = d->num_streams;
    const int bps = d->sample_bits == 8 ? 1 : 2;
    int64_t maxwb = 0;
    for (int i = 0; i < S; ++i) {
        if (d->stream_len[i] < 1 || d->window_len[i] < 1 || d->window_len[i] > 65536) return RFI_ERR_INVALID_ARG;
        if (!in[i] || !out[i]) return RFI_ERR_INVALID_ARG;
        if (bps == 2 && ((reinterpret_cast<uintptr_t>(in[i]) | reinterpret_cast<uintptr_t>(out[i])) & 1))
            return RFI_ERR_ALIGNMENT;
        if (mask && mask[i] && (reinterpret_cast<uintptr_t>(mask[i]) & 3)) return RFI_ERR_ALIGNMENT;
        if (counts && counts[i] && (reinterpret_cast<uintptr_t>(counts[i]) & 3)) return RFI_ERR_ALIGNMENT;
        if (median && median[i] && (reinterpret_cast<uintptr_t>(median[i]) & 3)) return RFI_ERR_ALIGNMENT;
        if (mad && mad[i] && (reinterpret_cast<uintptr_t>(mad[i]) & 3)) return RFI_ERR_ALIGNMENT;
        maxwb = std::max<int64_t>(maxwb, std::min<int64_t>(d->window_len[i], d->stream_len[i]) * bps);
    }

    // ---- an error pending from the caller's earlier CUDA work is left for the caller: refuse
    // before enqueueing anything, so that the launch checks below see only this call's launches
    if (cudaPeekAtLastError() != cudaSuccess) return RFI_ERR_CUDA;

    // ---- launch shape (fixed; no tuning runs, which would need scratch buffers)
    Shape sh{};
    sh.consumer_warps = 8;
    sh.groups = 1;
    sh.hist_copies = bps == 1 ? 1 : 2;
    sh.dynamic_tiles = 1;
    const int min_stage = static_cast<int>((maxwb + 127) / 128 * 128);
    // work list: grow the stage (windows per tile) until the list fits the scratch area
    TileSpec spec;
    std::memset(&spec, 0, sizeof(spec));
    spec.nseg = S;
    spec.bps = bps;
    int ntiles = 0;
    for (int stage = std::max(min_stage, 16384);; stage *= 2) {
        if (stage > 227 * 1024) return RFI_ERR_UNSUPPORTED;
        int64_t nt = 0;
        for (int i = 0; i < S; ++i) {
            const int64_t wb = static_cast<int64_t>(d->window_len[i]) * bps;
            const int64_t per = (wb % 16 == 0) ? std::max<int64_t>(1, stage / wb) : 1;
            const int64_t nw = (d->stream_len[i] + d->window_len[i] - 1) / d->window_len[i];
            spec.tile_off[i] = static_cast<int32_t>(std::min<int64_t>(nt, kMaxTiles + 1));
            spec.per[i] = static_cast<int32_t>(per);
            spec.nwin[i] = static_cast<int32_t>(std::min<int64_t>(nw, 0x7FFFFFFF));
            spec.len[i] = d->stream_len[i];
            spec.W[i] = d->window_len[i];
            nt += (nw + per - 1) / per;
        }
        if (nt <= kMaxTiles) {
            spec.tile_off[S] = static_cast<int32_t>(nt);
            ntiles = static_cast<int>(nt);
            sh.stage_bytes = stage;
            break;
        }
    }
    sh.stages = 2;
    while (sh.stages > 1 && persistent_smem_bytes(d->sample_bits, d->mode, sh) > 227u * 1024u) --sh.stages;
    if (persistent_smem_bytes(d->sample_bits, d->mode, sh) > 227u * 1024u) return RFI_ERR_UNSUPPORTED;
    const int occ = persistent_occupancy(d->sample_bits, d->mode, sh);
    if (occ < 1) return RFI_ERR_UNSUPPORTED;
    sh.ctas_per_sm = std::min(occ, 3);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RFI_ERR_CUDA;
    spec.ntiles = ntiles;

    // ---- the fixed scratch area
    uint8_t *scr = nullptr;
    rfi_status rs = scratch_address(&scr);
    if (rs != RFI_OK) return rs;
    Counters *ctr = reinterpret_cast<Counters *>(scr);
    Seg *segs = reinterpret_cast<Seg *>(scr + kCtrBytes);
    Tile *tiles = reinterpret_cast<Tile *>(scr + kCtrBytes + kSegBytes);

    Seg host_segs[kSegBatch];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ctr, 0, sizeof(Counters), st) != cudaSuccess) return RFI_ERR_CUDA;
    for (int b = 0; b < S; b += kSegBatch) {
        const int n = std::min(kSegBatch, S - b);
        for (int j = 0; j < n; ++j) {
            const int i = b + j;
            Seg &g = host_segs[j];
            std::memset(&g, 0, sizeof(Seg));
            g.in = static_cast<const uint8_t *>(in[i]);
            g.out = static_cast<uint8_t *>(out[i]);
            g.mask = mask ? mask[i] : nullptr;
            g.counts = counts ? counts[i] : nullptr;
            g.med = median ? median[i] : nullptr;
            g.mad = mad ? mad[i] : nullptr;
            g.len = d->stream_len[i];
            g.abs0 = 0;
            g.W = d->window_len[i];
            g.stream_id = d->stream_id ? d->stream_id[i] : static_cast<uint32_t>(i);
            g.mask_words = (d->window_len[i] + 31) / 32;
            g.vec = ((reinterpret_cast<uintptr_t>(in[i]) | reinterpret_cast<uintptr_t>(out[i])) % 16 == 0) &&
                    (static_cast<int64_t>(d->window_len[i]) * bps) % 16 == 0;
        }
        if (launch_write_segs(segs + b, host_segs, n, st) != cudaSuccess) return RFI_ERR_CUDA;
    }
    write_tiles_kernel<<<(ntiles + 255) / 256, 256, 0, st>>>(tiles, spec);
    if (cudaGetLastError() != cudaSuccess) return RFI_ERR_CUDA;

    Params p{};
    p.kq = kq;
    p.seed = d->seed;
    const int32_t lo = bps == 1 ? -128 : -2048, hi = bps == 1 ? 127 : 2047;
    p.cval = std::min(hi, std::max(lo, d->const_value));
    p.ncopies = sh.hist_copies;
    p.status = &ctr->status;
    p.flagged = &ctr->flagged;
    set_round_keys(p);
    const int grid = std::max(1, std::min(ntiles, sms * sh.ctas_per_sm));
    if (launch_persistent(d->sample_bits, d->mode, sh, grid, segs, tiles, ntiles, p, &ctr->tile_counter, 0, st) !=
        cudaSuccess)
        return RFI_ERR_CUDA;

    if (totals) {
        Counters h;
        if (cudaMemcpyAsync(&h, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return RFI_ERR_CUDA;
        uint64_t nwin = 0;
        for (int i = 0; i < S; ++i) nwin += static_cast<uint64_t>(spec.nwin[i]);
        const rfi_status dev_st = (h.status & kStatusTimeout)       ? RFI_ERR_TIMEOUT
                                  : (h.status & kStatusLayout)      ? RFI_ERR_UNSUPPORTED
                                  : (h.status & kStatusSampleRange) ? RFI_ERR_SAMPLE_RANGE
                                                                    : RFI_OK;
        totals->windows = nwin;
        totals->flagged = h.flagged;
        totals->device_status = static_cast<int32_t>(dev_st);
        return dev_st;
    }
    return RFI_OK;
}
