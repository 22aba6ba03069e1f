// librfi C ABI: plans, the batched and per-stream excision calls, statistics and the host
// pipelined variant. Semantics are stated in include/rfi.h.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "rfi.h"
#include "internal.h"
#include "plan_impl.h"

namespace {

using rfi::Seg;
using rfi::Shape;
using rfi::Tile;

#define RFI_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return RFI_ERR_CUDA;      \
    } while (0)

bool valid_shape(const rfi_launch_shape &s) {
    return s.consumer_warps >= 0 && s.stages >= 0 && s.stages <= 8 && s.ctas_per_sm >= 0 &&
           s.ctas_per_sm <= 4 && s.stage_bytes >= 0 && s.stage_bytes <= 227 * 1024 && s.dynamic_tiles >= 0 &&
           s.dynamic_tiles <= 2 && s.hist_copies >= 0 && s.hist_copies <= 4 && s.hist_copies != 3 &&
           (s.consumer_warps == 0 || s.consumer_warps == 4 || s.consumer_warps == 8 || s.consumer_warps == 16) &&
           s.groups >= 0 && s.groups <= 2 && !(s.groups == 2 && s.consumer_warps == 16) && s.warp_split >= 0 &&
           s.warp_split <= 2;
}

}  // namespace

namespace rfi {

rfi_status plan_choose_shape(rfi_plan_s *P, const rfi_launch_shape *req) {
    Shape s;
    const int bps = P->bits == 8 ? 1 : 2;
    int64_t maxwb = 0;
    bool uniform = true;
    for (int i = 0; i < P->S; ++i) {
        const int64_t first = std::min<int64_t>(P->W[i], P->len[i]) * bps;
        maxwb = std::max<int64_t>(maxwb, first);
        if (P->W[i] != P->W[0]) uniform = false;
    }
    const int min_stage = static_cast<int>((maxwb + 127) / 128 * 128);
    s.consumer_warps = (req && req->consumer_warps) ? req->consumer_warps : 8;
    s.groups = (req && req->groups) ? req->groups : 1;
    if (P->out_format != RFI_OUT_SAME) {  // the output formats are built for one group of 8 warps
        if ((req && req->groups > 1) || (req && req->consumer_warps && req->consumer_warps != 8))
            return RFI_ERR_UNSUPPORTED;
        s.consumer_warps = 8;
        s.groups = 1;
    }
    if (P->kmom >= 2 || P->power || P->ncopy > 0) {  // built for one group of 4 or 8 consumer warps
        if ((req && req->groups > 1) || s.consumer_warps > 8) return RFI_ERR_UNSUPPORTED;
        s.groups = 1;
    }
    // a Median-of-MAD plan on 4096-sample windows takes one 32 KiB stage: tiles of eight windows
    // share one histogram table in the multi-window estimation pass
    bool mom4096 = P->kmom >= 2 && P->bits == 8;
    for (int i = 0; i < P->S && mom4096; ++i) mom4096 = P->W[i] == 4096 && P->len[i] >= 8 * 4096;
    const bool mom_stage = mom4096 && !(req && (req->stage_bytes || req->stages));
    s.stage_bytes = std::max(min_stage, (req && req->stage_bytes) ? req->stage_bytes : (mom_stage ? 32768 : 16384));
    s.stage_bytes = (s.stage_bytes + 127) / 128 * 128;
    s.stages = (req && req->stages) ? req->stages : (mom_stage ? 1 : 2);
    s.hist_copies = P->bits == 8 ? 1 : ((req && req->hist_copies) ? req->hist_copies : 2);
    s.dynamic_tiles = (req && req->dynamic_tiles) ? req->dynamic_tiles : (uniform ? 2 : 1);
    const int want_ctas = (req && req->ctas_per_sm) ? req->ctas_per_sm : 4;  // as many as fit, up to 4
    // the shape is sized for the kernel with the histogram (the MoM stats pass)
    const int kmode = P->kmom >= 2 ? plan_stats_mode(P) : plan_kernel_mode(P);
    if (persistent_smem_bytes(P->bits, kmode, s) > 227u * 1024u) {
        if (req && req->stages) return RFI_ERR_UNSUPPORTED;
        while (s.stages > 1 && persistent_smem_bytes(P->bits, kmode, s) > 227u * 1024u) --s.stages;
        if (persistent_smem_bytes(P->bits, kmode, s) > 227u * 1024u) return RFI_ERR_UNSUPPORTED;
    }
    const int occ = persistent_occupancy(P->bits, kmode, s);
    if (occ < 1) return cudaGetLastError() != cudaSuccess ? RFI_ERR_CUDA : RFI_ERR_UNSUPPORTED;
    s.ctas_per_sm = std::min(want_ctas, occ);
    P->grid_apply = 0;
    if (P->kmom >= 2) {
        const int occ_apply = persistent_occupancy(P->bits, kModeApply + (P->fill ? 0 : P->mode), s);
        if (occ_apply < 1) return cudaGetLastError() != cudaSuccess ? RFI_ERR_CUDA : RFI_ERR_UNSUPPORTED;
        P->grid_apply = P->sm_count * occ_apply;  // clamped to the tile count with the grid
    }
    // the split-warp form only where it runs: int8 zero / constant / threshold, one group of 8
    s.warp_split = (req && req->warp_split) ? req->warp_split : 1;
    if (s.warp_split == 2 && !plan_warp_split_runs(P, s)) return RFI_ERR_UNSUPPORTED;
    P->shape = s;
    return RFI_OK;
}

bool plan_warp_split_runs(const rfi_plan_s *P, const Shape &s) {
    return P->kmom < 2 && !P->power && P->ncopy == 0 && P->out_format == RFI_OUT_SAME &&
           warp_split_runs(P->bits, plan_kernel_mode(P), s);
}

rfi_status plan_build_tiles(rfi_plan_s *P) {
    const int bps = P->bits == 8 ? 1 : 2;
    std::vector<Tile> tiles;
    for (int i = 0; i < P->S; ++i) {
        const int64_t wb = static_cast<int64_t>(P->W[i]) * bps;
        int64_t per = (wb % 16 == 0) ? std::max<int64_t>(1, P->shape.stage_bytes / wb) : 1;
        if (P->kmom >= 2) per = std::min<int64_t>(per, kApplyTileWindows);
        for (int64_t w0 = 0; w0 < P->nwin[i]; w0 += per) {
            const int64_t nw = std::min<int64_t>(per, P->nwin[i] - w0);
            const int64_t s0 = w0 * P->W[i];
            const int64_t s1 = std::min<int64_t>(P->len[i], (w0 + nw) * P->W[i]);
            Tile t;
            t.seg = static_cast<uint32_t>(i);
            t.w0 = static_cast<uint32_t>(w0);
            t.nw = static_cast<uint32_t>(nw);
            t.bytes = static_cast<uint32_t>((s1 - s0) * bps);
            tiles.push_back(t);
        }
    }
    // largest tiles first (a longest-processing-time order for the dynamic queue); stable keeps
    // each stream's tiles in stream order
    std::stable_sort(tiles.begin(), tiles.end(), [](const Tile &a, const Tile &b) { return a.bytes > b.bytes; });
    if (tiles.size() > 0x7FFFFFFFu) return RFI_ERR_UNSUPPORTED;
    P->tiles_host = std::move(tiles);
    P->ntiles = static_cast<int>(P->tiles_host.size());
    P->grid = std::max(1, std::min(P->ntiles, P->sm_count * P->shape.ctas_per_sm));
    if (P->kmom >= 2) P->grid_apply = std::max(1, std::min(P->ntiles, P->grid_apply));
    return RFI_OK;
}

rfi_status plan_alloc_workspace(rfi_plan_s *P) {
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t seg_b = al(sizeof(Seg) * plan_nsegs(P));
    const size_t tile_b = al(sizeof(Tile) * P->tiles_host.size());
    const size_t md_b = al(sizeof(int32_t) * P->total_windows);
    const size_t ctr_b = 256;
    const bool mom = P->kmom >= 2;
    if (mom) {
        P->mchunks.clear();
        for (int i = 0; i < P->S; ++i)
            for (int64_t a = 0; a < P->nwin[i]; a += kMomChunk)
                P->mchunks.push_back(MomChunk{P->woff[i], static_cast<int32_t>(a),
                                              static_cast<int32_t>(std::min<int64_t>(a + kMomChunk, P->nwin[i]))});
    }
    const size_t mc_b = mom ? al(sizeof(MomChunk) * P->mchunks.size()) : 0;
    const size_t pw_b = P->power ? al(2 * sizeof(uint64_t) * P->total_windows) : 0;
    const size_t var_b = al(sizeof(Variant) * P->variants.size());
    // the fill pass: unit offsets of the segments (256 mask words a unit; for small windows of a
    // multiple of 128 samples the units run over the words of the whole segment, else over
    // those of each window)
    std::vector<uint32_t> fwin;
    if (P->fill) {
        fwin.push_back(0);
        P->fill_packed = false;
        for (int i = 0; i < P->S; ++i) {
            const bool pk = fill_packs(P->W[i]);
            const int64_t units = pk ? ((P->len[i] + 31) / 32 + 255) / 256
                                     : P->nwin[i] * (((P->W[i] + 31) / 32 + 255) / 256);
            P->fill_packed = P->fill_packed || pk;
            fwin.push_back(fwin.back() + static_cast<uint32_t>(units));
        }
        P->nfwin = fwin.back();
        P->fill_grid = noise_fill_grid(P->sm_count, P->fill_packed);
    }
    // one allocation, each array at the next 256-byte boundary
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += al(bytes);
        return o;
    };
    const size_t o_ctr = take(ctr_b), o_seg = take(seg_b), o_tile = take(tile_b);
    const size_t o_med = take(md_b), o_mad = take(md_b);
    const size_t o_mom = mom ? take(md_b) : 0, o_mc = mom ? take(mc_b) : 0;
    const size_t o_pw = P->power ? take(pw_b) : 0;
    const size_t o_var = take(var_b);
    const size_t o_fw = P->fill ? take(sizeof(uint32_t) * fwin.size()) : 0;
    P->ws_bytes = off;
    if (P->ws) cudaFree(P->ws);
    P->ws = nullptr;
    if (cudaMalloc(&P->ws, P->ws_bytes) != cudaSuccess) {
        cudaGetLastError();
        P->ws = nullptr;
        return RFI_ERR_OOM;
    }
    uint8_t *b = static_cast<uint8_t *>(P->ws);
    P->d_ctr = reinterpret_cast<DevCounters *>(b + o_ctr);
    P->d_segs = reinterpret_cast<Seg *>(b + o_seg);
    P->d_tiles = reinterpret_cast<Tile *>(b + o_tile);
    P->d_med = reinterpret_cast<int32_t *>(b + o_med);
    P->d_mad = reinterpret_cast<int32_t *>(b + o_mad);
    RFI_CUDA(cudaMemset(P->ws, 0, P->ws_bytes));
    RFI_CUDA(cudaMemcpy(P->d_tiles, P->tiles_host.data(), sizeof(Tile) * P->tiles_host.size(),
                        cudaMemcpyHostToDevice));
    if (mom) {
        P->d_mom = reinterpret_cast<int32_t *>(b + o_mom);
        P->d_mchunks = reinterpret_cast<MomChunk *>(b + o_mc);
        RFI_CUDA(cudaMemcpy(P->d_mchunks, P->mchunks.data(), sizeof(MomChunk) * P->mchunks.size(),
                            cudaMemcpyHostToDevice));
    }
    if (P->power) P->d_pow = reinterpret_cast<uint64_t *>(b + o_pw);
    if (!P->variants.empty()) {
        P->d_var = reinterpret_cast<Variant *>(b + o_var);
        RFI_CUDA(cudaMemcpy(P->d_var, P->variants.data(), sizeof(Variant) * P->variants.size(),
                            cudaMemcpyHostToDevice));
    }
    if (P->fill) {
        P->d_fwin = reinterpret_cast<uint32_t *>(b + o_fw);
        RFI_CUDA(cudaMemcpy(P->d_fwin, fwin.data(), sizeof(uint32_t) * fwin.size(), cudaMemcpyHostToDevice));
    }
    P->segs_valid = false;
    return RFI_OK;
}

Params plan_params(const rfi_plan_s *P) {
    Params p{};
    p.kq = P->kq;
    p.seed = P->seed;
    p.cval = P->cval;
    p.ncopies = P->shape.hist_copies;
    p.status = &P->d_ctr->status;
    p.flagged = &P->d_ctr->flagged;
    set_round_keys(p);
    p.copies = P->ncopy | (P->S << 4);
    p.var_off = P->d_var ? static_cast<int32_t>(reinterpret_cast<const char *>(P->d_var) -
                                                reinterpret_cast<const char *>(&P->d_ctr->status))
                         : 0;
    return p;
}

// Enqueue the persistent launch (with its counter reset) on st.
rfi_status plan_enqueue_batched(rfi_plan_s *P, cudaStream_t st) {
    RFI_CUDA(cudaMemsetAsync(P->d_ctr, 0, sizeof(DevCounters), st));
    const int inject = (P->flags & RFI_PLAN_INJECT_TIMEOUT) ? 1 : 0;
    if (P->kmom < 2) {
        const Params p = plan_params(P);
        RFI_CUDA(launch_persistent(P->bits, plan_kernel_mode(P), P->shape, P->grid, P->d_segs, P->d_tiles,
                                   P->ntiles, p, &P->d_ctr->tile_counter, inject, st));
        if (P->fill) RFI_CUDA(launch_noise_fill(P->bits, P->fill_packed, P->d_segs, P->S, P->d_fwin, P->nfwin, p, P->fill_grid, st));
        return RFI_OK;
    }
    // Median of MAD (Eq. 3): M and D of every window, the sliding median of the MADs, then Eq. 1
    // and Eq. 2 with each window's M and its MoM (segment entries S..2S-1)
    const Params p = plan_params(P);
    RFI_CUDA(launch_persistent(P->bits, plan_stats_mode(P), P->shape, P->grid, P->d_segs, P->d_tiles, P->ntiles, p,
                               &P->d_ctr->tile_counter, inject, st));
    RFI_CUDA(launch_mom(P->bits, P->d_mchunks, static_cast<int>(P->mchunks.size()), P->d_mad, P->d_mom, P->kmom,
                        st));
    RFI_CUDA(cudaMemsetAsync(&P->d_ctr->tile_counter, 0, sizeof(unsigned), st));
    RFI_CUDA(launch_persistent(P->bits, kModeApply + (P->fill ? 0 : P->mode), P->shape, P->grid_apply, P->d_segs + P->S,
                               P->d_tiles, P->ntiles, p, &P->d_ctr->tile_counter, 0, st));
    // the apply segments hold each window's M and its MoM: the noise spread of Eq. 3
    if (P->fill)
        RFI_CUDA(launch_noise_fill(P->bits, P->fill_packed, P->d_segs + P->S, P->S, P->d_fwin, P->nfwin, p, P->fill_grid, st));
    return RFI_OK;
}

rfi_status plan_build_graph(rfi_plan_s *P) {
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    if (P->graph) cudaGraphDestroy(P->graph);
    P->gexec = nullptr;
    P->graph = nullptr;
    cudaStream_t cs;
    RFI_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    rfi_status rs = RFI_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rs = RFI_ERR_CUDA;
    } else {
        rs = plan_enqueue_batched(P, cs);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (rs == RFI_OK && e != cudaSuccess) rs = RFI_ERR_CUDA;
        if (rs == RFI_OK && cudaGraphInstantiate(&P->gexec, g, 0) != cudaSuccess) rs = RFI_ERR_CUDA;
        if (rs == RFI_OK) P->graph = g;
        else if (g) cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    return rs;
}

std::vector<Seg> plan_segs(const rfi_plan_s *P, const void *const *in, void *const *out, uint32_t *const *mask,
                           uint32_t *const *counts) {
    const int bps = P->bits == 8 ? 1 : 2;
    std::vector<Seg> segs(plan_nsegs(P));
    for (int i = 0; i < P->S; ++i) {
        Seg &g = segs[i];
        std::memset(&g, 0, sizeof(Seg));
        g.in = static_cast<const uint8_t *>(in[i]);
        g.out = static_cast<uint8_t *>(out[i]);
        g.mask = mask ? mask[i] : nullptr;
        if (P->fill && !g.mask) g.mask = P->d_fmask + P->fmask_off[i];  // the fill pass reads the flags
        g.counts = counts ? counts[i] : nullptr;
        g.med = P->d_med + P->woff[i];
        g.mad = P->d_mad + P->woff[i];
        g.power = P->power ? P->d_pow + 2 * P->woff[i] : nullptr;
        g.len = P->len[i];
        g.abs0 = 0;
        g.W = P->W[i];
        g.stream_id = P->sid[i];
        g.mask_words = (P->W[i] + 31) / 32;
        g.vec = ((reinterpret_cast<uintptr_t>(in[i]) | reinterpret_cast<uintptr_t>(out[i])) % 16 == 0) &&
                (static_cast<int64_t>(P->W[i]) * bps) % 16 == 0;
        if (P->kmom >= 2) {
            // apply pass: reads M and the MoM, writes the outputs; stats pass: writes M and D only
            Seg &a = segs[P->S + i];
            a = g;
            a.mad = P->d_mom + P->woff[i];
            g.out = const_cast<uint8_t *>(g.in);
            g.mask = nullptr;
            g.counts = nullptr;
        }
    }
    return segs;
}

rfi_status plan_check_buffers(const rfi_plan_s *P, const void *const *in, void *const *out,
                              uint32_t *const *mask, uint32_t *const *counts) {
    if (!in || !out) return RFI_ERR_INVALID_ARG;
    for (int i = 0; i < P->S; ++i) {
        if (!in[i] || !out[i]) return RFI_ERR_INVALID_ARG;
        if (P->write_flagged && in[i] != out[i]) return RFI_ERR_INVALID_ARG;
        if (P->bits == 12 && ((reinterpret_cast<uintptr_t>(in[i]) | reinterpret_cast<uintptr_t>(out[i])) & 1))
            return RFI_ERR_ALIGNMENT;
        if (P->out_format != RFI_OUT_SAME && (reinterpret_cast<uintptr_t>(out[i]) & 1)) return RFI_ERR_ALIGNMENT;
        if (mask && mask[i] && (reinterpret_cast<uintptr_t>(mask[i]) & 3)) return RFI_ERR_ALIGNMENT;
        if (counts && counts[i] && (reinterpret_cast<uintptr_t>(counts[i]) & 3)) return RFI_ERR_ALIGNMENT;
    }
    return RFI_OK;
}

}  // namespace rfi

using namespace rfi;

extern "C" {

const char *rfi_version(void) { return "librfi 1.0 (sm_103a)"; }

const char *rfi_status_string(rfi_status s) {
    switch (s) {
        case RFI_OK: return "ok";
        case RFI_ERR_INVALID_ARG: return "invalid argument";
        case RFI_ERR_UNSUPPORTED: return "unsupported request";
        case RFI_ERR_ALIGNMENT: return "misaligned buffer";
        case RFI_ERR_OOM: return "out of memory or over budget";
        case RFI_ERR_CUDA: return "CUDA runtime error";
        case RFI_ERR_SAMPLE_RANGE: return "12-bit sample outside [-2048, 2047]";
        case RFI_ERR_TIMEOUT: return "bounded device wait timed out";
        case RFI_ERR_BUSY: return "busy: no free slot";
    }
    return "unknown status";
}

static rfi_status plan_create(const rfi_plan_desc *d, int32_t nvar, const rfi_variant *vars, rfi_plan_t *out_plan);

rfi_status rfi_plan_create(const rfi_plan_desc *d, rfi_plan_t *out_plan) { return plan_create(d, 0, nullptr, out_plan); }

rfi_status rfi_plan_create_copies(const rfi_plan_desc *d, int32_t nvariants, const rfi_variant *variants,
                                  rfi_plan_t *out_plan) {
    if (!d || !out_plan || !variants || nvariants < 1 || nvariants > kMaxCopies) return RFI_ERR_INVALID_ARG;
    return plan_create(d, nvariants, variants, out_plan);
}

static rfi_status plan_create(const rfi_plan_desc *d, int32_t nvar, const rfi_variant *vars, rfi_plan_t *out_plan) {
    if (!d || !out_plan) return RFI_ERR_INVALID_ARG;
    *out_plan = nullptr;
    if (nvar > 0) {
        for (int v = 0; v < nvar; ++v) {
            if (!(vars[v].k > 0.0) || !std::isfinite(vars[v].k) || vars[v].k > 1.0e6) return RFI_ERR_INVALID_ARG;
            if (vars[v].mode < RFI_REPLACE_ZERO || vars[v].mode > RFI_REPLACE_NOISE) return RFI_ERR_INVALID_ARG;
            if (static_cast<int64_t>(std::floor(vars[v].k * 1.4826 * 65536.0 + 0.5)) < 1) return RFI_ERR_INVALID_ARG;
        }
        if ((d->flags & (RFI_PLAN_PER_STREAM | RFI_PLAN_POWER)) || d->mom_windows >= 2) return RFI_ERR_UNSUPPORTED;
    }
    if (d->sample_bits != 8 && d->sample_bits != 12) return RFI_ERR_INVALID_ARG;
    if (d->num_streams < 1 || !d->stream_len || !d->window_len) return RFI_ERR_INVALID_ARG;
    if (!(d->k > 0.0) || !std::isfinite(d->k) || d->k > 1.0e6) return RFI_ERR_INVALID_ARG;
    if (d->mode < RFI_REPLACE_ZERO || d->mode > RFI_REPLACE_NOISE) return RFI_ERR_INVALID_ARG;
    const uint32_t known = RFI_PLAN_PER_STREAM | RFI_PLAN_BATCHED | RFI_PLAN_GRAPH | RFI_PLAN_AUTOTUNE |
                           RFI_PLAN_INJECT_TIMEOUT | RFI_PLAN_POWER | RFI_PLAN_NO_SPLIT | RFI_PLAN_NOISE_PASS |
                           RFI_PLAN_WRITE_FLAGGED;
    if (d->flags & ~known) return RFI_ERR_INVALID_ARG;
    if ((d->flags & RFI_PLAN_PER_STREAM) && (d->flags & (RFI_PLAN_BATCHED | RFI_PLAN_GRAPH)))
        return RFI_ERR_INVALID_ARG;
    if (d->shape && !valid_shape(*d->shape)) return RFI_ERR_INVALID_ARG;
    if (d->mom_windows < 0 || d->mom_windows > (1 << 20)) return RFI_ERR_INVALID_ARG;
    if (d->mom_windows >= 2 && (d->flags & RFI_PLAN_PER_STREAM)) return RFI_ERR_UNSUPPORTED;
    if ((d->flags & RFI_PLAN_POWER) && ((d->flags & RFI_PLAN_PER_STREAM) || d->mom_windows >= 2))
        return RFI_ERR_UNSUPPORTED;
    if (d->out_format < RFI_OUT_SAME || d->out_format > RFI_OUT_BF16) return RFI_ERR_INVALID_ARG;
    if ((d->flags & RFI_PLAN_WRITE_FLAGGED) &&
        (d->sample_bits != 8 || (d->flags & (RFI_PLAN_PER_STREAM | RFI_PLAN_POWER)) || d->mom_windows >= 2 ||
         d->out_format != RFI_OUT_SAME || nvar > 0))
        return RFI_ERR_UNSUPPORTED;
    if (d->out_format != RFI_OUT_SAME &&
        ((d->flags & (RFI_PLAN_PER_STREAM | RFI_PLAN_POWER)) || d->mom_windows >= 2 || nvar > 0 ||
         (d->out_format == RFI_OUT_BF16 && d->sample_bits == 12)))
        return RFI_ERR_UNSUPPORTED;
    // Kq = round_half_up(k * 1.4826 * 2^16) (fixed-point multiple of Eq. 1)
    const int64_t kq = static_cast<int64_t>(std::floor(d->k * 1.4826 * 65536.0 + 0.5));
    if (kq < 1) return RFI_ERR_INVALID_ARG;
    uint64_t total_w = 0, total_s = 0;
    for (int i = 0; i < d->num_streams; ++i) {
        if (d->stream_len[i] < 1 || d->window_len[i] < 1 || d->window_len[i] > 65536) return RFI_ERR_INVALID_ARG;
        const int64_t nw = (d->stream_len[i] + d->window_len[i] - 1) / d->window_len[i];
        if (nw > 0x7FFFFFFF) return RFI_ERR_UNSUPPORTED;
        total_w += static_cast<uint64_t>(nw);
        total_s += static_cast<uint64_t>(d->stream_len[i]);
    }
    if (total_w > 0x7FFFFFFFull) return RFI_ERR_UNSUPPORTED;

    rfi_plan_s *P = new (std::nothrow) rfi_plan_s();
    if (!P) return RFI_ERR_OOM;
    P->bits = d->sample_bits;
    P->S = d->num_streams;
    P->mode = d->mode;
    P->flags = d->flags;
    P->k = d->k;
    P->kq = kq;
    const int32_t lo = P->bits == 8 ? -128 : -2048, hi = P->bits == 8 ? 127 : 2047;
    P->cval = std::min(hi, std::max(lo, d->const_value));
    P->seed = d->seed;
    P->kmom = d->mom_windows >= 2 ? d->mom_windows : 0;
    P->power = (d->flags & RFI_PLAN_POWER) != 0;
    P->out_format = d->out_format;
    P->ncopy = nvar;
    for (int v = 0; v < nvar; ++v) {
        Variant vr;
        vr.kq = static_cast<int64_t>(std::floor(vars[v].k * 1.4826 * 65536.0 + 0.5));
        vr.seed = vars[v].seed;
        vr.cval = std::min(hi, std::max(lo, vars[v].const_value));
        vr.mode = vars[v].mode;
        P->variants.push_back(vr);
    }
    P->len.assign(d->stream_len, d->stream_len + P->S);
    P->W.assign(d->window_len, d->window_len + P->S);
    P->sid.resize(P->S);
    for (int i = 0; i < P->S; ++i) P->sid[i] = d->stream_id ? d->stream_id[i] : static_cast<uint32_t>(i);
    P->nwin.resize(P->S);
    P->woff.resize(P->S);
    int64_t acc = 0;
    for (int i = 0; i < P->S; ++i) {
        P->nwin[i] = (P->len[i] + P->W[i] - 1) / P->W[i];
        P->woff[i] = acc;
        acc += P->nwin[i];
    }
    P->total_windows = total_w;
    P->total_samples = total_s;
    // RFI_PLAN_NOISE_PASS: digital noise as a second kernel, for batched plain noise plans over
    // segments of < 2^31 samples (others keep it in the excision kernel)
    bool short_segs = true;
    for (int i = 0; i < P->S; ++i) short_segs = short_segs && P->len[i] < (int64_t{1} << 31);
    P->write_flagged = (P->flags & RFI_PLAN_WRITE_FLAGGED) != 0;
    P->fill = (P->flags & RFI_PLAN_NOISE_PASS) && P->mode == RFI_REPLACE_NOISE && !(P->flags & RFI_PLAN_PER_STREAM) &&
              !P->power && P->ncopy == 0 && P->out_format == RFI_OUT_SAME && short_segs && !P->write_flagged;
    // small windows of 2^l samples: the multi-window form of the 8-bit kernel (several windows
    // per histogram, reduce and set of barriers)
    if (P->bits == 8 && P->ncopy == 0 && !P->power && P->out_format == RFI_OUT_SAME &&
        !(P->flags & RFI_PLAN_PER_STREAM) && !P->write_flagged) {
        for (int i = 0; i < P->S && !P->multi; ++i) {
            const int32_t W = P->W[i];
            P->multi = W >= 512 && W <= 8192 && (W & (W - 1)) == 0 && P->len[i] >= 2 * static_cast<int64_t>(W);
        }
    }

    rfi_status rs = RFI_OK;
    if (cudaGetDevice(&P->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return RFI_ERR_CUDA;
    }
    // windows of very different sizes: one internal plan per stage class
    if (!(P->flags & (RFI_PLAN_PER_STREAM | RFI_PLAN_NO_SPLIT)) && P->ncopy == 0) {
        const int bps = P->bits == 8 ? 1 : 2;
        std::vector<std::vector<int>> cls(3);
        for (int i = 0; i < P->S; ++i)
            cls[window_class(std::min<int64_t>(P->W[i], P->len[i]) * bps)].push_back(i);
        int nonempty = 0;
        for (auto &c : cls) nonempty += c.empty() ? 0 : 1;
        if (nonempty > 1) {
            for (auto &c : cls) {
                if (c.empty()) continue;
                std::vector<int64_t> len;
                std::vector<int32_t> W;
                std::vector<uint32_t> sid;
                for (int i : c) {
                    len.push_back(P->len[i]);
                    W.push_back(P->W[i]);
                    sid.push_back(P->sid[i]);
                }
                rfi_plan_desc cd = *d;
                cd.num_streams = static_cast<int32_t>(c.size());
                cd.stream_len = len.data();
                cd.window_len = W.data();
                cd.stream_id = sid.data();
                cd.flags = d->flags | RFI_PLAN_NO_SPLIT;
                rfi_plan_t child = nullptr;
                rs = rfi_plan_create(&cd, &child);
                if (rs != RFI_OK) {
                    rfi_plan_destroy(P);
                    return rs;
                }
                P->parts.push_back(child);
                P->part_streams.push_back(c);
            }
            P->part_st.assign(P->parts.size(), nullptr);
            P->part_ev.assign(P->parts.size(), nullptr);
            for (size_t k = 0; k < P->parts.size(); ++k) {
                if ((k > 0 && cudaStreamCreateWithFlags(&P->part_st[k], cudaStreamNonBlocking) != cudaSuccess) ||
                    cudaEventCreateWithFlags(&P->part_ev[k], cudaEventDisableTiming) != cudaSuccess) {
                    cudaGetLastError();
                    rfi_plan_destroy(P);
                    return RFI_ERR_CUDA;
                }
            }
            *out_plan = P;
            return RFI_OK;
        }
    }
    rs = plan_choose_shape(P, d->shape);
    if (rs == RFI_OK) rs = plan_build_tiles(P);
    if (rs == RFI_OK) rs = plan_alloc_workspace(P);
    if (rs == RFI_OK && (P->flags & RFI_PLAN_AUTOTUNE) && !(P->flags & RFI_PLAN_PER_STREAM) && P->kmom < 2 &&
        !P->power && P->ncopy == 0 && P->out_format == RFI_OUT_SAME)
        rs = plan_autotune(P, d->shape);
    if (rs == RFI_OK && (P->flags & RFI_PLAN_GRAPH)) rs = plan_build_graph(P);
    if (rs != RFI_OK) {
        rfi_plan_destroy(P);
        return rs;
    }
    *out_plan = P;
    return RFI_OK;
}

rfi_status rfi_excise(rfi_plan_t P, const void *const *in, void *const *out, uint32_t *const *mask,
                      uint32_t *const *counts, void *stream) {
    if (!P) return RFI_ERR_INVALID_ARG;
    if (!P->parts.empty()) {
        if (!in || !out) return RFI_ERR_INVALID_ARG;
        // part 0 on the caller's stream, the others on their own streams after a fork event;
        // the caller's stream then waits for every part
        cudaStream_t st0 = static_cast<cudaStream_t>(stream);
        if (cudaEventRecord(P->part_ev[0], st0) != cudaSuccess) return RFI_ERR_CUDA;
        for (size_t k = 0; k < P->parts.size(); ++k) {
            const auto a = part_args<const void *>(P, k, in);
            const auto b = part_args<void *>(P, k, out);
            const auto m = part_args<uint32_t *>(P, k, mask);
            const auto c = part_args<uint32_t *>(P, k, counts);
            cudaStream_t sk = k == 0 ? st0 : P->part_st[k];
            if (k > 0 && cudaStreamWaitEvent(sk, P->part_ev[0], 0) != cudaSuccess) return RFI_ERR_CUDA;
            const rfi_status rs = rfi_excise(P->parts[k], a.data(), b.data(), mask ? m.data() : nullptr,
                                             counts ? c.data() : nullptr, sk);
            if (k > 0 && (cudaEventRecord(P->part_ev[k], sk) != cudaSuccess ||
                          cudaStreamWaitEvent(st0, P->part_ev[k], 0) != cudaSuccess))
                return RFI_ERR_CUDA;
            if (rs != RFI_OK) return rs;
        }
        P->last_windows = P->total_windows;
        return RFI_OK;
    }
    if (P->ncopy > 0) return RFI_ERR_INVALID_ARG;  // digital-copy plans take rfi_excise_copies
    rfi_status rs = plan_check_buffers(P, in, out, mask, counts);
    if (rs != RFI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (P->fill && !P->d_fmask && !(P->flags & RFI_PLAN_PER_STREAM)) {
        // the fill pass reads the flags: streams called without a mask use the plan's own
        bool need = !mask;
        for (int i = 0; i < P->S && !need; ++i) need = !mask[i];
        if (need) {
            P->fmask_off.assign(P->S, 0);
            int64_t words = 0;
            for (int i = 0; i < P->S; ++i) {
                P->fmask_off[i] = words;
                words += P->nwin[i] * ((P->W[i] + 31) / 32);
            }
            if (cudaMalloc(&P->d_fmask, sizeof(uint32_t) * static_cast<size_t>(words)) != cudaSuccess) {
                cudaGetLastError();
                P->d_fmask = nullptr;
                return RFI_ERR_OOM;
            }
        }
    }
    std::vector<Seg> segs = plan_segs(P, in, out, mask, counts);
    P->last_windows = P->total_windows;
    if (P->flags & RFI_PLAN_PER_STREAM) {
        RFI_CUDA(cudaMemsetAsync(P->d_ctr, 0, sizeof(DevCounters), st));
        const Params p = plan_params(P);
        for (int i = 0; i < P->S; ++i)
            RFI_CUDA(launch_stream(P->bits, P->mode, P->shape.consumer_warps, segs[i], 0, P->nwin[i], p, st));
        return RFI_OK;
    }
    return plan_run_batched(P, segs, st);
}

rfi_status rfi_excise_copies(rfi_plan_t P, const void *const *in, void *const *out, uint32_t *const *mask,
                             uint32_t *const *counts, void *stream) {
    if (!P || P->ncopy < 1 || !in || !out) return RFI_ERR_INVALID_ARG;
    std::vector<Seg> segs;
    for (int v = 0; v < P->ncopy; ++v) {
        void *const *o = out + static_cast<size_t>(v) * P->S;
        uint32_t *const *m = mask ? mask + static_cast<size_t>(v) * P->S : nullptr;
        uint32_t *const *c = counts ? counts + static_cast<size_t>(v) * P->S : nullptr;
        rfi_status rs = plan_check_buffers(P, in, o, m, c);
        if (rs != RFI_OK) return rs;
        const std::vector<Seg> sv = plan_segs(P, in, o, m, c);
        segs.insert(segs.end(), sv.begin(), sv.begin() + P->S);
    }
    P->last_windows = P->total_windows;
    return plan_run_batched(P, segs, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace rfi {

// Refresh the device segment table if the buffers changed, then run the batched pass.
rfi_status plan_run_batched(rfi_plan_s *P, const std::vector<Seg> &segs, cudaStream_t st) {
    const int nsegs = plan_nsegs(P);
    if (!P->segs_valid || std::memcmp(segs.data(), P->segs_host.data(), sizeof(Seg) * nsegs) != 0) {
        for (int i = 0; i < nsegs; i += kSegBatch)
            RFI_CUDA(launch_write_segs(P->d_segs + i, segs.data() + i, std::min(kSegBatch, nsegs - i), st));
        P->segs_host = segs;
        P->segs_valid = true;
        P->last_seg_writes = (nsegs + kSegBatch - 1) / kSegBatch;
    } else {
        P->last_seg_writes = 0;
    }
    if (P->gexec) {
        RFI_CUDA(cudaGraphLaunch(P->gexec, st));
        return RFI_OK;
    }
    return plan_enqueue_batched(P, st);
}

}  // namespace rfi

extern "C" {

rfi_status rfi_stats(rfi_plan_t P, int32_t *const *median, int32_t *const *mad, rfi_totals *totals, void *stream) {
    if (!P) return RFI_ERR_INVALID_ARG;
    if (!P->parts.empty()) {
        rfi_totals sum{0, 0, RFI_OK};
        rfi_status dev = RFI_OK;
        for (size_t k = 0; k < P->parts.size(); ++k) {
            const auto a = part_args<int32_t *>(P, k, median);
            const auto b = part_args<int32_t *>(P, k, mad);
            rfi_totals t{};
            const rfi_status rs = rfi_stats(P->parts[k], median ? a.data() : nullptr, mad ? b.data() : nullptr, &t,
                                            stream);
            if (rs == RFI_ERR_INVALID_ARG || rs == RFI_ERR_CUDA) return rs;
            if (dev == RFI_OK && rs != RFI_OK) dev = rs;
            sum.windows += t.windows;
            sum.flagged += t.flagged;
        }
        sum.device_status = dev;
        if (totals) *totals = sum;
        return dev;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < P->S; ++i) {
        const size_t b = sizeof(int32_t) * P->nwin[i];
        if (median && median[i])
            RFI_CUDA(cudaMemcpyAsync(median[i], P->d_med + P->woff[i], b, cudaMemcpyDeviceToDevice, st));
        if (mad && mad[i])
            RFI_CUDA(cudaMemcpyAsync(mad[i], P->d_mad + P->woff[i], b, cudaMemcpyDeviceToDevice, st));
    }
    DevCounters h;
    RFI_CUDA(cudaMemcpyAsync(&h, P->d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    RFI_CUDA(cudaStreamSynchronize(st));
    const rfi_status dev = (h.status & kStatusTimeout)       ? RFI_ERR_TIMEOUT
                           : (h.status & kStatusLayout)      ? RFI_ERR_UNSUPPORTED
                           : (h.status & kStatusSampleRange) ? RFI_ERR_SAMPLE_RANGE
                                                             : RFI_OK;
    if (totals) {
        totals->windows = P->last_windows;
        totals->flagged = h.flagged;
        totals->device_status = static_cast<int32_t>(dev);
    }
    return dev;
}

rfi_status rfi_stats_mom(rfi_plan_t P, int32_t *const *mom, void *stream) {
    if (!P) return RFI_ERR_INVALID_ARG;
    if (!P->parts.empty()) {
        for (size_t k = 0; k < P->parts.size(); ++k) {
            const auto a = part_args<int32_t *>(P, k, mom);
            const rfi_status rs = rfi_stats_mom(P->parts[k], mom ? a.data() : nullptr, stream);
            if (rs != RFI_OK) return rs;
        }
        return RFI_OK;
    }
    if (P->kmom < 2) return RFI_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < P->S; ++i)
        if (mom && mom[i])
            RFI_CUDA(cudaMemcpyAsync(mom[i], P->d_mom + P->woff[i], sizeof(int32_t) * P->nwin[i],
                                     cudaMemcpyDeviceToDevice, st));
    return RFI_OK;
}

rfi_status rfi_stats_power(rfi_plan_t P, uint64_t *const *power, void *stream) {
    if (!P) return RFI_ERR_INVALID_ARG;
    if (!P->parts.empty()) {
        for (size_t k = 0; k < P->parts.size(); ++k) {
            const auto a = part_args<uint64_t *>(P, k, power);
            const rfi_status rs = rfi_stats_power(P->parts[k], power ? a.data() : nullptr, stream);
            if (rs != RFI_OK) return rs;
        }
        return RFI_OK;
    }
    if (!P->power) return RFI_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < P->S; ++i)
        if (power && power[i])
            RFI_CUDA(cudaMemcpyAsync(power[i], P->d_pow + 2 * P->woff[i], 2 * sizeof(uint64_t) * P->nwin[i],
                                     cudaMemcpyDeviceToDevice, st));
    return RFI_OK;
}

rfi_status rfi_improvement_db(const uint64_t *power, int64_t nwin, int32_t windows_per_point,
                              int32_t points_per_block, double *db, double *s_unfiltered, double *s_filtered) {
    if (!power || nwin < 1 || windows_per_point < 1 || points_per_block < 2 || !db) return RFI_ERR_INVALID_ARG;
    const int64_t npt = nwin / windows_per_point;
    const int64_t nb = npt / points_per_block;
    double s[2] = {0.0, 0.0};
    for (int side = 0; side < 2; ++side) {
        double acc = 0.0;
        int64_t used = 0;
        std::vector<double> pt(points_per_block);
        for (int64_t b = 0; b < nb; ++b) {
            double mean = 0.0;
            for (int32_t q = 0; q < points_per_block; ++q) {
                double v = 0.0;
                const int64_t w0 = (b * points_per_block + q) * windows_per_point;
                for (int32_t k = 0; k < windows_per_point; ++k) v += static_cast<double>(power[2 * (w0 + k) + side]);
                pt[q] = v;
                mean += v;
            }
            mean /= points_per_block;
            double var = 0.0;
            for (double v : pt) var += (v - mean) * (v - mean);
            const double rms = std::sqrt(var / points_per_block);
            if (rms > 0.0) {
                acc += mean / rms;
                ++used;
            }
        }
        if (used == 0) return RFI_ERR_INVALID_ARG;
        s[side] = acc / static_cast<double>(used);
    }
    *db = 10.0 * std::log10(s[1] / s[0]);
    if (s_unfiltered) *s_unfiltered = s[0];
    if (s_filtered) *s_filtered = s[1];
    return RFI_OK;
}

rfi_status rfi_plan_get_info(rfi_plan_t P, rfi_plan_info *info) {
    if (!P || !info) return RFI_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    if (!P->parts.empty()) {
        uint64_t most = 0;
        for (rfi_plan_s *c : P->parts) {
            rfi_plan_info ci{};
            rfi_plan_get_info(c, &ci);
            info->workspace_bytes += ci.workspace_bytes;
            info->tiles += ci.tiles;
            info->grid = std::max(info->grid, ci.grid);
            info->kernels_per_call += ci.kernels_per_call;
            if (ci.total_samples > most) {
                most = ci.total_samples;
                info->shape = ci.shape;
            }
        }
        info->k_q16 = P->kq;
        info->total_windows = P->total_windows;
        info->total_samples = P->total_samples;
        info->sm_count = P->sm_count;
        return RFI_OK;
    }
    info->k_q16 = P->kq;
    info->total_windows = P->total_windows;
    info->total_samples = P->total_samples;
    info->workspace_bytes = P->ws_bytes + P->host_pipe_bytes;
    info->tiles = P->ntiles;
    info->grid = P->grid;
    info->shape.consumer_warps = P->shape.consumer_warps;
    info->shape.stages = P->shape.stages;
    info->shape.ctas_per_sm = P->shape.ctas_per_sm;
    info->shape.stage_bytes = P->shape.stage_bytes;
    info->shape.dynamic_tiles = P->shape.dynamic_tiles;
    info->shape.hist_copies = P->shape.hist_copies;
    info->shape.groups = P->shape.groups;
    info->shape.warp_split = P->shape.warp_split;
    info->sm_count = P->sm_count;
    info->kernels_per_call = (P->flags & RFI_PLAN_PER_STREAM) ? P->S : (P->kmom >= 2 ? 3 : 1) + (P->fill ? 1 : 0);
    return RFI_OK;
}

rfi_status rfi_plan_destroy(rfi_plan_t P) {
    if (!P) return RFI_OK;
    for (rfi_plan_s *c : P->parts) rfi_plan_destroy(c);
    for (cudaStream_t s : P->part_st)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : P->part_ev)
        if (e) cudaEventDestroy(e);
    plan_release_host_pipe(P);
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->ws) cudaFree(P->ws);
    if (P->d_fmask) cudaFree(P->d_fmask);
    cudaGetLastError();
    delete P;
    return RFI_OK;
}

}  // extern "C"
