// Host-side plan state shared by plan.cpp, host_pipe.cpp and autotune.cpp.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "rfi.h"
#include "internal.h"

namespace rfi {

// Buffers of the chunked host pipeline (rfi_excise_host), allocated on first use.
struct HostPipe {
    static constexpr int kSlots = 3;
    int64_t chunk_bytes = 0;     // input bytes per slot
    uint8_t *in[kSlots] = {};
    uint8_t *out[kSlots] = {};
    uint32_t *mask[kSlots] = {};
    uint32_t *counts[kSlots] = {};
    cudaEvent_t h2d[kSlots] = {}, comp[kSlots] = {}, d2h[kSlots] = {};
    cudaStream_t s_comp = nullptr, s_d2h = nullptr;
    bool ready = false;
};

}  // namespace rfi

struct rfi_plan_s {
    int bits = 8, S = 0, mode = 0;
    uint32_t flags = 0;
    double k = 0;
    int64_t kq = 0;
    int32_t cval = 0;
    uint64_t seed = 0;
    std::vector<int64_t> len;
    std::vector<int32_t> W;
    std::vector<uint32_t> sid;
    std::vector<int64_t> nwin, woff;
    uint64_t total_windows = 0, total_samples = 0, last_windows = 0;
    int device = 0, sm_count = 0;
    rfi::Shape shape{};
    std::vector<rfi::Tile> tiles_host;
    int ntiles = 0, grid = 0;
    int grid_apply = 0;  // Median of MAD: grid of the apply pass (no histogram: more CTAs fit)
    // device workspace
    void *ws = nullptr;
    size_t ws_bytes = 0;
    rfi::DevCounters *d_ctr = nullptr;
    rfi::Seg *d_segs = nullptr;
    rfi::Tile *d_tiles = nullptr;
    int32_t *d_med = nullptr, *d_mad = nullptr;
    // Median of MAD (Eq. 3): kmom >= 2; segment table holds 2S entries (stats pass, apply pass)
    int kmom = 0;
    int32_t *d_mom = nullptr;
    // RFI_PLAN_POWER: {sum x^2, sum z^2} per window
    bool power = false;
    // some stream has windows of 2^l samples, 512 <= 2^l <= 8192: the multi-window form
    bool multi = false;
    // RFI_PLAN_WRITE_FLAGGED: in place, only changed chunks are stored
    bool write_flagged = false;
    uint64_t *d_pow = nullptr;
    int out_format = RFI_OUT_SAME;  // fused output format
    // digital noise as a second pass (noise_fill): the excision pass replaces with 0, then the
    // fill kernel writes the noise of every flagged sample; d_fwin: S + 1 unit offsets
    bool fill = false;
    uint32_t *d_fwin = nullptr;
    uint32_t nfwin = 0;
    bool fill_packed = false;  // some segment's fill units are packed (fill_packs)
    int fill_grid = 0;
    uint32_t *d_fmask = nullptr;  // flag masks of streams called without one (allocated on demand)
    std::vector<int64_t> fmask_off;
    // digital copy: the variants (segment table holds ncopy * S entries)
    int ncopy = 0;
    std::vector<rfi::Variant> variants;
    rfi::Variant *d_var = nullptr;
    rfi::MomChunk *d_mchunks = nullptr;
    std::vector<rfi::MomChunk> mchunks;
    std::vector<rfi::Seg> segs_host;
    bool segs_valid = false;
    int last_seg_writes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    rfi::HostPipe pipe;
    size_t host_pipe_bytes = 0;
    // a plan split by window-size class: one internal plan per class and its stream indices
    std::vector<rfi_plan_s *> parts;
    // parts after the first run on their own streams, forked from and joined back into the
    // caller's stream with events, so that one part's tail overlaps the next part's kernels
    std::vector<cudaStream_t> part_st;
    std::vector<cudaEvent_t> part_ev;  // [0]: the fork; [k]: part k's end
    std::vector<std::vector<int>> part_streams;
};

namespace rfi {

rfi_status plan_choose_shape(rfi_plan_s *P, const rfi_launch_shape *req);
// Whether the split-warp form (kModeWarpSplit) can run this plan with shape s.
bool plan_warp_split_runs(const rfi_plan_s *P, const Shape &s);
rfi_status plan_build_tiles(rfi_plan_s *P);
rfi_status plan_alloc_workspace(rfi_plan_s *P);
rfi_status plan_enqueue_batched(rfi_plan_s *P, cudaStream_t st);
rfi_status plan_build_graph(rfi_plan_s *P);
rfi_status plan_autotune(rfi_plan_s *P, const rfi_launch_shape *req);
void plan_release_host_pipe(rfi_plan_s *P);
Params plan_params(const rfi_plan_s *P);
std::vector<Seg> plan_segs(const rfi_plan_s *P, const void *const *in, void *const *out, uint32_t *const *mask,
                           uint32_t *const *counts);
rfi_status plan_check_buffers(const rfi_plan_s *P, const void *const *in, void *const *out,
                              uint32_t *const *mask, uint32_t *const *counts);
rfi_status plan_run_batched(rfi_plan_s *P, const std::vector<Seg> &segs, cudaStream_t st);
inline int plan_nsegs(const rfi_plan_s *P) {
    return P->kmom >= 2 ? 2 * P->S : (P->ncopy > 0 ? P->ncopy * P->S : P->S);
}
// Stage class of a window of wb bytes: 0 up to 16 KiB, 1 up to 32 KiB, 2 larger.
inline int window_class(int64_t wb) { return wb <= 16384 ? 0 : (wb <= 32768 ? 1 : 2); }
// Per-part pointer arrays of a split plan (entries in the part's stream order).
template <class T>
std::vector<T> part_args(const rfi_plan_s *P, size_t k, T const *all) {
    std::vector<T> v;
    for (int i : P->part_streams[k]) v.push_back(all ? all[i] : T());
    return v;
}
// Kernel mode of a per-window MAD plan (the power-metered form when RFI_PLAN_POWER is set).
inline int plan_kernel_mode(const rfi_plan_s *P) {
    const int fmt = P->out_format == RFI_OUT_F16 ? kModeF16 : (P->out_format == RFI_OUT_BF16 ? kModeBF16 : 0);
    if (P->ncopy > 0) return kModeCopies;
    const int m = (P->fill && P->kmom < 2 ? 0 : P->mode) | (P->power ? kModePower : 0) | fmt;
    if (P->write_flagged) return m | kModeFlaggedOnly;
    return m | (P->multi && m < 4 ? kModeMulti : 0);
}
// Kernel mode of the estimation pass of a Median-of-MAD plan.
inline int plan_stats_mode(const rfi_plan_s *P) { return kModeStats | (P->multi ? kModeMulti : 0); }

}  // namespace rfi
