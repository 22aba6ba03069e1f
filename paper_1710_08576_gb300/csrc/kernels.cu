// Width dispatch, shared-memory sizing and the segment-table writer.
#include "kernels_impl.cuh"

namespace rfi {

cudaError_t launch_persistent_b8(int, const Shape &, int, const Seg *, const Tile *, int, const Params &,
                                 unsigned *, int, cudaStream_t);
cudaError_t launch_persistent_b12(int, const Shape &, int, const Seg *, const Tile *, int, const Params &,
                                  unsigned *, int, cudaStream_t);
int persistent_occupancy_b8(int, const Shape &);
int persistent_occupancy_b12(int, const Shape &);
cudaError_t launch_persistent_mom_b8(int, const Shape &, int, const Seg *, const Tile *, int, const Params &,
                                     unsigned *, int, cudaStream_t);
cudaError_t launch_persistent_mom_b12(int, const Shape &, int, const Seg *, const Tile *, int, const Params &,
                                      unsigned *, int, cudaStream_t);
int persistent_occupancy_mom_b8(int, const Shape &);
cudaError_t launch_persistent_multi_b8(int, const Shape &, int, const Seg *, const Tile *, int, const Params &,
                                       unsigned *, int, cudaStream_t);
int persistent_occupancy_multi_b8(int, const Shape &);
cudaError_t launch_persistent_fo_b8(int, const Shape &, int, const Seg *, const Tile *, int, const Params &,
                                    unsigned *, int, cudaStream_t);
int persistent_occupancy_fo_b8(int, const Shape &);
cudaError_t launch_persistent_split_b8(int, const Shape &, int, const Seg *, const Tile *, int, const Params &,
                                       unsigned *, int, cudaStream_t);
int persistent_occupancy_split_b8(int, const Shape &);
int persistent_occupancy_mom_b12(int, const Shape &);
cudaError_t launch_mom_b8(const MomChunk *, int, const int32_t *, int32_t *, int, cudaStream_t);
cudaError_t launch_mom_b12(const MomChunk *, int, const int32_t *, int32_t *, int, cudaStream_t);
cudaError_t launch_stream_b8(int, int, const Seg &, int64_t, int64_t, const Params &, cudaStream_t);
cudaError_t launch_stream_b12(int, int, const Seg &, int64_t, int64_t, const Params &, cudaStream_t);

size_t persistent_smem_bytes(int bits, int mode, const Shape &s) {
    mode = shape_mode(bits, mode, s);
    return bits == 8
               ? dev::layout<8>(s.hist_copies, s.stages, s.stage_bytes, s.consumer_warps, s.groups, mode).total
               : dev::layout<12>(s.hist_copies, s.stages, s.stage_bytes, s.consumer_warps, s.groups, mode).total;
}

size_t stream_smem_bytes(int bits, int mode, int consumer_warps, int ncopies, int window_bytes) {
    const int wb = dev::align_up(window_bytes, 128);
    return bits == 8 ? dev::layout<8>(ncopies, 1, wb, consumer_warps, 1, mode).total
                     : dev::layout<12>(ncopies, 1, wb, consumer_warps, 1, mode).total;
}

int persistent_occupancy(int bits, int mode, const Shape &s) {
    mode = shape_mode(bits, mode, s);
    if (mode & kModeWarpSplit) return persistent_occupancy_split_b8(mode, s);
    if (mode & kModeMulti) return bits == 8 ? persistent_occupancy_multi_b8(mode, s) : 0;
    if (mode & kModeFlaggedOnly) return bits == 8 ? persistent_occupancy_fo_b8(mode, s) : 0;
    if (mode >= kModeStats)
        return bits == 8 ? persistent_occupancy_mom_b8(mode, s) : persistent_occupancy_mom_b12(mode, s);
    return bits == 8 ? persistent_occupancy_b8(mode, s) : persistent_occupancy_b12(mode, s);
}

cudaError_t launch_persistent(int bits, int mode, const Shape &s, int grid, const Seg *segs, const Tile *tiles,
                              int ntiles, const Params &p, unsigned *counter, int inject, cudaStream_t st) {
    mode = shape_mode(bits, mode, s);
    if (mode & kModeWarpSplit)
        return launch_persistent_split_b8(mode, s, grid, segs, tiles, ntiles, p, counter, inject, st);
    if (mode & kModeMulti)
        return bits == 8 ? launch_persistent_multi_b8(mode, s, grid, segs, tiles, ntiles, p, counter, inject, st)
                         : cudaErrorInvalidValue;
    if (mode & kModeFlaggedOnly)
        return bits == 8 ? launch_persistent_fo_b8(mode, s, grid, segs, tiles, ntiles, p, counter, inject, st)
                         : cudaErrorInvalidValue;
    if (mode >= kModeStats)
        return bits == 8 ? launch_persistent_mom_b8(mode, s, grid, segs, tiles, ntiles, p, counter, inject, st)
                         : launch_persistent_mom_b12(mode, s, grid, segs, tiles, ntiles, p, counter, inject, st);
    return bits == 8 ? launch_persistent_b8(mode, s, grid, segs, tiles, ntiles, p, counter, inject, st)
                     : launch_persistent_b12(mode, s, grid, segs, tiles, ntiles, p, counter, inject, st);
}

cudaError_t launch_mom(int bits, const MomChunk *chunks, int nchunks, const int32_t *D, int32_t *Mm, int kmom,
                       cudaStream_t st) {
    return bits == 8 ? launch_mom_b8(chunks, nchunks, D, Mm, kmom, st)
                     : launch_mom_b12(chunks, nchunks, D, Mm, kmom, st);
}

cudaError_t launch_stream(int bits, int mode, int consumer_warps, const Seg &seg, int64_t w_begin, int64_t nw,
                          const Params &p, cudaStream_t st) {
    return bits == 8 ? launch_stream_b8(mode, consumer_warps, seg, w_begin, nw, p, st)
                     : launch_stream_b12(mode, consumer_warps, seg, w_begin, nw, p, st);
}

struct SegBatch {
    Seg s[kSegBatch];
};

__global__ void write_segs_kernel(Seg *dst, SegBatch b, int n) {
    const int i = threadIdx.x;
    if (i < n) dst[i] = b.s[i];
}

cudaError_t launch_write_segs(Seg *dst, const Seg *src_host, int n, cudaStream_t st) {
    if (n <= 0 || n > kSegBatch) return cudaErrorInvalidValue;
    SegBatch b;
    for (int i = 0; i < n; ++i) b.s[i] = src_host[i];
    write_segs_kernel<<<1, kSegBatch, 0, st>>>(dst, b, n);
    return cudaGetLastError();
}

}  // namespace rfi
