// 12-bit instantiations of the excision kernels (split per width to compile in parallel).
#include "kernels_impl.cuh"

namespace rfi {

cudaError_t launch_persistent_b12(int mode, const Shape &s, int grid, const Seg *segs, const Tile *tiles,
                                  int ntiles, const Params &p, unsigned *counter, int inject, cudaStream_t st) {
    RFI_DISPATCH_PERSISTENT(12, dev::persistent_launch_t, mode, s.consumer_warps, s.groups, s, grid, segs, tiles,
                            ntiles, p, counter, inject, st);
    return cudaErrorInvalidValue;
}

int persistent_occupancy_b12(int mode, const Shape &s) {
    RFI_DISPATCH_PERSISTENT(12, dev::persistent_occ_t, mode, s.consumer_warps, s.groups, s);
    return 0;
}

cudaError_t launch_stream_b12(int mode, int consumer_warps, const Seg &seg, int64_t w_begin, int64_t nw,
                              const Params &p, cudaStream_t st) {
    RFI_DISPATCH_MODE_CW(12, dev::stream_launch_t, mode, consumer_warps, seg, w_begin, nw, p, st);
    return cudaErrorInvalidValue;
}

}  // namespace rfi
