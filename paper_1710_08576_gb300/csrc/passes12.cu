// 12-bit instantiations of the Median-of-MAD passes (Eq. 3), the power-metered and digital-copy
// passes and the fused output formats.
#include "passes_impl.cuh"

namespace rfi {

cudaError_t launch_persistent_mom_b12(int mode, const Shape &s, int grid, const Seg *segs, const Tile *tiles,
                                      int ntiles, const Params &p, unsigned *counter, int inject,
                                      cudaStream_t st) {
    RFI_DISPATCH_MOM(12, dev::persistent_launch_t, mode, s.consumer_warps, s.groups, s, grid, segs, tiles, ntiles,
                     p, counter, inject, st);
    RFI_DISPATCH_FMT12(dev::persistent_launch_t, mode, s.consumer_warps, s.groups, s, grid, segs, tiles, ntiles, p,
                      counter, inject, st);
    return cudaErrorInvalidValue;
}

int persistent_occupancy_mom_b12(int mode, const Shape &s) {
    RFI_DISPATCH_MOM(12, dev::persistent_occ_t, mode, s.consumer_warps, s.groups, s);
    RFI_DISPATCH_FMT12(dev::persistent_occ_t, mode, s.consumer_warps, s.groups, s);
    return 0;
}

cudaError_t launch_mom_b12(const MomChunk *chunks, int nchunks, const int32_t *D, int32_t *Mm, int kmom,
                           cudaStream_t st) {
    return dev::mom_launch_t<4096>(chunks, nchunks, D, Mm, kmom, st);
}

}  // namespace rfi
