// 8-bit instantiations of the split-warp form of the persistent kernel (zero, constant and
// threshold replacement, also write-flagged; one consumer group of 8 warps: 4 histogram warps,
// 4 replace warps).
#include "kernels_impl.cuh"

namespace rfi {

static_assert(kModeWarpSplit == 1024 && kModeFlaggedOnly == 512, "mode numbers of the cases below");

#define RFI_DISPATCH_SPLIT(FN, MODE, CW, G, ...)                                                      \
    do {                                                                                              \
        switch (MODE * 1000 + CW * 10 + G) {                                                          \
            RFI_CASE_MCG(8, FN, 1024, 8, 1, __VA_ARGS__)                                              \
            RFI_CASE_MCG(8, FN, 1025, 8, 1, __VA_ARGS__)                                              \
            RFI_CASE_MCG(8, FN, 1026, 8, 1, __VA_ARGS__)                                              \
            RFI_CASE_MCG(8, FN, 1536, 8, 1, __VA_ARGS__)                                              \
            RFI_CASE_MCG(8, FN, 1537, 8, 1, __VA_ARGS__)                                              \
            RFI_CASE_MCG(8, FN, 1538, 8, 1, __VA_ARGS__)                                              \
            default: break;                                                                           \
        }                                                                                             \
    } while (0)

cudaError_t launch_persistent_split_b8(int mode, const Shape &s, int grid, const Seg *segs, const Tile *tiles,
                                       int ntiles, const Params &p, unsigned *counter, int inject, cudaStream_t st) {
    RFI_DISPATCH_SPLIT(dev::persistent_launch_t, mode, s.consumer_warps, s.groups, s, grid, segs, tiles, ntiles, p,
                       counter, inject, st);
    return cudaErrorInvalidValue;
}

int persistent_occupancy_split_b8(int mode, const Shape &s) {
    RFI_DISPATCH_SPLIT(dev::persistent_occ_t, mode, s.consumer_warps, s.groups, s);
    return 0;
}

}  // namespace rfi
