// 8-bit instantiations of the in-place form that writes back only what changes
// (RFI_PLAN_WRITE_FLAGGED), one consumer group of 4, 8 or 16 warps.
#include "kernels_impl.cuh"

namespace rfi {

#define RFI_CASES_FO(FN, M, ...)                                                                      \
    RFI_CASE_MCG(8, FN, M, 4, 1, __VA_ARGS__) RFI_CASE_MCG(8, FN, M, 8, 1, __VA_ARGS__)            \
    RFI_CASE_MCG(8, FN, M, 16, 1, __VA_ARGS__)
#define RFI_DISPATCH_FO(FN, MODE, CW, G, ...)                                                         \
    do {                                                                                              \
        switch (MODE * 1000 + CW * 10 + G) {                                                          \
            RFI_CASES_FO(FN, 512, __VA_ARGS__)                                                        \
            RFI_CASES_FO(FN, 513, __VA_ARGS__)                                                        \
            RFI_CASES_FO(FN, 514, __VA_ARGS__)                                                        \
            RFI_CASES_FO(FN, 515, __VA_ARGS__)                                                        \
            default: break;                                                                           \
        }                                                                                             \
    } while (0)

static_assert(kModeFlaggedOnly == 512, "mode numbers of the cases below");

cudaError_t launch_persistent_fo_b8(int mode, const Shape &s, int grid, const Seg *segs, const Tile *tiles,
                                    int ntiles, const Params &p, unsigned *counter, int inject, cudaStream_t st) {
    RFI_DISPATCH_FO(dev::persistent_launch_t, mode, s.consumer_warps, s.groups, s, grid, segs, tiles, ntiles, p,
                    counter, inject, st);
    return cudaErrorInvalidValue;
}

int persistent_occupancy_fo_b8(int mode, const Shape &s) {
    RFI_DISPATCH_FO(dev::persistent_occ_t, mode, s.consumer_warps, s.groups, s);
    return 0;
}

}  // namespace rfi
