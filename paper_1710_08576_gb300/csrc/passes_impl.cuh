// The passes beyond plain excision: for the Median of MAD (Eq. 3), the sliding lower median of
// the last k_mom per-window MADs of each stream and the estimation-only / apply instantiations
// of the persistent kernel around it; the power-metered excision (per-window sums of x^2 and
// z^2 for the improvement metric of Section III-A); and the digital-copy pass (several (k,
// replacement) variants from one histogram per window). Instantiated per sample width in
// passes8.cu / passes12.cu.
#pragma once

#include "kernels_impl.cuh"

namespace rfi {
namespace dev {

// One warp per chunk of kMomChunk consecutive windows of one stream. The warp builds a
// histogram of the MADs of the k_mom windows before the chunk, then slides: per window it
// adds the window's MAD, drops the one k_mom windows back, and finds the lower median of the
// (at most k_mom) MADs in the histogram with a two-level search (32-bin groups, then bins).
// MAD values are histogram bins: [0, 255] for int8 samples, [0, 4095] for 12-bit.
template <int NB>
__global__ void __launch_bounds__(32) mom_kernel(const MomChunk *__restrict__ chunks, const int32_t *__restrict__ D,
                                                 int32_t *__restrict__ Mm, int kmom) {
    constexpr int NC = NB / 32;                  // groups of 32 bins
    constexpr int CPL = NC >= 32 ? NC / 32 : 1;  // groups per lane
    __shared__ uint32_t h[NB];
    __shared__ uint32_t hc[NC];
    __shared__ int32_t add[kMomChunk], drop[kMomChunk], res[kMomChunk];
    const int lane = threadIdx.x;
    const MomChunk c = chunks[blockIdx.x];
    const int32_t *d = D + c.base;
    auto bin = [](int32_t v) { return v < 0 ? 0 : (v > NB - 1 ? NB - 1 : v); };
    for (int i = lane; i < NB; i += 32) h[i] = 0u;
    for (int i = lane; i < NC; i += 32) hc[i] = 0u;
    __syncwarp();
    const int n = c.b - c.a;
    // the histogram enters the chunk holding window a - 1's MADs: windows [a - kmom, a)
    const int lo = c.a - kmom > 0 ? c.a - kmom : 0;
    for (int i = lo + lane; i < c.a; i += 32) {
        const int v = bin(d[i]);
        atomicAdd(&h[v], 1u);
        atomicAdd(&hc[v >> 5], 1u);
    }
    for (int i = lane; i < n; i += 32) {
        add[i] = bin(d[c.a + i]);
        const int j = c.a + i - kmom;
        drop[i] = j >= 0 ? bin(d[j]) : -1;
    }
    __syncwarp();
    for (int i = 0; i < n; ++i) {
        const int j = c.a + i;
        if (lane == 0) {
            const int v = add[i], u = drop[i];
            h[v] += 1u;
            hc[v >> 5] += 1u;
            if (u >= 0) {
                h[u] -= 1u;
                hc[u >> 5] -= 1u;
            }
        }
        __syncwarp();
        const uint32_t cnt = static_cast<uint32_t>(j + 1 < kmom ? j + 1 : kmom);
        const uint32_t need = (cnt + 1) >> 1;  // lower median: the ceil(cnt/2)-th smallest
        // groups: lane l holds groups [l*CPL, (l+1)*CPL)
        uint32_t s = 0u;
        if (lane * CPL < NC) {
#pragma unroll
            for (int q = 0; q < CPL; ++q) s += hc[lane * CPL + q];
        }
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        const int fl = __ffs(__ballot_sync(0xFFFFFFFFu, incl >= need)) - 1;
        uint32_t base = __shfl_sync(0xFFFFFFFFu, incl - s, fl);
        int g = fl * CPL;
#pragma unroll
        for (int q = 0; q < CPL - 1; ++q) {
            const uint32_t x = hc[g];
            if (base + x >= need) break;
            base += x;
            ++g;
        }
        const uint32_t f = h[32 * g + lane];
        uint32_t fi = f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, fi, o);
            if (lane >= o) fi += t;
        }
        const int b = __ffs(__ballot_sync(0xFFFFFFFFu, base + fi >= need)) - 1;
        if (lane == 0) res[i] = 32 * g + b;
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) Mm[c.base + c.a + i] = res[i];
}

template <int NB>
cudaError_t mom_launch_t(const MomChunk *chunks, int nchunks, const int32_t *D, int32_t *Mm, int kmom,
                         cudaStream_t st) {
    if (nchunks <= 0) return cudaSuccess;
    mom_kernel<NB><<<nchunks, 32, 0, st>>>(chunks, D, Mm, kmom);
    return cudaGetLastError();
}

// These passes run with one consumer group of 4 or 8 warps.
#define RFI_CASES_MOM_CW(BITS, FN, M, ...) \
    RFI_CASE_MCG(BITS, FN, M, 4, 1, __VA_ARGS__) RFI_CASE_MCG(BITS, FN, M, 8, 1, __VA_ARGS__)
#define RFI_DISPATCH_MOM(BITS, FN, MODE, CW, G, ...)                    \
    do {                                                                \
        switch (MODE * 1000 + CW * 10 + G) {                            \
            RFI_CASES_MOM_CW(BITS, FN, 4, __VA_ARGS__)                  \
            RFI_CASES_MOM_CW(BITS, FN, 8, __VA_ARGS__)                  \
            RFI_CASES_MOM_CW(BITS, FN, 9, __VA_ARGS__)                  \
            RFI_CASES_MOM_CW(BITS, FN, 10, __VA_ARGS__)                 \
            RFI_CASES_MOM_CW(BITS, FN, 11, __VA_ARGS__)                 \
            RFI_CASES_MOM_CW(BITS, FN, 16, __VA_ARGS__)                 \
            RFI_CASES_MOM_CW(BITS, FN, 17, __VA_ARGS__)                 \
            RFI_CASES_MOM_CW(BITS, FN, 18, __VA_ARGS__)                 \
            RFI_CASES_MOM_CW(BITS, FN, 19, __VA_ARGS__)                 \
            RFI_CASES_MOM_CW(BITS, FN, 32, __VA_ARGS__)                 \
            default: break;                                             \
        }                                                               \
    } while (0)

// The fused output formats run with one group of 8 consumer warps: fp16 for both widths,
// bf16 for int8 only.
#define RFI_CASES_FMT(BITS, FN, F, ...)                                                         \
    RFI_CASE_MCG(BITS, FN, (F + 0), 8, 1, __VA_ARGS__) RFI_CASE_MCG(BITS, FN, (F + 1), 8, 1, __VA_ARGS__) \
    RFI_CASE_MCG(BITS, FN, (F + 2), 8, 1, __VA_ARGS__) RFI_CASE_MCG(BITS, FN, (F + 3), 8, 1, __VA_ARGS__)
#define RFI_DISPATCH_FMT8(FN, MODE, CW, G, ...)              \
    do {                                                     \
        switch (MODE * 1000 + CW * 10 + G) {                 \
            RFI_CASES_FMT(8, FN, 64, __VA_ARGS__)            \
            RFI_CASES_FMT(8, FN, 128, __VA_ARGS__)           \
            default: break;                                  \
        }                                                    \
    } while (0)
#define RFI_DISPATCH_FMT12(FN, MODE, CW, G, ...)             \
    do {                                                     \
        switch (MODE * 1000 + CW * 10 + G) {                 \
            RFI_CASES_FMT(12, FN, 64, __VA_ARGS__)           \
            default: break;                                  \
        }                                                    \
    } while (0)

}  // namespace dev
}  // namespace rfi
