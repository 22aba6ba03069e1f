// Digital noise as a second pass (Eq. 2's noise replacement, value as in noise_value).
//
// The excision pass of a noise plan created with RFI_PLAN_NOISE_PASS runs as a zero-replacement
// pass: it writes 0 at every flagged sample, the flag mask and every window's M and D. This
// kernel then overwrites the flagged samples with M + the Philox noise of spread 1.4826·D, keyed
// by the absolute sample index as always, so the result is the same bits as the one-pass form.
// Inside the excision kernel the flagged samples are found and shared out between the window's
// warps around its barriers, a fixed cost per window; here every warp works on its own block of
// the mask at full occupancy, with idle lanes where a block holds few flags.
//
// Work: segment s covers blocks [fblk[s], fblk[s + 1]) of kFillBlockWords = 64 mask words
// (2048 samples; a window's mask words are consecutive, windows follow one another). Lane l of
// a warp holds words 2l and 2l + 1 of its block; the warp numbers the block's flagged samples
// with a shuffle scan and evaluates Philox for 32 of them at a time, each lane finding its
// sample's owner lane by a shuffle binary search and the bit by a popcount search.

#include "core.cuh"

namespace rfi {
namespace dev {

constexpr int kFillThreads = 256;
static_assert(kFillBlockWords == 64, "two mask words per lane");

template <int BITS>
__device__ __forceinline__ void fill_store(uint8_t *out, uint32_t pos, int32_t z) {
    if (BITS == 8) out[pos] = static_cast<uint8_t>(z);
    else reinterpret_cast<int16_t *>(out)[pos] = static_cast<int16_t>(z);
}

// Segments hold fewer than 2^31 samples (the plan routes longer ones through the one-pass form),
// so every index below fits 32 bits.
template <int BITS>
__global__ void __launch_bounds__(kFillThreads) noise_fill_kernel(const Seg *__restrict__ segs, int nseg,
                                                                 const uint32_t *__restrict__ fblk, uint32_t nblk,
                                                                 Params p) {
    constexpr unsigned kAll = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const KeysPre key{p};
    int s = 0;
    for (uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nblk; b += nwarps) {
        while (s + 1 < nseg && fblk[s + 1] <= b) ++s;  // a warp's blocks ascend
        const Seg &g = segs[s];
        const uint32_t mw = static_cast<uint32_t>(g.mask_words), W = static_cast<uint32_t>(g.W);
        const uint32_t len = static_cast<uint32_t>(g.len);
        const uint32_t nwords = ((len + W - 1) / W) * mw;
        const uint32_t word0 = (b - fblk[s]) * static_cast<uint32_t>(kFillBlockWords);
        const uint32_t wa = word0 + 2u * static_cast<uint32_t>(lane);
        const uint32_t ma = wa < nwords ? g.mask[wa] : 0u;
        const uint32_t mb = wa + 1u < nwords ? g.mask[wa + 1u] : 0u;
        if (!__any_sync(kAll, (ma | mb) != 0u)) continue;
        const uint32_t cnt = __popc(ma) + __popc(mb);
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kAll, inc, o);
            if (lane >= o) inc += y;
        }
        const uint32_t total = __shfl_sync(kAll, inc, 31);
        const uint32_t excl = inc - cnt;
        if (W % 32u == 0u && mw % 64u == 0u) {
            // the block lies in one window k, and sample = 32 * word + bit
            const uint32_t k = word0 / mw;
            const int32_t M = g.med[k];
            const uint32_t S = 97164u * static_cast<uint32_t>(g.mad[k]);
            for (uint32_t q0 = 0; q0 < total; q0 += 32) {
                const uint32_t q = q0 + static_cast<uint32_t>(lane);
                // owner: the last lane whose first number is <= q (lanes without flags share
                // the next lane's first number, so the search passes over them)
                int L = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const uint32_t e = __shfl_sync(kAll, excl, L + step);
                    if (e <= q) L += step;
                }
                const uint32_t eL = __shfl_sync(kAll, excl, L);
                const uint32_t aL = __shfl_sync(kAll, ma, L), bL = __shfl_sync(kAll, mb, L);
                if (q < total) {
                    const uint32_t j = q - eL, ca = __popc(aL);
                    const bool first = j < ca;
                    const uint32_t bit = static_cast<uint32_t>(nth_set_bit(first ? aL : bL, static_cast<int>(first ? j : j - ca)));
                    const uint32_t pos = 32u * (word0 + 2u * static_cast<uint32_t>(L) + (first ? 0u : 1u)) + bit;
                    if (pos < len) {
                        const int32_t z = noise_value(M, S, key, g.stream_id, g.abs0 + static_cast<int64_t>(pos),
                                                      Geo<BITS>::kLo, Geo<BITS>::kHi);
                        fill_store<BITS>(g.out, pos, z);
                    }
                }
            }
        } else {
            // general windows: each lane brings the window, M, spread and first sample of its
            // two words (a window's last word holds W mod 32 samples when 32 does not divide W)
            const uint32_t ka = wa / mw;
            const uint32_t kb = ka + ((wa + 1u - ka * mw) == mw ? 1u : 0u);
            const uint32_t sa = ka * W + (wa - ka * mw) * 32u;
            const uint32_t sb = kb * W + (wa + 1u - kb * mw) * 32u;
            const bool la = ma != 0u, lb = mb != 0u;
            const int32_t Ma = la ? g.med[ka] : 0, Mb = lb ? g.med[kb] : 0;
            const uint32_t Sa = la ? 97164u * static_cast<uint32_t>(g.mad[ka]) : 0u;
            const uint32_t Sb = lb ? 97164u * static_cast<uint32_t>(g.mad[kb]) : 0u;
            for (uint32_t q0 = 0; q0 < total; q0 += 32) {
                const uint32_t q = q0 + static_cast<uint32_t>(lane);
                int L = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const uint32_t e = __shfl_sync(kAll, excl, L + step);
                    if (e <= q) L += step;
                }
                const uint32_t eL = __shfl_sync(kAll, excl, L);
                const uint32_t aL = __shfl_sync(kAll, ma, L), bL = __shfl_sync(kAll, mb, L);
                const int32_t MaL = __shfl_sync(kAll, Ma, L), MbL = __shfl_sync(kAll, Mb, L);
                const uint32_t SaL = __shfl_sync(kAll, Sa, L), SbL = __shfl_sync(kAll, Sb, L);
                const uint32_t saL = __shfl_sync(kAll, sa, L), sbL = __shfl_sync(kAll, sb, L);
                if (q < total) {
                    const uint32_t j = q - eL, ca = __popc(aL);
                    const bool first = j < ca;
                    const uint32_t bit = static_cast<uint32_t>(nth_set_bit(first ? aL : bL, static_cast<int>(first ? j : j - ca)));
                    const uint32_t pos = (first ? saL : sbL) + bit;
                    if (pos < len) {
                        const int32_t z = noise_value(first ? MaL : MbL, first ? SaL : SbL, key, g.stream_id,
                                                      g.abs0 + static_cast<int64_t>(pos), Geo<BITS>::kLo, Geo<BITS>::kHi);
                        fill_store<BITS>(g.out, pos, z);
                    }
                }
            }
        }
    }
}

}  // namespace dev

int noise_fill_grid(int sm_count) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dev::noise_fill_kernel<8>, dev::kFillThreads, 0) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return sm_count * n;
}

cudaError_t launch_noise_fill(int bits, const Seg *segs, int nseg, const uint32_t *fblk, uint32_t nblk, const Params &p,
                              int grid, cudaStream_t st) {
    if (nblk == 0) return cudaSuccess;
    if (bits == 8) dev::noise_fill_kernel<8><<<grid, dev::kFillThreads, 0, st>>>(segs, nseg, fblk, nblk, p);
    else dev::noise_fill_kernel<12><<<grid, dev::kFillThreads, 0, st>>>(segs, nseg, fblk, nblk, p);
    return cudaGetLastError();
}

}  // namespace rfi
