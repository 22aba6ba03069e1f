// Digital noise as a second pass (Eq. 2's noise replacement, value as in noise_value).
//
// The excision pass of a noise plan created with RFI_PLAN_NOISE_PASS runs as a zero-replacement
// pass: it writes 0 at every flagged sample, the flag mask and every window's M and D. This
// kernel then overwrites the flagged samples with M + the Philox noise of spread 1.4826·D, keyed
// by the absolute sample index as always, so the result is the same bits as the one-pass form.
//
// Work: a unit is a run of 256 mask words; warp g of the grid takes units g, g + nwarps, ...
// (segment s holds units [fwin[s], fwin[s + 1])), so that at any time the warps read masks and
// write samples close to one another (giving each warp a run of consecutive units instead
// made the k = 3 call of the 60-stream benchmark 40 % slower). Windows of at most kFillPackMax
// samples, a multiple of 128 (fill_packs), are packed: the segment's mask is one array of words
// (window k's at k * mw, word j covering samples 32j .. 32j + 31 of the segment) cut into units
// regardless of the windows, so a unit spans several windows and each lane takes M and D of the
// window its four words belong to. Otherwise every window has ceil(mw / 256) units of its own,
// and a unit of a window whose count is 0 is skipped. The unit goes in two halves of 128 words: lane l reads words
// 4l .. 4l + 3 of a half, and the warp moves their flagged samples into its ring of positions:
//  - a word with at least kFillDense flags goes whole: lane j tests bit j and a ballot with a
//    prefix popcount gives each flagged lane its place in the ring;
//  - from the other words every lane gives up one flag per step (its lowest remaining one),
//    compacted the same way.
// Whenever 32 positions wait in the ring, every lane takes one and evaluates its noise. A ring
// entry carries the window's M and D with the position, so the ring runs on across the warp's
// units of a segment and its last fewer-than-32 positions go out only when the segment changes
// or the warp ends. Every lane of a batch but those of such a last one has a sample.

#include "core.cuh"

namespace rfi {
namespace dev {

constexpr int kFillThreads = 256;
constexpr int kFillRing = 64;   // positions a warp's ring holds: fewer than 32 wait between steps
constexpr int kFillDense = 2;   // flags from which a mask word is expanded whole

template <int BITS>
__device__ __forceinline__ void fill_store(uint8_t *out, uint32_t pos, int32_t z) {
    if (BITS == 8) out[pos] = static_cast<uint8_t>(z);
    else reinterpret_cast<int16_t *>(out)[pos] = static_cast<int16_t>(z);
}

// The warp's ring: queued positions (segment-relative sample index, with the window's M in the
// low and D in the high 16 bits of md) and the batches that empty it.
template <int BITS>
struct FillRing {
    uint2 *q;
    uint32_t head, tail;  // positions taken / queued so far
    const Seg *g;
    const KeysPre *key;
    int lane;

    __device__ __forceinline__ void emit(uint2 e) const {
        const int32_t M = static_cast<int16_t>(e.y & 0xFFFFu);
        const uint32_t sigq = 97164u * (e.y >> 16);
        const int32_t z = noise_value(M, sigq, *key, g->stream_id, g->abs0 + static_cast<int64_t>(e.x),
                                      Geo<BITS>::kLo, Geo<BITS>::kHi);
        fill_store<BITS>(g->out, e.x, z);
    }
    // Queue the flagged lanes' positions (every lane calls this), then empty a full batch.
    __device__ __forceinline__ void put(bool fl, uint32_t pos, uint32_t md) {
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, fl);
        if (fl) q[(tail + static_cast<uint32_t>(__popc(bal & ((1u << lane) - 1u)))) & (kFillRing - 1)] = make_uint2(pos, md);
        tail += static_cast<uint32_t>(__popc(bal));
        if (tail - head >= 32u) {
            __syncwarp();
            const uint2 e = q[(head + static_cast<uint32_t>(lane)) & (kFillRing - 1)];
            __syncwarp();  // read before the next step refills the slot
            head += 32u;
            emit(e);
        }
    }
    // The positions still waiting (fewer than 32).
    __device__ __forceinline__ void drain() {
        if (tail == head) return;
        __syncwarp();
        if (static_cast<uint32_t>(lane) < tail - head) emit(q[(head + static_cast<uint32_t>(lane)) & (kFillRing - 1)]);
        __syncwarp();
        head = tail;
    }
};

// Segments hold fewer than 2^31 samples (the plan routes longer ones through the one-pass form),
// so every segment-relative index below fits 32 bits.
// PACK: some segment of the launch is packed (the instantiation without it is the per-window
// form alone, with fewer registers).
template <int BITS, bool PACK>
__global__ void __launch_bounds__(kFillThreads) noise_fill_kernel(const Seg *__restrict__ segs, int nseg,
                                                                 const uint32_t *__restrict__ fwin, uint32_t nunits,
                                                                 Params p) {
    __shared__ uint2 ring_s[kFillThreads / 32][kFillRing];
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const KeysPre key{p};
    FillRing<BITS> R{ring_s[threadIdx.x >> 5], 0u, 0u, segs, &key, lane};
    int s = 0;
    for (uint32_t u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nunits; u += nwarps) {
        if (fwin[s + 1] <= u) {  // a warp's units ascend: the queue belongs to the segment
            R.drain();
            while (s + 1 < nseg && fwin[s + 1] <= u) ++s;
            R.g = &segs[s];
        }
        const Seg &g = segs[s];
        const uint32_t mw = static_cast<uint32_t>(g.mask_words);
        const uint32_t local = u - fwin[s];
        const bool packed = PACK && fill_packs(g.W);
        const uint32_t *mk = g.mask;
        uint32_t j00, jend, pos0 = 0u, md = 0u;
        if (packed) {
            j00 = local << 8;
            jend = min(j00 + 256u, static_cast<uint32_t>((g.len + 31) >> 5));  // the words holding samples
        } else {
            const uint32_t upw = (mw + 255u) >> 8;  // units per window
            const uint32_t k = local / upw;
            j00 = (local - k * upw) << 8;
            jend = min(j00 + 256u, mw);
            if (g.counts && g.counts[k] == 0u) continue;
            md = (static_cast<uint32_t>(g.med[k]) & 0xFFFFu) | (static_cast<uint32_t>(g.mad[k]) << 16);
            mk += static_cast<size_t>(k) * mw;
            pos0 = k * static_cast<uint32_t>(g.W);
        }
        // a packed segment's words of a lane lie in one window (mw is a multiple of 4)
        const bool vec = (mw & 3u) == 0u && (reinterpret_cast<uintptr_t>(mk) & 15u) == 0u;
        const int lg = PACK && (mw & (mw - 1u)) == 0u ? __ffs(mw) - 1 : -1;  // log2 mw, or -1
        for (uint32_t j0 = j00; j0 < jend; j0 += 128u) {
            const uint32_t jl = j0 + 4u * static_cast<uint32_t>(lane);  // this lane's first word
            uint32_t m[4];
            uint32_t mdl = md;
            if (vec) {
                const uint4 a = jl < jend ? *reinterpret_cast<const uint4 *>(mk + jl) : make_uint4(0u, 0u, 0u, 0u);
                m[0] = a.x;
                m[1] = a.y;
                m[2] = a.z;
                m[3] = a.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) m[i] = jl + i < jend ? mk[jl + i] : 0u;
            }
            if (packed && jl < jend) {
                const uint32_t k = lg >= 0 ? jl >> lg : jl / mw;
                mdl = (static_cast<uint32_t>(g.med[k]) & 0xFFFFu) | (static_cast<uint32_t>(g.mad[k]) << 16);
            }
            if (!__any_sync(0xFFFFFFFFu, (m[0] | m[1] | m[2] | m[3]) != 0u)) continue;  // on to the next half
            // dense words, one at a time over the whole warp
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t wi = m[i];
                const bool d = __popc(wi) >= kFillDense;
                uint32_t dense = __ballot_sync(0xFFFFFFFFu, d);
                if (d) m[i] = 0u;
                while (dense) {
                    const int src = __ffs(dense) - 1;
                    dense &= dense - 1u;
                    const uint32_t w = __shfl_sync(0xFFFFFFFFu, wi, src);
                    const uint32_t mdw = PACK ? __shfl_sync(0xFFFFFFFFu, mdl, src) : mdl;
                    const uint32_t pos = pos0 + 32u * (j0 + 4u * static_cast<uint32_t>(src) + i) + static_cast<uint32_t>(lane);
                    R.put(((w >> lane) & 1u) != 0u, pos, mdw);
                }
            }
            // the other words: each lane gives up its lowest remaining flag per step
            while (__any_sync(0xFFFFFFFFu, (m[0] | m[1] | m[2] | m[3]) != 0u)) {
                const bool h0 = m[0] != 0u, h1 = m[1] != 0u, h2 = m[2] != 0u;
                const uint32_t i = h0 ? 0u : (h1 ? 1u : (h2 ? 2u : 3u));
                const uint32_t cur = h0 ? m[0] : (h1 ? m[1] : (h2 ? m[2] : m[3]));
                const uint32_t pos = pos0 + 32u * (jl + i) + static_cast<uint32_t>(__ffs(cur) - 1);
                const uint32_t rest = cur & (cur - 1u);
                if (h0) m[0] = rest;
                else if (h1) m[1] = rest;
                else if (h2) m[2] = rest;
                else m[3] = rest;
                R.put(cur != 0u, pos, mdl);
            }
        }
    }
    R.drain();
}

}  // namespace dev

int noise_fill_grid(int sm_count, bool packed) {
    int n = 0;
    const cudaError_t e = packed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dev::noise_fill_kernel<8, true>, dev::kFillThreads, 0)
                                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dev::noise_fill_kernel<8, false>, dev::kFillThreads, 0);
    if (e != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return sm_count * n;
}

cudaError_t launch_noise_fill(int bits, bool packed, const Seg *segs, int nseg, const uint32_t *fwin, uint32_t nunits,
                              const Params &p, int grid, cudaStream_t st) {
    if (nunits == 0) return cudaSuccess;
    if (bits == 8) {
        if (packed) dev::noise_fill_kernel<8, true><<<grid, dev::kFillThreads, 0, st>>>(segs, nseg, fwin, nunits, p);
        else dev::noise_fill_kernel<8, false><<<grid, dev::kFillThreads, 0, st>>>(segs, nseg, fwin, nunits, p);
    } else {
        if (packed) dev::noise_fill_kernel<12, true><<<grid, dev::kFillThreads, 0, st>>>(segs, nseg, fwin, nunits, p);
        else dev::noise_fill_kernel<12, false><<<grid, dev::kFillThreads, 0, st>>>(segs, nseg, fwin, nunits, p);
    }
    return cudaGetLastError();
}

}  // namespace rfi
