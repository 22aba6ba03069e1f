// rfi_excise_host: excision of host-resident streams with the host->device copy, the kernel and
// the device->host copy of consecutive chunks overlapped on three streams and three buffer slots.

#include <algorithm>
#include <cstring>

#include <cuda_runtime.h>

#include "rfi.h"
#include "internal.h"
#include "plan_impl.h"

namespace rfi {

namespace {
constexpr int64_t kChunkTarget = 128ll << 20;  // input bytes per chunk
}

void plan_release_host_pipe(rfi_plan_s *P) {
    HostPipe &h = P->pipe;
    for (int i = 0; i < HostPipe::kSlots; ++i) {
        if (h.in[i]) cudaFree(h.in[i]);
        if (h.out[i]) cudaFree(h.out[i]);
        if (h.mask[i]) cudaFree(h.mask[i]);
        if (h.counts[i]) cudaFree(h.counts[i]);
        if (h.h2d[i]) cudaEventDestroy(h.h2d[i]);
        if (h.comp[i]) cudaEventDestroy(h.comp[i]);
        if (h.d2h[i]) cudaEventDestroy(h.d2h[i]);
        h.in[i] = h.out[i] = nullptr;
        h.mask[i] = h.counts[i] = nullptr;
        h.h2d[i] = h.comp[i] = h.d2h[i] = nullptr;
    }
    if (h.s_comp) cudaStreamDestroy(h.s_comp);
    if (h.s_d2h) cudaStreamDestroy(h.s_d2h);
    h.s_comp = h.s_d2h = nullptr;
    h.ready = false;
    P->host_pipe_bytes = 0;
    cudaGetLastError();
}

namespace {

// windows per chunk of stream i
int64_t chunk_windows(const rfi_plan_s *P, int i) {
    const int bps = P->bits == 8 ? 1 : 2;
    return std::max<int64_t>(1, kChunkTarget / (static_cast<int64_t>(P->W[i]) * bps));
}

rfi_status ensure_pipe(rfi_plan_s *P) {
    HostPipe &h = P->pipe;
    if (h.ready) return RFI_OK;
    const int bps = P->bits == 8 ? 1 : 2;
    int64_t in_b = 0, mask_b = 0, cnt_b = 0;
    for (int i = 0; i < P->S; ++i) {
        const int64_t cw = std::min(chunk_windows(P, i), P->nwin[i]);
        in_b = std::max(in_b, cw * P->W[i] * bps);
        mask_b = std::max(mask_b, cw * ((P->W[i] + 31) / 32) * 4);
        cnt_b = std::max(cnt_b, cw * 4);
    }
    in_b = (in_b + 255) / 256 * 256;
    h.chunk_bytes = in_b;
    bool ok = true;
    for (int s = 0; s < HostPipe::kSlots && ok; ++s) {
        ok = cudaMalloc(&h.in[s], in_b) == cudaSuccess && cudaMalloc(&h.out[s], in_b) == cudaSuccess &&
             cudaMalloc(&h.mask[s], mask_b) == cudaSuccess && cudaMalloc(&h.counts[s], cnt_b) == cudaSuccess &&
             cudaEventCreateWithFlags(&h.h2d[s], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&h.comp[s], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&h.d2h[s], cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaStreamCreateWithFlags(&h.s_comp, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&h.s_d2h, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        plan_release_host_pipe(P);
        return RFI_ERR_OOM;
    }
    P->host_pipe_bytes = HostPipe::kSlots * (2 * in_b + mask_b + cnt_b);
    h.ready = true;
    return RFI_OK;
}

}  // namespace

}  // namespace rfi

using namespace rfi;

extern "C" rfi_status rfi_excise_host(rfi_plan_t P, const void *const *in, void *const *out,
                                      uint32_t *const *mask, uint32_t *const *counts, void *stream) {
    if (!P) return RFI_ERR_INVALID_ARG;
    if (!P->parts.empty()) {
        if (!in || !out) return RFI_ERR_INVALID_ARG;
        for (size_t k = 0; k < P->parts.size(); ++k) {
            const auto a = part_args<const void *>(P, k, in);
            const auto b = part_args<void *>(P, k, out);
            const auto m = part_args<uint32_t *>(P, k, mask);
            const auto c = part_args<uint32_t *>(P, k, counts);
            const rfi_status rs = rfi_excise_host(P->parts[k], a.data(), b.data(), mask ? m.data() : nullptr,
                                                  counts ? c.data() : nullptr, stream);
            if (rs != RFI_OK) return rs;
        }
        P->last_windows = P->total_windows;
        return RFI_OK;
    }
    if (P->kmom >= 2) return RFI_ERR_UNSUPPORTED;  // Eq. 3 needs every earlier window's MAD
    if (P->power) return RFI_ERR_UNSUPPORTED;      // the chunk kernels do not meter power
    if (P->out_format != RFI_OUT_SAME) return RFI_ERR_UNSUPPORTED;
    rfi_status rs = plan_check_buffers(P, in, out, mask, counts);
    if (rs != RFI_OK) return rs;
    rs = ensure_pipe(P);
    if (rs != RFI_OK) return rs;
    HostPipe &h = P->pipe;
    cudaStream_t s_h2d = static_cast<cudaStream_t>(stream);
    const int bps = P->bits == 8 ? 1 : 2;
    const Params p = plan_params(P);
#define RFI_PIPE(call)                                   \
    do {                                                 \
        if ((call) != cudaSuccess) return RFI_ERR_CUDA;  \
    } while (0)
    // the counters are reset on the compute stream, which every kernel below follows
    RFI_PIPE(cudaMemsetAsync(P->d_ctr, 0, sizeof(DevCounters), h.s_comp));
    int64_t q = 0;  // chunk sequence number
    for (int i = 0; i < P->S; ++i) {
        const int64_t cw = chunk_windows(P, i);
        const int64_t mw = (P->W[i] + 31) / 32;
        for (int64_t w0 = 0; w0 < P->nwin[i]; w0 += cw, ++q) {
            const int slot = static_cast<int>(q % HostPipe::kSlots);
            const int64_t nw = std::min(cw, P->nwin[i] - w0);
            const int64_t s0 = w0 * P->W[i];
            const int64_t ns = std::min<int64_t>(P->len[i], (w0 + nw) * P->W[i]) - s0;
            if (q >= HostPipe::kSlots) RFI_PIPE(cudaStreamWaitEvent(s_h2d, h.d2h[slot], 0));
            RFI_PIPE(cudaMemcpyAsync(h.in[slot], static_cast<const uint8_t *>(in[i]) + s0 * bps, ns * bps,
                                     cudaMemcpyHostToDevice, s_h2d));
            RFI_PIPE(cudaEventRecord(h.h2d[slot], s_h2d));
            RFI_PIPE(cudaStreamWaitEvent(h.s_comp, h.h2d[slot], 0));
            Seg g;
            std::memset(&g, 0, sizeof(g));
            g.in = h.in[slot];
            g.out = h.out[slot];
            g.mask = (mask && mask[i]) ? h.mask[slot] : nullptr;
            g.counts = (counts && counts[i]) ? h.counts[slot] : nullptr;
            g.med = P->d_med + P->woff[i] + w0;
            g.mad = P->d_mad + P->woff[i] + w0;
            g.len = ns;
            g.abs0 = s0;
            g.W = P->W[i];
            g.stream_id = P->sid[i];
            g.mask_words = static_cast<int32_t>(mw);
            g.vec = (static_cast<int64_t>(P->W[i]) * bps) % 16 == 0;
            RFI_PIPE(launch_stream(P->bits, P->mode, P->shape.consumer_warps, g, 0, nw, p, h.s_comp));
            RFI_PIPE(cudaEventRecord(h.comp[slot], h.s_comp));
            RFI_PIPE(cudaStreamWaitEvent(h.s_d2h, h.comp[slot], 0));
            RFI_PIPE(cudaMemcpyAsync(static_cast<uint8_t *>(out[i]) + s0 * bps, h.out[slot], ns * bps,
                                     cudaMemcpyDeviceToHost, h.s_d2h));
            if (g.mask)
                RFI_PIPE(cudaMemcpyAsync(mask[i] + w0 * mw, h.mask[slot], nw * mw * 4, cudaMemcpyDeviceToHost,
                                         h.s_d2h));
            if (g.counts)
                RFI_PIPE(cudaMemcpyAsync(counts[i] + w0, h.counts[slot], nw * 4, cudaMemcpyDeviceToHost, h.s_d2h));
            RFI_PIPE(cudaEventRecord(h.d2h[slot], h.s_d2h));
        }
    }
    RFI_PIPE(cudaStreamSynchronize(h.s_d2h));
    RFI_PIPE(cudaStreamSynchronize(h.s_comp));
    RFI_PIPE(cudaStreamSynchronize(s_h2d));
#undef RFI_PIPE
    P->last_windows = P->total_windows;
    return RFI_OK;
}
