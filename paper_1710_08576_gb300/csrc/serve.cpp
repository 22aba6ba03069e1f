// Serving: real-time excision of chunked sample streams plus backfill requests, continuously
// batched into persistent-kernel passes. Semantics are stated in include/rfi.h.
//
// Memory: one device arena of memory_budget bytes holds the per-stream rings, the buffers of
// the (at most two) passes in flight, and the device copies of host requests (first-fit).
// Streams: three positions per ring, all absolute sample indices. produced (pushed),
// sched (windows handed to a pass), completed (windows whose pass finished), released (output
// read and freed). A push needs room between produced and released + capacity.
// Passes: copies run on a copy stream, kernels on a compute stream that waits for every copy
// enqueued before the pass was built, so a pass only sees landed data.

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "rfi.h"
#include "internal.h"

namespace rfi {
namespace {

constexpr int kSlots = 2;                 // passes in flight
constexpr int kMaxPassTiles = 262144;     // work-list entries per pass
constexpr int kDefaultReqWindows = 1024;  // request windows per pass

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

struct Arena {
    uint8_t *base = nullptr;
    size_t size = 0, used = 0, peak = 0;
    std::vector<std::pair<size_t, size_t>> free_;  // (offset, bytes), sorted by offset
    bool alloc(size_t bytes, size_t *off) {
        bytes = al256(bytes);
        for (size_t i = 0; i < free_.size(); ++i) {
            if (free_[i].second >= bytes) {
                *off = free_[i].first;
                free_[i].first += bytes;
                free_[i].second -= bytes;
                if (free_[i].second == 0) free_.erase(free_.begin() + static_cast<long>(i));
                used += bytes;
                peak = std::max(peak, used);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = al256(bytes);
        used -= bytes;
        auto it = std::lower_bound(free_.begin(), free_.end(), std::make_pair(off, size_t(0)));
        it = free_.insert(it, {off, bytes});
        // merge with neighbours
        size_t i = static_cast<size_t>(it - free_.begin());
        if (i + 1 < free_.size() && free_[i].first + free_[i].second == free_[i + 1].first) {
            free_[i].second += free_[i + 1].second;
            free_.erase(free_.begin() + static_cast<long>(i) + 1);
        }
        if (i > 0 && free_[i - 1].first + free_[i - 1].second == free_[i].first) {
            free_[i - 1].second += free_[i].second;
            free_.erase(free_.begin() + static_cast<long>(i));
        }
    }
    size_t largest_free() const {
        size_t m = 0;
        for (auto &f : free_) m = std::max(m, f.second);
        return m;
    }
};

struct Ring {
    int32_t W = 0;
    uint32_t sid = 0;
    int64_t start = 0, cap = 0, nslots = 0, mw = 0;
    uint8_t *in = nullptr, *out = nullptr;
    uint32_t *mask = nullptr, *counts = nullptr;
    int32_t *med = nullptr, *mad = nullptr;
    int64_t produced = 0, sched = 0, completed = 0, released = 0;
    bool flushing = false, finished = false;
};

struct Chunk {
    uint64_t ticket;
    int32_t stream;
    int64_t end;        // absolute index one past the chunk
    cudaEvent_t ev;     // recorded after the chunk's copy
    bool assigned = false;
};

struct Request {
    uint64_t ticket = 0;
    rfi_request_desc d{};
    int bps = 1;
    int64_t nwin = 0, next_w = 0, mw = 0;
    const uint8_t *din = nullptr;
    uint8_t *dout = nullptr;
    uint32_t *dmask = nullptr, *dcounts = nullptr;
    size_t off = 0, bytes = 0;
    bool host = false, arena = false;
    cudaEvent_t ev_submit = nullptr, ev_done = nullptr;
    bool pass_done = false;  // the pass with its last windows has finished
    float lat_ms = 0.f;      // submit -> last pass (device requests)
};

// Per-pass upload: the segment table followed by the work list, staged in pinned memory and
// copied to the device in one transfer.
struct Slot {
    uint8_t *d_buf = nullptr;  // device: segs at 0, tiles at tiles_off
    uint8_t *h_buf = nullptr;  // pinned host staging of the same layout
    size_t tiles_off = 0;
    int max_segs = 0;
};

struct Pass {
    int64_t seq = 0;
    int slot = 0;
    cudaEvent_t ev0 = nullptr, ev = nullptr;  // pass start and end on the compute stream
    std::vector<std::pair<int, int64_t>> completes;  // (stream, completed position after)
    std::vector<size_t> chunks;                      // indices into the chunk list
    std::vector<uint64_t> requests;                  // requests whose last windows ran here
};

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t i = static_cast<size_t>(pos);
    const double f = pos - i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace
}  // namespace rfi

struct rfi_server_s {
    int bits = 8, bps = 1, S = 0, mode = 0;
    int64_t kq = 0;
    int32_t cval = 0;
    uint64_t seed = 0;
    int max_requests = 1, req_windows = rfi::kDefaultReqWindows;
    int sm_count = 0;
    rfi::Arena arena;
    std::vector<rfi::Ring> rings;
    std::deque<rfi::Chunk> chunks;   // pending and recently done chunks
    size_t chunk_base = 0;           // index of chunks.front() in ticket order
    std::vector<rfi::Request> reqs;  // active requests
    std::vector<rfi::Pass> inflight;
    rfi::Slot slots[rfi::kSlots];
    bool slot_busy[rfi::kSlots] = {false, false};
    rfi::DevCounters *d_ctr = nullptr;  // status and flagged total of every pass (never reset)
    cudaStream_t s_copy = nullptr, s_comp = nullptr, s_back = nullptr;
    cudaEvent_t ev_copies = nullptr;
    uint64_t next_ticket = 1;
    int64_t pass_seq = 0, passes_done = 0;
    // results: latency (us) of every finished chunk and request
    std::unordered_map<uint64_t, double> done_lat;       // ticket -> latency, until taken
    std::deque<std::pair<uint64_t, double>> recent;      // finished, oldest first, until taken
    std::vector<double> chunk_lat, req_lat;              // all finished, for the percentiles
    double busy_s = 0;                                   // sum of pass durations (device clock)
    uint64_t samples_done = 0, req_samples_done = 0, flagged = 0, requests_done = 0;
    uint32_t status = 0;
    double t_first = -1, t_last = 0;
};

using namespace rfi;

namespace {

#define SRV_CUDA(x)                                          \
    do {                                                     \
        if ((x) != cudaSuccess) return RFI_ERR_CUDA;         \
    } while (0)

Params server_params(const rfi_server_s *s, DevCounters *ctr) {  // ctr: the server's counters
    Params p{};
    p.kq = s->kq;
    p.seed = s->seed;
    p.cval = s->cval;
    p.ncopies = s->bits == 8 ? 1 : 2;
    p.status = &ctr->status;
    p.flagged = &ctr->flagged;
    set_round_keys(p);
    return p;
}

void touch(rfi_server_s *s) {
    if (s->t_first < 0) s->t_first = now_s();
}

// Retire finished passes and requests (non-blocking).
rfi_status poll_all(rfi_server_s *s) {
    while (!s->inflight.empty()) {
        Pass &ps = s->inflight.front();
        const cudaError_t q = cudaEventQuery(ps.ev);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) return RFI_ERR_CUDA;
        for (auto &cp : ps.completes) {
            Ring &r = s->rings[cp.first];
            s->samples_done += static_cast<uint64_t>(cp.second - r.completed);
            r.completed = cp.second;
        }
        for (uint64_t t : ps.requests)
            for (auto &rq : s->reqs)
                if (rq.ticket == t) {
                    rq.pass_done = true;
                    if (!rq.host) cudaEventElapsedTime(&rq.lat_ms, rq.ev_submit, ps.ev);
                }
        for (size_t ci : ps.chunks) {
            Chunk &ch = s->chunks[ci - s->chunk_base];
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ch.ev, ps.ev);
            s->done_lat[ch.ticket] = 1000.0 * ms;
            s->recent.push_back({ch.ticket, 1000.0 * ms});
            s->chunk_lat.push_back(1000.0 * ms);
            cudaEventDestroy(ch.ev);
            ch.ev = nullptr;
        }
        float pass_ms = 0.f;
        cudaEventElapsedTime(&pass_ms, ps.ev0, ps.ev);
        s->busy_s += 1e-3 * pass_ms;
        s->slot_busy[ps.slot] = false;
        cudaEventDestroy(ps.ev0);
        cudaEventDestroy(ps.ev);
        s->passes_done = ps.seq + 1;
        s->t_last = now_s();
        s->inflight.erase(s->inflight.begin());
    }
    // drop chunks from the front once their latency is recorded
    while (!s->chunks.empty() && s->chunks.front().assigned && s->chunks.front().ev == nullptr) {
        s->chunks.pop_front();
        ++s->chunk_base;
    }
    // requests: done when their last pass finished (and, for host requests, the copy back)
    for (size_t i = 0; i < s->reqs.size();) {
        Request &rq = s->reqs[i];
        bool done = false;
        if (rq.next_w == rq.nwin && rq.pass_done) {
            if (rq.host) {
                const cudaError_t q = cudaEventQuery(rq.ev_done);
                if (q == cudaSuccess) done = true;
                else if (q != cudaErrorNotReady) return RFI_ERR_CUDA;
            } else {
                done = true;
            }
        }
        if (done) {
            float ms = rq.lat_ms;  // device request: submit -> end of its last pass
            if (rq.host) cudaEventElapsedTime(&ms, rq.ev_submit, rq.ev_done);  // ... -> copied back
            s->done_lat[rq.ticket] = 1000.0 * ms;
            s->recent.push_back({rq.ticket, 1000.0 * ms});
            s->req_lat.push_back(1000.0 * ms);
            s->req_samples_done += static_cast<uint64_t>(rq.d.len);
            ++s->requests_done;
            if (rq.arena) s->arena.release(rq.off, rq.bytes);
            cudaEventDestroy(rq.ev_submit);
            if (rq.ev_done) cudaEventDestroy(rq.ev_done);
            s->reqs.erase(s->reqs.begin() + static_cast<long>(i));
            s->t_last = now_s();
        } else {
            ++i;
        }
    }
    return RFI_OK;
}

void add_tiles(std::vector<Tile> &tiles, uint32_t seg, int64_t len, int32_t W, int bps, int stage_bytes) {
    const int64_t wb = static_cast<int64_t>(W) * bps;
    const int64_t per = (wb % 16 == 0) ? std::max<int64_t>(1, stage_bytes / wb) : 1;
    const int64_t nwin = (len + W - 1) / W;
    for (int64_t w0 = 0; w0 < nwin; w0 += per) {
        const int64_t nw = std::min<int64_t>(per, nwin - w0);
        const int64_t s1 = std::min<int64_t>(len, (w0 + nw) * W);
        tiles.push_back(Tile{seg, static_cast<uint32_t>(w0), static_cast<uint32_t>(nw),
                             static_cast<uint32_t>((s1 - w0 * W) * bps)});
    }
}

}  // namespace

extern "C" {

rfi_status rfi_server_create(const rfi_server_desc *d, rfi_server_t *out) {
    if (!d || !out) return RFI_ERR_INVALID_ARG;
    *out = nullptr;
    if ((d->sample_bits != 8 && d->sample_bits != 12) || d->num_streams < 1 || !d->window_len)
        return RFI_ERR_INVALID_ARG;
    if (!(d->k > 0.0) || !std::isfinite(d->k) || d->k > 1.0e6) return RFI_ERR_INVALID_ARG;
    if (d->mode < RFI_REPLACE_ZERO || d->mode > RFI_REPLACE_NOISE || d->max_requests < 1 ||
        d->request_windows_per_step < 0 || d->ring_samples < 1)
        return RFI_ERR_INVALID_ARG;
    const int64_t kq = static_cast<int64_t>(std::floor(d->k * 1.4826 * 65536.0 + 0.5));
    if (kq < 1) return RFI_ERR_INVALID_ARG;
    for (int i = 0; i < d->num_streams; ++i) {
        if (d->window_len[i] < 1 || d->window_len[i] > 65536) return RFI_ERR_INVALID_ARG;
        if (d->ring_samples < d->window_len[i]) return RFI_ERR_INVALID_ARG;
        if (d->stream_start && (d->stream_start[i] < 0 || d->stream_start[i] % d->window_len[i]))
            return RFI_ERR_INVALID_ARG;
    }
    rfi_server_s *s = new (std::nothrow) rfi_server_s();
    if (!s) return RFI_ERR_OOM;
    s->bits = d->sample_bits;
    s->bps = d->sample_bits == 8 ? 1 : 2;
    s->S = d->num_streams;
    s->mode = d->mode;
    s->kq = kq;
    const int32_t lo = s->bits == 8 ? -128 : -2048, hi = s->bits == 8 ? 127 : 2047;
    s->cval = std::min(hi, std::max(lo, d->const_value));
    s->seed = d->seed;
    s->max_requests = d->max_requests;
    s->req_windows = d->request_windows_per_step ? d->request_windows_per_step : kDefaultReqWindows;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete s;
        return RFI_ERR_CUDA;
    }
    // sizes
    s->rings.resize(s->S);
    size_t ring_bytes = 0;
    for (int i = 0; i < s->S; ++i) {
        Ring &r = s->rings[i];
        r.W = d->window_len[i];
        r.sid = d->stream_id ? d->stream_id[i] : static_cast<uint32_t>(i);
        r.start = d->stream_start ? d->stream_start[i] : 0;
        r.cap = (d->ring_samples + r.W - 1) / r.W * r.W;
        r.nslots = r.cap / r.W;
        r.mw = (r.W + 31) / 32;
        r.produced = r.sched = r.completed = r.released = r.start;
        ring_bytes += 2 * al256(r.cap * s->bps) + al256(r.nslots * r.mw * 4) + 3 * al256(r.nslots * 4);
    }
    const int max_segs = 2 * s->S + s->max_requests;
    const size_t tiles_off = al256(sizeof(Seg) * max_segs);
    const size_t slot_bytes = tiles_off + al256(sizeof(Tile) * kMaxPassTiles);
    const size_t need = ring_bytes + kSlots * slot_bytes + 256;
    if (d->memory_budget < need) {
        delete s;
        return RFI_ERR_OOM;
    }
    s->arena.size = d->memory_budget;
    if (cudaMalloc(&s->arena.base, s->arena.size) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return RFI_ERR_OOM;
    }
    s->arena.free_.push_back({0, s->arena.size});
    auto take = [&](size_t bytes) {
        size_t off = 0;
        s->arena.alloc(bytes, &off);  // fits: checked against `need` above
        return s->arena.base + off;
    };
    for (auto &r : s->rings) {
        r.in = take(r.cap * s->bps);
        r.out = take(r.cap * s->bps);
        r.mask = reinterpret_cast<uint32_t *>(take(r.nslots * r.mw * 4));
        r.counts = reinterpret_cast<uint32_t *>(take(r.nslots * 4));
        r.med = reinterpret_cast<int32_t *>(take(r.nslots * 4));
        r.mad = reinterpret_cast<int32_t *>(take(r.nslots * 4));
    }
    bool ok = true;
    s->d_ctr = reinterpret_cast<DevCounters *>(take(256));
    for (int k = 0; k < kSlots && ok; ++k) {
        Slot &sl = s->slots[k];
        sl.max_segs = max_segs;
        sl.tiles_off = tiles_off;
        sl.d_buf = take(slot_bytes);
        ok = cudaMallocHost(&sl.h_buf, slot_bytes) == cudaSuccess;
    }
    ok = ok && cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->s_back, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->ev_copies, cudaEventDisableTiming) == cudaSuccess &&
         cudaMemset(s->arena.base, 0, need) == cudaSuccess;
    if (!ok) {
        rfi_server_destroy(s);
        return RFI_ERR_CUDA;
    }
    *out = s;
    return RFI_OK;
}

rfi_status rfi_server_push(rfi_server_t s, int32_t stream, const void *samples, int64_t n, int32_t on_device,
                           uint64_t *ticket) {
    if (!s || !samples || n < 1 || stream < 0 || stream >= s->S) return RFI_ERR_INVALID_ARG;
    Ring &r = s->rings[stream];
    if (r.flushing || r.finished) return RFI_ERR_INVALID_ARG;
    rfi_status rs = poll_all(s);
    if (rs != RFI_OK) return rs;
    if (r.produced - r.released + n > r.cap) return RFI_ERR_BUSY;
    touch(s);
    Chunk ch;
    ch.ticket = s->next_ticket++;
    ch.stream = stream;
    ch.end = r.produced + n;
    // arrival: recorded before the copy, so the latency covers copy, wait for a pass and the pass
    SRV_CUDA(cudaEventCreate(&ch.ev));
    SRV_CUDA(cudaEventRecord(ch.ev, s->s_copy));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const uint8_t *src = static_cast<const uint8_t *>(samples);
    int64_t left = n, a = r.produced;
    while (left > 0) {
        const int64_t pos = (a - r.start) % r.cap;
        const int64_t m = std::min(left, r.cap - pos);
        SRV_CUDA(cudaMemcpyAsync(r.in + pos * s->bps, src, m * s->bps, kind, s->s_copy));
        src += m * s->bps;
        a += m;
        left -= m;
    }
    r.produced += n;
    s->chunks.push_back(ch);
    if (ticket) *ticket = ch.ticket;
    return RFI_OK;
}

rfi_status rfi_server_submit(rfi_server_t s, const rfi_request_desc *q, uint64_t *ticket) {
    if (!s || !q || !q->in || !q->out || q->len < 1 || q->window_len < 1 || q->window_len > 65536 || q->abs0 < 0 ||
        q->abs0 % q->window_len)
        return RFI_ERR_INVALID_ARG;
    rfi_status rs = poll_all(s);
    if (rs != RFI_OK) return rs;
    if (static_cast<int>(s->reqs.size()) >= s->max_requests) return RFI_ERR_BUSY;
    Request rq;
    rq.d = *q;
    rq.bps = s->bps;
    rq.nwin = (q->len + q->window_len - 1) / q->window_len;
    rq.mw = (q->window_len + 31) / 32;
    rq.host = !q->on_device;
    if (rq.host) {
        const size_t b_in = al256(q->len * s->bps), b_mask = al256(rq.nwin * rq.mw * 4), b_cnt = al256(rq.nwin * 4);
        rq.bytes = 2 * b_in + b_mask + b_cnt;
        if (rq.bytes > s->arena.size) return RFI_ERR_OOM;
        if (!s->arena.alloc(rq.bytes, &rq.off)) return RFI_ERR_BUSY;
        rq.arena = true;
        uint8_t *b = s->arena.base + rq.off;
        rq.din = b;
        rq.dout = b + b_in;
        rq.dmask = reinterpret_cast<uint32_t *>(b + 2 * b_in);
        rq.dcounts = reinterpret_cast<uint32_t *>(b + 2 * b_in + b_mask);
        if (cudaMemcpyAsync(const_cast<uint8_t *>(rq.din), q->in, q->len * s->bps, cudaMemcpyHostToDevice,
                            s->s_copy) != cudaSuccess) {
            s->arena.release(rq.off, rq.bytes);
            return RFI_ERR_CUDA;
        }
        SRV_CUDA(cudaEventCreateWithFlags(&rq.ev_done, cudaEventDefault));
    } else {
        if (s->bps == 2 && ((reinterpret_cast<uintptr_t>(q->in) | reinterpret_cast<uintptr_t>(q->out)) & 1))
            return RFI_ERR_ALIGNMENT;
        rq.din = static_cast<const uint8_t *>(q->in);
        rq.dout = static_cast<uint8_t *>(q->out);
        rq.dmask = q->mask;
        rq.dcounts = q->counts;
    }
    if ((rq.dmask && (reinterpret_cast<uintptr_t>(rq.dmask) & 3)) ||
        (rq.dcounts && (reinterpret_cast<uintptr_t>(rq.dcounts) & 3))) {
        if (rq.arena) s->arena.release(rq.off, rq.bytes);
        return RFI_ERR_ALIGNMENT;
    }
    touch(s);
    SRV_CUDA(cudaEventCreate(&rq.ev_submit));
    SRV_CUDA(cudaEventRecord(rq.ev_submit, s->s_copy));
    rq.ticket = s->next_ticket++;
    if (ticket) *ticket = rq.ticket;
    s->reqs.push_back(rq);
    return RFI_OK;
}

rfi_status rfi_server_step(rfi_server_t s, int32_t *launched) {
    if (!s) return RFI_ERR_INVALID_ARG;
    if (launched) *launched = 0;
    rfi_status rs = poll_all(s);
    if (rs != RFI_OK) return rs;
    int slot = -1;
    for (int k = 0; k < kSlots; ++k)
        if (!s->slot_busy[k]) {
            slot = k;
            break;
        }
    if (slot < 0) return RFI_OK;  // two passes in flight already
    Slot &sl = s->slots[slot];
    std::vector<Seg> segs;
    std::vector<Tile> tiles;
    Pass ps;
    ps.slot = slot;
    int max_wb = 16384;
    int64_t budget = kMaxPassTiles;  // windows this pass may take
    auto add_seg = [&](const Seg &g) {
        segs.push_back(g);
        max_wb = std::max<int>(max_wb, g.W * s->bps);
    };
    // rings: every complete window that has arrived (the partial tail too once flushed)
    for (int i = 0; i < s->S && budget > 0; ++i) {
        Ring &r = s->rings[i];
        int64_t ready = r.start + (r.produced - r.start) / r.W * r.W;
        if (r.flushing) ready = r.produced;
        if (ready <= r.sched) continue;
        int64_t a = r.sched;
        int64_t end = std::min<int64_t>(ready, a + budget * r.W);
        while (a < end) {
            const int64_t wabs = (a - r.start) / r.W;
            const int64_t slot_w = wabs % r.nslots;
            const int64_t nw_to_wrap = r.nslots - slot_w;
            const int64_t len = std::min<int64_t>(end - a, nw_to_wrap * r.W);
            Seg g;
            std::memset(&g, 0, sizeof(g));
            g.in = r.in + slot_w * r.W * s->bps;
            g.out = r.out + slot_w * r.W * s->bps;
            g.mask = r.mask + slot_w * r.mw;
            g.counts = r.counts + slot_w;
            g.med = r.med + slot_w;
            g.mad = r.mad + slot_w;
            g.len = len;
            g.abs0 = a;
            g.W = r.W;
            g.stream_id = r.sid;
            g.mask_words = static_cast<int32_t>(r.mw);
            g.vec = (static_cast<int64_t>(r.W) * s->bps) % 16 == 0;
            add_seg(g);
            budget -= (len + r.W - 1) / r.W;
            a += len;
        }
        r.sched = end;
        if (r.flushing && r.sched == r.produced) r.finished = true;
        ps.completes.push_back({i, r.sched});
    }
    // requests: a bounded slice of each
    for (auto &rq : s->reqs) {
        if (rq.next_w >= rq.nwin || budget <= 0) continue;
        const int64_t nw = std::min<int64_t>({static_cast<int64_t>(s->req_windows), rq.nwin - rq.next_w, budget});
        const int64_t W = rq.d.window_len;
        const int64_t s0 = rq.next_w * W;
        Seg g;
        std::memset(&g, 0, sizeof(g));
        g.in = rq.din + s0 * s->bps;
        g.out = rq.dout + s0 * s->bps;
        g.mask = rq.dmask ? rq.dmask + rq.next_w * rq.mw : nullptr;
        g.counts = rq.dcounts ? rq.dcounts + rq.next_w : nullptr;
        g.len = std::min<int64_t>(nw * W, rq.d.len - s0);
        g.abs0 = rq.d.abs0 + s0;
        g.W = static_cast<int32_t>(W);
        g.stream_id = rq.d.stream_id;
        g.mask_words = static_cast<int32_t>(rq.mw);
        g.vec = ((reinterpret_cast<uintptr_t>(g.in) | reinterpret_cast<uintptr_t>(g.out)) % 16 == 0) &&
                (W * s->bps) % 16 == 0;
        add_seg(g);
        budget -= nw;
        rq.next_w += nw;
        if (rq.next_w == rq.nwin) ps.requests.push_back(rq.ticket);
    }
    if (segs.empty()) return RFI_OK;
    // launch shape for this pass
    Shape sh{};
    sh.consumer_warps = 8;
    sh.groups = 1;
    sh.hist_copies = s->bits == 8 ? 1 : 2;
    sh.dynamic_tiles = 2;  // static round robin: no work-list cursor to reset between passes
    sh.stage_bytes = (max_wb + 127) / 128 * 128;
    sh.stages = 2;
    while (sh.stages > 1 && persistent_smem_bytes(s->bits, s->mode, sh) > 227u * 1024u) --sh.stages;
    if (persistent_smem_bytes(s->bits, s->mode, sh) > 227u * 1024u) return RFI_ERR_UNSUPPORTED;
    const int occ = persistent_occupancy(s->bits, s->mode, sh);
    if (occ < 1) return RFI_ERR_UNSUPPORTED;
    sh.ctas_per_sm = std::min(occ, 3);
    for (size_t i = 0; i < segs.size(); ++i)
        add_tiles(tiles, static_cast<uint32_t>(i), segs[i].len, segs[i].W, s->bps, sh.stage_bytes);
    if (static_cast<int>(tiles.size()) > kMaxPassTiles || static_cast<int>(segs.size()) > sl.max_segs)
        return RFI_ERR_UNSUPPORTED;
    // one pinned upload: segment table, then the work list (the slot is free, so its staging
    // buffer is no longer read by an earlier copy)
    std::memcpy(sl.h_buf, segs.data(), sizeof(Seg) * segs.size());
    std::memcpy(sl.h_buf + sl.tiles_off, tiles.data(), sizeof(Tile) * tiles.size());
    // the pass sees every copy enqueued so far
    SRV_CUDA(cudaEventRecord(s->ev_copies, s->s_copy));
    SRV_CUDA(cudaStreamWaitEvent(s->s_comp, s->ev_copies, 0));
    SRV_CUDA(cudaEventCreate(&ps.ev0));
    SRV_CUDA(cudaEventRecord(ps.ev0, s->s_comp));
    const size_t up = sl.tiles_off + sizeof(Tile) * tiles.size();
    SRV_CUDA(cudaMemcpyAsync(sl.d_buf, sl.h_buf, up, cudaMemcpyHostToDevice, s->s_comp));
    const int ntiles = static_cast<int>(tiles.size());
    const int grid = std::max(1, std::min(ntiles, s->sm_count * sh.ctas_per_sm));
    SRV_CUDA(launch_persistent(s->bits, s->mode, sh, grid, reinterpret_cast<const Seg *>(sl.d_buf),
                               reinterpret_cast<const Tile *>(sl.d_buf + sl.tiles_off), ntiles,
                               server_params(s, s->d_ctr), nullptr, 0, s->s_comp));
    SRV_CUDA(cudaEventCreate(&ps.ev));
    SRV_CUDA(cudaEventRecord(ps.ev, s->s_comp));
    // host requests finishing here: copy results back after the pass
    for (uint64_t t : ps.requests) {
        for (auto &rq : s->reqs) {
            if (rq.ticket != t || !rq.host) continue;
            // on their own stream, so that later pushes do not wait for this pass
            SRV_CUDA(cudaStreamWaitEvent(s->s_back, ps.ev, 0));
            SRV_CUDA(cudaMemcpyAsync(rq.d.out, rq.dout, rq.d.len * s->bps, cudaMemcpyDeviceToHost, s->s_back));
            if (rq.d.mask)
                SRV_CUDA(cudaMemcpyAsync(rq.d.mask, rq.dmask, rq.nwin * rq.mw * 4, cudaMemcpyDeviceToHost, s->s_back));
            if (rq.d.counts)
                SRV_CUDA(cudaMemcpyAsync(rq.d.counts, rq.dcounts, rq.nwin * 4, cudaMemcpyDeviceToHost, s->s_back));
            SRV_CUDA(cudaEventRecord(rq.ev_done, s->s_back));
        }
    }
    // a chunk is done with the pass that excises the last window ending inside it (its trailing
    // partial window belongs to the chunk that completes it, or to the flush)
    for (size_t k = 0; k < s->chunks.size(); ++k) {
        Chunk &ch = s->chunks[k];
        if (ch.assigned) continue;
        const Ring &r = s->rings[ch.stream];
        const int64_t need = r.flushing ? ch.end : r.start + (ch.end - r.start) / r.W * r.W;
        if (need <= r.sched) {
            ch.assigned = true;
            ps.chunks.push_back(k + s->chunk_base);
        }
    }
    ps.seq = s->pass_seq++;
    s->slot_busy[slot] = true;
    s->inflight.push_back(ps);
    if (launched) *launched = 1;
    return RFI_OK;
}

rfi_status rfi_server_poll(rfi_server_t s, uint64_t ticket, int32_t *done, double *latency_us) {
    if (!s || !done) return RFI_ERR_INVALID_ARG;
    rfi_status rs = poll_all(s);
    if (rs != RFI_OK) return rs;
    *done = 0;
    auto it = s->done_lat.find(ticket);
    if (it != s->done_lat.end()) {
        *done = 1;
        if (latency_us) *latency_us = it->second;
        return RFI_OK;
    }
    return ticket >= s->next_ticket || ticket == 0 ? RFI_ERR_INVALID_ARG : RFI_OK;
}

rfi_status rfi_server_read(rfi_server_t s, int32_t stream, int64_t start, int64_t n, void *dst, uint32_t *mask_dst,
                           int32_t on_device, int32_t release) {
    if (!s || stream < 0 || stream >= s->S || n < 1 || !dst) return RFI_ERR_INVALID_ARG;
    rfi_status rs = poll_all(s);
    if (rs != RFI_OK) return rs;
    Ring &r = s->rings[stream];
    if (start < r.released || start + n > r.completed || (start - r.start) % r.W) return RFI_ERR_INVALID_ARG;
    const bool tail_end = start + n == r.completed && r.finished;
    if (n % r.W && !tail_end) return RFI_ERR_INVALID_ARG;
    if (release && start != r.released) return RFI_ERR_INVALID_ARG;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    uint8_t *d = static_cast<uint8_t *>(dst);
    uint32_t *m = mask_dst;
    int64_t a = start, left = n;
    while (left > 0) {
        const int64_t pos = (a - r.start) % r.cap;
        const int64_t len = std::min(left, r.cap - pos);
        SRV_CUDA(cudaMemcpyAsync(d, r.out + pos * s->bps, len * s->bps, kind, s->s_copy));
        if (m) {
            const int64_t nw = (len + r.W - 1) / r.W;
            SRV_CUDA(cudaMemcpyAsync(m, r.mask + (pos / r.W) * r.mw, nw * r.mw * 4, kind, s->s_copy));
            m += nw * r.mw;
        }
        d += len * s->bps;
        a += len;
        left -= len;
    }
    SRV_CUDA(cudaStreamSynchronize(s->s_copy));
    if (release) r.released = start + n;
    return RFI_OK;
}

rfi_status rfi_server_view(rfi_server_t s, int32_t stream, int64_t start, const void **out, const uint32_t **mask,
                           int64_t *n) {
    if (!s || stream < 0 || stream >= s->S || !out || !n) return RFI_ERR_INVALID_ARG;
    rfi_status rs = poll_all(s);
    if (rs != RFI_OK) return rs;
    const Ring &r = s->rings[stream];
    if (start < r.released || start > r.completed || (start - r.start) % r.W) return RFI_ERR_INVALID_ARG;
    const int64_t pos = (start - r.start) % r.cap;
    *out = r.out + pos * s->bps;
    if (mask) *mask = r.mask + (pos / r.W) * r.mw;
    *n = std::min(r.completed - start, r.cap - pos);
    return RFI_OK;
}

rfi_status rfi_server_release(rfi_server_t s, int32_t stream, int64_t upto) {
    if (!s || stream < 0 || stream >= s->S) return RFI_ERR_INVALID_ARG;
    rfi_status rs = poll_all(s);
    if (rs != RFI_OK) return rs;
    Ring &r = s->rings[stream];
    if (upto < r.released || upto > r.completed) return RFI_ERR_INVALID_ARG;
    if ((upto - r.start) % r.W && !(upto == r.completed && r.finished)) return RFI_ERR_INVALID_ARG;
    r.released = upto;
    return RFI_OK;
}

rfi_status rfi_server_take_latencies(rfi_server_t s, uint64_t *tickets, double *latency_us, int64_t cap,
                                     int64_t *n) {
    if (!s || !n || cap < 0 || (cap > 0 && (!tickets || !latency_us))) return RFI_ERR_INVALID_ARG;
    rfi_status rs = poll_all(s);
    if (rs != RFI_OK) return rs;
    int64_t k = 0;
    while (k < cap && !s->recent.empty()) {
        tickets[k] = s->recent.front().first;
        latency_us[k] = s->recent.front().second;
        s->done_lat.erase(tickets[k]);
        s->recent.pop_front();
        ++k;
    }
    *n = k;
    return RFI_OK;
}

rfi_status rfi_server_flush(rfi_server_t s, int32_t stream) {
    if (!s || stream < 0 || stream >= s->S) return RFI_ERR_INVALID_ARG;
    s->rings[stream].flushing = true;
    if (s->rings[stream].produced == s->rings[stream].sched) s->rings[stream].finished = true;
    return RFI_OK;
}

rfi_status rfi_server_position(rfi_server_t s, int32_t stream, int64_t *produced, int64_t *completed,
                               int64_t *released) {
    if (!s || stream < 0 || stream >= s->S) return RFI_ERR_INVALID_ARG;
    rfi_status rs = poll_all(s);
    if (rs != RFI_OK) return rs;
    const Ring &r = s->rings[stream];
    if (produced) *produced = r.produced;
    if (completed) *completed = r.completed;
    if (released) *released = r.released;
    return RFI_OK;
}

rfi_status rfi_server_drain(rfi_server_t s, double timeout_seconds) {
    if (!s) return RFI_ERR_INVALID_ARG;
    const double t0 = now_s();
    for (;;) {
        int32_t launched = 0;
        rfi_status rs = rfi_server_step(s, &launched);
        if (rs != RFI_OK) return rs;
        bool pending = !s->inflight.empty() || !s->reqs.empty();
        for (auto &r : s->rings) {
            const int64_t ready = r.flushing ? r.produced : r.start + (r.produced - r.start) / r.W * r.W;
            if (ready > r.sched) pending = true;
        }
        if (!pending) return RFI_OK;
        if (now_s() - t0 > timeout_seconds) return RFI_ERR_TIMEOUT;
        if (!launched && !s->inflight.empty()) {
            cudaEventSynchronize(s->inflight.front().ev);
        } else if (!launched) {
            for (auto &rq : s->reqs)
                if (rq.host && rq.pass_done) cudaEventSynchronize(rq.ev_done);
        }
    }
}

rfi_status rfi_server_get_stats(rfi_server_t s, rfi_server_stats *st) {
    if (!s || !st) return RFI_ERR_INVALID_ARG;
    rfi_status rs = poll_all(s);
    if (rs != RFI_OK) return rs;
    DevCounters c;  // totals of the passes that finished (and of any still running)
    SRV_CUDA(cudaMemcpyAsync(&c, s->d_ctr, sizeof(c), cudaMemcpyDeviceToHost, s->s_back));
    SRV_CUDA(cudaStreamSynchronize(s->s_back));
    s->flagged = c.flagged;
    s->status = c.status;
    std::memset(st, 0, sizeof(*st));
    const std::vector<double> &cl = s->chunk_lat, &rl = s->req_lat;
    st->passes = static_cast<uint64_t>(s->passes_done);
    st->chunks_done = cl.size();
    st->requests_done = s->requests_done;
    st->samples_done = s->samples_done;
    st->request_samples_done = s->req_samples_done;
    st->flagged = s->flagged;
    st->chunk_latency_p50_us = percentile(cl, 0.5);
    st->chunk_latency_p99_us = percentile(cl, 0.99);
    st->chunk_latency_max_us = cl.empty() ? 0.0 : *std::max_element(cl.begin(), cl.end());
    st->request_latency_p50_us = percentile(rl, 0.5);
    st->request_latency_p99_us = percentile(rl, 0.99);
    st->wall_seconds = s->t_first < 0 ? 0.0 : std::max(0.0, s->t_last - s->t_first);
    st->gpu_busy_seconds = s->busy_s;
    st->arena_bytes = s->arena.size;
    st->arena_peak_bytes = s->arena.peak;
    st->device_status = (s->status & kStatusTimeout)       ? RFI_ERR_TIMEOUT
                        : (s->status & kStatusLayout)      ? RFI_ERR_UNSUPPORTED
                        : (s->status & kStatusSampleRange) ? RFI_ERR_SAMPLE_RANGE
                                                           : RFI_OK;
    return RFI_OK;
}

rfi_status rfi_server_destroy(rfi_server_t s) {
    if (!s) return RFI_OK;
    if (s->s_comp) cudaStreamSynchronize(s->s_comp);
    if (s->s_copy) cudaStreamSynchronize(s->s_copy);
    if (s->s_back) cudaStreamSynchronize(s->s_back);
    for (auto &ch : s->chunks)
        if (ch.ev) cudaEventDestroy(ch.ev);
    for (auto &ps : s->inflight) {
        if (ps.ev0) cudaEventDestroy(ps.ev0);
        if (ps.ev) cudaEventDestroy(ps.ev);
    }
    for (auto &rq : s->reqs) {
        if (rq.ev_submit) cudaEventDestroy(rq.ev_submit);
        if (rq.ev_done) cudaEventDestroy(rq.ev_done);
    }
    for (auto &sl : s->slots)
        if (sl.h_buf) cudaFreeHost(sl.h_buf);
    if (s->ev_copies) cudaEventDestroy(s->ev_copies);
    if (s->s_copy) cudaStreamDestroy(s->s_copy);
    if (s->s_comp) cudaStreamDestroy(s->s_comp);
    if (s->s_back) cudaStreamDestroy(s->s_back);
    if (s->arena.base) cudaFree(s->arena.base);
    cudaGetLastError();
    delete s;
    return RFI_OK;
}

}  // extern "C"
