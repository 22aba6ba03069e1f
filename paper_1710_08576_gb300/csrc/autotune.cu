// Autotuner for the persistent kernel's launch shape: consumer warps per CTA, shared-memory
// stages, stage size (windows per tile), resident CTAs per SM, tile queue (atomic or static) and,
// for 12-bit samples, histogram copies. Every candidate that fits is timed with CUDA events on a
// scratch copy of the plan's own window layout (capped at 256 MiB of input) filled with
// noise-like samples; the fastest shape is kept. Results are cached per process by
// (device, sample width, mode, window layout), and in the file named by the environment
// variable RFI_TUNE_CACHE when it is set (one "key<TAB>shape" line per entry).

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "rfi.h"
#include "internal.h"
#include "plan_impl.h"

namespace rfi {

namespace {

constexpr int64_t kScratchBudget = 256ll << 20;

// Noise-like scratch samples: a sum of four hashed bytes (roughly Gaussian) scaled to the sample
// width's typical spread, plus rare large impulses; only the timing depends on these values.
__global__ void fill_scratch(uint8_t *buf, int64_t n, int bits) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint32_t h = static_cast<uint32_t>(i) * 2654435761u ^ static_cast<uint32_t>(i >> 32) * 2246822519u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        h *= 3266489917u;
        h ^= h >> 16;
        int v = static_cast<int>((h & 255u) + ((h >> 8) & 255u) + ((h >> 16) & 255u) + (h >> 24)) - 510;
        const bool burst = (h % 997u) < 3u;
        if (bits == 8) {
            v = v / 9 + (burst ? ((h & 1u) ? 100 : -100) : 0);
            buf[i] = static_cast<uint8_t>(static_cast<int8_t>(v < -128 ? -128 : (v > 127 ? 127 : v)));
        } else {
            v = (v * 4) / 5 + (burst ? ((h & 1u) ? 1500 : -1500) : 0);
            reinterpret_cast<int16_t *>(buf)[i] = static_cast<int16_t>(v < -2048 ? -2048 : (v > 2047 ? 2047 : v));
        }
    }
}

std::vector<Tile> tiles_for(int bits, const std::vector<int64_t> &len, const std::vector<int32_t> &W,
                            int stage_bytes) {
    const int bps = bits == 8 ? 1 : 2;
    std::vector<Tile> tiles;
    for (size_t i = 0; i < len.size(); ++i) {
        const int64_t wb = static_cast<int64_t>(W[i]) * bps;
        const int64_t per = (wb % 16 == 0) ? std::max<int64_t>(1, stage_bytes / wb) : 1;
        const int64_t nwin = (len[i] + W[i] - 1) / W[i];
        for (int64_t w0 = 0; w0 < nwin; w0 += per) {
            const int64_t nw = std::min<int64_t>(per, nwin - w0);
            const int64_t s1 = std::min<int64_t>(len[i], (w0 + nw) * W[i]);
            tiles.push_back(Tile{static_cast<uint32_t>(i), static_cast<uint32_t>(w0), static_cast<uint32_t>(nw),
                                 static_cast<uint32_t>((s1 - w0 * W[i]) * bps)});
        }
    }
    std::stable_sort(tiles.begin(), tiles.end(), [](const Tile &a, const Tile &b) { return a.bytes > b.bytes; });
    return tiles;
}

std::mutex g_cache_mu;
std::map<std::string, Shape> g_cache;

std::string cache_key(const rfi_plan_s *P) {
    cudaDeviceProp prop;
    std::string k;
    if (cudaGetDeviceProperties(&prop, P->device) == cudaSuccess) k = prop.name;
    char buf[96];
    std::snprintf(buf, sizeof(buf), "|%d|%d|%d|", P->bits, plan_kernel_mode(P), P->S);
    k += buf;
    for (int i = 0; i < P->S; ++i) {
        std::snprintf(buf, sizeof(buf), "%d:%lld,", P->W[i], static_cast<long long>(P->len[i] / P->W[i]));
        k += buf;
    }
    return k;
}

bool cache_file_lookup(const std::string &key, Shape *out) {
    const char *path = std::getenv("RFI_TUNE_CACHE");
    if (!path || !*path) return false;
    std::ifstream f(path);
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        const size_t tab = line.find('\t');
        if (tab == std::string::npos || line.compare(0, tab, key) != 0 || tab != key.size()) continue;
        std::istringstream is(line.substr(tab + 1));
        Shape s{};
        if (is >> s.consumer_warps >> s.stages >> s.ctas_per_sm >> s.stage_bytes >> s.dynamic_tiles >> s.hist_copies >>
            s.groups) {
            if (!(is >> s.warp_split)) s.warp_split = 1;  // entries written before the split-warp form
            *out = s;
            found = true;  // the last entry for a key wins
        }
    }
    return found;
}

void cache_file_store(const std::string &key, const Shape &s) {
    const char *path = std::getenv("RFI_TUNE_CACHE");
    if (!path || !*path) return;
    std::ofstream f(path, std::ios::app);
    f << key << '\t' << s.consumer_warps << ' ' << s.stages << ' ' << s.ctas_per_sm << ' ' << s.stage_bytes << ' '
      << s.dynamic_tiles << ' ' << s.hist_copies << ' ' << s.groups << ' ' << s.warp_split << '\n';
}

struct Scratch {
    uint8_t *in = nullptr, *out = nullptr;
    uint32_t *mask = nullptr, *counts = nullptr;
    int32_t *md = nullptr;
    Seg *segs = nullptr;
    Tile *tiles = nullptr;
    DevCounters *ctr = nullptr;
    ~Scratch() {
        cudaFree(in);
        cudaFree(out);
        cudaFree(mask);
        cudaFree(counts);
        cudaFree(md);
        cudaFree(segs);
        cudaFree(tiles);
        cudaFree(ctr);
    }
};

}  // namespace

rfi_status plan_autotune(rfi_plan_s *P, const rfi_launch_shape *req) {
    const std::string key = cache_key(P);
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        auto it = g_cache.find(key);
        Shape cached{};
        bool hit = it != g_cache.end();
        if (hit) cached = it->second;
        else if (cache_file_lookup(key, &cached)) {
            hit = persistent_occupancy(P->bits, plan_kernel_mode(P), cached) >= cached.ctas_per_sm;
            if (hit) g_cache[key] = cached;
        }
        if (hit) {
            P->shape = cached;
            rfi_status rs = plan_build_tiles(P);
            return rs == RFI_OK ? plan_alloc_workspace(P) : rs;
        }
    }
    const int bps = P->bits == 8 ? 1 : 2;
    // scratch layout: every stream, each cut to an equal share of the budget (whole windows,
    // at least one window)
    const int64_t share = std::max<int64_t>(1, kScratchBudget / bps / P->S);
    std::vector<int64_t> slen(P->S), soff(P->S);
    std::vector<int64_t> mwoff(P->S), woff(P->S);
    int64_t tot = 0, totw = 0, totmw = 0;
    for (int i = 0; i < P->S; ++i) {
        const int64_t nw = std::max<int64_t>(1, std::min<int64_t>(P->nwin[i], share / P->W[i]));
        slen[i] = std::min<int64_t>(P->len[i], nw * P->W[i]);
        soff[i] = tot;
        woff[i] = totw;
        mwoff[i] = totmw;
        tot += (slen[i] * bps + 255) / 256 * 256;
        totw += nw;
        totmw += nw * ((P->W[i] + 31) / 32);
    }
    Scratch sc;
    if (cudaMalloc(&sc.in, tot) != cudaSuccess || cudaMalloc(&sc.out, tot) != cudaSuccess ||
        cudaMalloc(&sc.mask, totmw * 4) != cudaSuccess || cudaMalloc(&sc.counts, totw * 4) != cudaSuccess ||
        cudaMalloc(&sc.md, totw * 8) != cudaSuccess || cudaMalloc(&sc.segs, sizeof(Seg) * P->S) != cudaSuccess ||
        cudaMalloc(&sc.ctr, sizeof(DevCounters)) != cudaSuccess) {
        cudaGetLastError();
        return RFI_ERR_OOM;
    }
    fill_scratch<<<1024, 256>>>(sc.in, tot / bps, P->bits);
    if (cudaStreamSynchronize(0) != cudaSuccess) return RFI_ERR_CUDA;
    std::vector<Seg> segs(P->S);
    for (int i = 0; i < P->S; ++i) {
        Seg &g = segs[i];
        std::memset(&g, 0, sizeof(g));
        g.in = sc.in + soff[i];
        g.out = sc.out + soff[i];
        g.mask = sc.mask + mwoff[i];
        g.counts = sc.counts + woff[i];
        g.med = sc.md + woff[i];
        g.mad = sc.md + totw + woff[i];
        g.len = slen[i];
        g.W = P->W[i];
        g.stream_id = P->sid[i];
        g.mask_words = (P->W[i] + 31) / 32;
        g.vec = (static_cast<int64_t>(P->W[i]) * bps) % 16 == 0;
    }
    if (cudaMemcpy(sc.segs, segs.data(), sizeof(Seg) * P->S, cudaMemcpyHostToDevice) != cudaSuccess)
        return RFI_ERR_CUDA;

    // candidate shapes
    int64_t maxwb = 0;
    bool uniform = true;
    for (int i = 0; i < P->S; ++i) {
        maxwb = std::max<int64_t>(maxwb, std::min<int64_t>(P->W[i], P->len[i]) * bps);
        uniform = uniform && P->W[i] == P->W[0];
    }
    const int min_stage = static_cast<int>((maxwb + 127) / 128 * 128);
    std::vector<Shape> cands;
    for (int cw : {4, 8, 16})
      for (int grp : {1, 2})
        for (int ctas : {1, 2, 3, 4})
            for (int stages : {1, 2, 3, 4, 6})
                for (int mult : {1, 2, 4})
                    for (int dyn : {1, 2})
                        for (int hc : {1, 2, 4})
                        for (int ws : {1, 2}) {
                            if (P->bits == 8 && hc != 1) continue;
                            if (!uniform && dyn == 2) continue;
                            if (grp == 2 && cw == 16) continue;
                            Shape s{cw, stages, ctas, min_stage * mult, dyn, P->bits == 8 ? 1 : hc, grp, ws};
                            if (ws == 2 && !plan_warp_split_runs(P, s)) continue;
                            if (req && req->warp_split && req->warp_split != ws) continue;
                            if (req) {
                                if (req->consumer_warps && req->consumer_warps != cw) continue;
                                if (req->stages && req->stages != stages) continue;
                                if (req->ctas_per_sm && req->ctas_per_sm != ctas) continue;
                                if (req->dynamic_tiles && req->dynamic_tiles != dyn) continue;
                                if (req->hist_copies && P->bits == 12 && req->hist_copies != hc) continue;
                                if (req->stage_bytes && req->stage_bytes != s.stage_bytes) continue;
                                if (req->groups && req->groups != grp) continue;
                            }
                            if (s.stage_bytes > 96 * 1024 && mult > 1) continue;
                            if (grp * (cw + 1) * 32 * ctas > 2048) continue;
                            if (persistent_smem_bytes(P->bits, plan_kernel_mode(P), s) * ctas > 228u * 1024u) continue;
                            cands.push_back(s);
                        }
    if (cands.empty()) return RFI_ERR_UNSUPPORTED;

    cudaStream_t st;
    cudaEvent_t e0, e1;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return RFI_ERR_CUDA;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Params p{};
    p.kq = P->kq;
    p.seed = P->seed;
    p.cval = P->cval;
    p.status = &sc.ctr->status;
    p.flagged = &sc.ctr->flagged;
    set_round_keys(p);
    Shape best{};
    float best_ms = 1e30f;
    std::vector<Tile> cur;
    int cur_stage = -1;
    for (const Shape &s : cands) {
        if (persistent_occupancy(P->bits, plan_kernel_mode(P), s) < s.ctas_per_sm) {
            cudaGetLastError();
            continue;
        }
        if (s.stage_bytes != cur_stage) {
            cur = tiles_for(P->bits, slen, P->W, s.stage_bytes);
            cudaFree(sc.tiles);
            sc.tiles = nullptr;
            if (cudaMalloc(&sc.tiles, sizeof(Tile) * cur.size()) != cudaSuccess ||
                cudaMemcpy(sc.tiles, cur.data(), sizeof(Tile) * cur.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cur_stage = s.stage_bytes;
        }
        p.ncopies = s.hist_copies;
        const int nt = static_cast<int>(cur.size());
        const int grid = std::max(1, std::min(nt, P->sm_count * s.ctas_per_sm));
        float ms_min = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 4 && ok; ++rep) {
            ok = cudaMemsetAsync(sc.ctr, 0, sizeof(DevCounters), st) == cudaSuccess;
            ok = ok && cudaEventRecord(e0, st) == cudaSuccess;
            ok = ok && launch_persistent(P->bits, plan_kernel_mode(P), s, grid, sc.segs, sc.tiles, nt, p, &sc.ctr->tile_counter,
                                         0, st) == cudaSuccess;
            ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0;
            if (ok && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ms_min = std::min(ms_min, ms);
        }
        if (!ok) {
            cudaGetLastError();
            continue;
        }
        if (ms_min < best_ms) {
            best_ms = ms_min;
            best = s;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (best_ms >= 1e29f) return RFI_ERR_UNSUPPORTED;
    P->shape = best;
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        g_cache[key] = best;
        cache_file_store(key, best);
    }
    rfi_status rs = plan_build_tiles(P);
    return rs == RFI_OK ? plan_alloc_workspace(P) : rs;
}

}  // namespace rfi
