// Synthetic antenna-voltage feed: Gaussian receiver noise plus impulsive broadband bursts
// plus an optional slow baseline drift, rounded and saturated to int8 or 12-bit samples.
//
// This module only MAKES inputs. It holds none of the excision method's arithmetic (no
// median, MAD, threshold, replacement or Philox) and is shared by the CPU oracle and the
// GPU path as their common input source.
//
// The feed stands in for the digitised baseband stream of one antenna polarisation
// (Section II-C: 400 MHz bandwidth sampled at the 800 MHz Nyquist rate). Broadband RFI is
// modelled after Section II-A: groups of strong impulses riding on Gaussian sky/receiver
// noise, and after the RFI emulator of Section III-B (a burst with a fixed on-period).
//
// Every sample is a pure function of (seed, stream, absolute sample index): any chunk
// [i0, i0+n) can be generated on its own and equals the same slice of the whole stream.
//
// Random numbers come from a counter-based hash: the SplitMix64 output function
// (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
// applied to a key derived from (seed, stream, domain) xor-ed with a counter.
//   domain 1: Gaussian noise (Box-Muller; two 53-bit uniforms per pair of samples)
//   domain 2: burst start (a burst starts at sample i with probability burst_rate:
//             a Bernoulli process, i.e. geometric gaps, the discrete Poisson process)
//   domain 3: burst length U{1..burst_len_max}
//   domain 4: burst amplitude U[amp_lo, amp_hi]*sigma and sign
//   domain 5: drift phase of the stream
// Sample value: x = sat(rint(sigma*z + drift + sum of bursts covering i)),
// rint = round half to even, sat = clamp to [-128,127] (8 bit) or [-2048,2047] (12 bit).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>
#include <algorithm>

extern "C" {

typedef struct {
    uint64_t seed;
    double sigma;          // noise standard deviation, LSB
    double burst_rate;     // probability that a burst starts at a given sample
    int32_t burst_len_max; // burst length is uniform on {1..burst_len_max}
    int32_t bits;          // 8 (int8 container) or 12 (int16 container)
    double amp_lo, amp_hi; // burst amplitude uniform on [amp_lo, amp_hi] * sigma
    double drift_amp;      // drift amplitude, LSB (0 = none)
    double drift_period;   // drift period, samples
} synth_params;

}  // extern "C"

namespace {

inline uint64_t sm64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

inline uint64_t domain_key(uint64_t seed, uint32_t stream, uint32_t domain) {
    return sm64(sm64(seed) ^ ((uint64_t)stream << 8 | (uint64_t)domain));
}

inline double u53(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }  // [0,1)

const double kTwoPi = 6.283185307179586476925286766559;

void fill_range(void *out, const synth_params *p, uint32_t stream, int64_t i0, int64_t n) {
    const uint64_t k_noise = domain_key(p->seed, stream, 1);
    const uint64_t k_start = domain_key(p->seed, stream, 2);
    const uint64_t k_len = domain_key(p->seed, stream, 3);
    const uint64_t k_amp = domain_key(p->seed, stream, 4);
    const double phase = kTwoPi * u53(sm64(domain_key(p->seed, stream, 5)));
    const int lmax = p->burst_len_max > 0 ? p->burst_len_max : 1;
    // burst starts at i iff hash < threshold; rate 0 disables bursts
    uint64_t thr = 0;
    if (p->burst_rate >= 1.0) thr = ~0ull;
    else if (p->burst_rate > 0.0) thr = (uint64_t)(p->burst_rate * 18446744073709551616.0);
    const int32_t lo = p->bits == 8 ? -128 : -2048, hi = p->bits == 8 ? 127 : 2047;

    const int64_t B = 4096;
    std::vector<double> acc(B);
    for (int64_t b0 = i0; b0 < i0 + n; b0 += B) {
        const int64_t m = std::min(B, i0 + n - b0);
        // Gaussian noise (Box-Muller on pairs (2j, 2j+1)) and drift
        for (int64_t t = 0; t < m; ++t) {
            const int64_t i = b0 + t;
            const uint64_t j = (uint64_t)i >> 1;
            const double u1 = 1.0 - u53(sm64(k_noise ^ (2 * j)));  // (0,1]
            const double u2 = u53(sm64(k_noise ^ (2 * j + 1)));
            const double r = std::sqrt(-2.0 * std::log(u1));
            const double z = (i & 1) ? r * std::sin(kTwoPi * u2) : r * std::cos(kTwoPi * u2);
            double v = p->sigma * z;
            if (p->drift_amp != 0.0)
                v += p->drift_amp * std::sin(kTwoPi * (double)i / p->drift_period + phase);
            acc[t] = v;
        }
        // bursts whose span [s, s+len) meets [b0, b0+m)
        if (thr) {
            const int64_t s_lo = std::max<int64_t>(0, b0 - lmax + 1);
            for (int64_t s = s_lo; s < b0 + m; ++s) {
                if (sm64(k_start ^ (uint64_t)s) >= thr) continue;
                const int64_t len = 1 + (int64_t)(u53(sm64(k_len ^ (uint64_t)s)) * lmax);
                if (s + len <= b0) continue;
                const uint64_t ha = sm64(k_amp ^ (uint64_t)s);
                const double a = (p->amp_lo + (p->amp_hi - p->amp_lo) * u53(ha)) * p->sigma;
                const double sa = (ha & 1) ? -a : a;
                const int64_t e = std::min(s + len, b0 + m);
                for (int64_t i = std::max(s, b0); i < e; ++i) acc[i - b0] += sa;
            }
        }
        for (int64_t t = 0; t < m; ++t) {
            double r = std::rint(acc[t]);
            int32_t x = r < lo ? lo : (r > hi ? hi : (int32_t)r);
            if (p->bits == 8) ((int8_t *)out)[b0 - i0 + t] = (int8_t)x;
            else ((int16_t *)out)[b0 - i0 + t] = (int16_t)x;
        }
    }
}

}  // namespace

extern "C" {

// Fill out[0..n) with samples i0..i0+n-1 of stream `stream`. Returns 0, or -1 on bad args.
int synth_fill(void *out, const synth_params *p, uint32_t stream, int64_t i0, int64_t n,
               int nthreads) {
    if (!out || !p || n < 0 || i0 < 0 || (p->bits != 8 && p->bits != 12)) return -1;
    if (p->drift_amp != 0.0 && !(p->drift_period > 0.0)) return -1;
    if (n == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    const int64_t min_part = 1 << 16;
    int64_t parts = std::min<int64_t>(nthreads, (n + min_part - 1) / min_part);
    if (parts <= 1) {
        fill_range(out, p, stream, i0, n);
        return 0;
    }
    const size_t es = p->bits == 8 ? 1 : 2;
    std::vector<std::thread> th;
    const int64_t per = (n + parts - 1) / parts;
    for (int64_t q = 0; q < parts; ++q) {
        const int64_t a = q * per, e = std::min(n, a + per);
        if (a >= e) break;
        th.emplace_back(fill_range, (char *)out + a * es, p, stream, i0 + a, e - a);
    }
    for (auto &t : th) t.join();
    return 0;
}

}  // extern "C"
