// CPU oracle for windowed median / MAD broadband RFI excision (Buch et al., "Implementing and
// Characterizing Real-time Broadband RFI Excision for the GMRT Wideband Backend", Section II-D).
//
// TEST INFRASTRUCTURE. This file is the slow, obviously-correct definition that the CUDA path
// is checked against. Only the test suite, the package smoke check and the benchmark's CPU
// baseline leg may load it. It shares no code, header, table or constant generator with the
// CUDA path; every value it uses it derives here, from the paper or from the readings listed
// below.
//
// What it computes, per non-overlapping data window of n samples (Section II-D), and the
// Median-of-MAD variant (Eq. 3, oracle_excise_mom) that replaces D by the median of the MADs of
// the last k_mom windows:
//   M = M(x)                      median of the window (std::sort, lower median s[(n-1)/2])
//   D = M(|x_i - M|)              median absolute deviation, same lower-median rule
//   tau_U = M + n_s*(1.4826*D)    Eq. 1 (n_s is the paper's threshold multiple "n")
//   tau_L = M - n_s*(1.4826*D)
//   z_i = K if x_i >= tau_U or x_i <= tau_L, else x_i      Eq. 2
// with the replacement K chosen among the options named in Section II-D: a constant (zero
// or a given value), the threshold itself, or digital noise.
//
// Readings where the paper is silent (each is also listed in the design notes):
//   * even n: lower median s[(n-1)/2], for M and for D alike.
//   * n_s*1.4826 is held in Q16 fixed point: Kq = floor(n_s*1.4826*65536 + 0.5), and the
//     comparisons of Eq. 2 are made exactly in integers: x*2^16 >= M*2^16 + Kq*D.
//   * D = 0: nothing is flagged (a constant window flags nothing).
//   * threshold replacement: tau rounded toward M (floor(tau_U) above, ceil(tau_L) below).
//   * digital noise: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed, counter
//     (idx_lo, idx_hi, stream_id, 0) with idx the absolute sample index in the stream; the
//     eight 16-bit halves u_j of the four outputs give S2 = 2*sum(u_j) - 8*65535, and the
//     replacement is M + round_half_away(S2 * 97164*D / (107020*65536)), i.e. an approximately
//     Gaussian value with standard deviation 1.4826*D centred on M.
//   * every replacement is saturated to the sample range ([-128,127] or [-2048,2047]).
//   * windows start at absolute sample 0 of the stream; the last window may be shorter.
//   * 12-bit input outside [-2048,2047] is an error (status 6).
//   * Eq. 3 (Median of MAD): the k successive windows are the k_mom windows ending at the
//     current one (causal, sliding by one window); at the start of a stream, the windows that
//     exist. Lower median of those MADs. The thresholds stay centred on the window's own
//     median; the MoM takes D's place in Eq. 1, in the threshold replacement and in the noise
//     spread, and a MoM of 0 flags nothing.
//
// Build: g++ -O2 -std=c++17 -fPIC -shared -pthread (see build.py in this directory).

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

namespace {

const int ORACLE_OK = 0;
const int ORACLE_BAD_ARG = 1;
const int ORACLE_SAMPLE_RANGE = 6;

// ---- Philox4x32-10, from its definition in Salmon, Moraes, Dror and Shaw, "Parallel random
// numbers: as easy as 1, 2, 3" (SC'11). Each round multiplies the even words by
// the two round multipliers, and the odd words are xor-ed with the high halves of those
// products and with the round key; the key is bumped by the two Weyl constants between rounds.
const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        const uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        const uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n1 = (uint32_t)p1;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        const uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

int64_t k_q16(double n_sigma) {
    // n*1.4826 in Q16, rounded half up (1.4826 as printed in Section II-D)
    const double v = n_sigma * 1.4826 * 65536.0;
    int64_t f = (int64_t)v;              // v > 0: truncation == floor
    if (v - (double)f >= 0.5) f += 1;
    return f;
}

int64_t floor_div(int64_t a, int64_t b) {  // b > 0
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

int32_t sat(int64_t v, int32_t lo, int32_t hi) { return v < lo ? lo : (v > hi ? hi : (int32_t)v); }

// Digital-noise replacement value for absolute sample idx of stream stream_id.
int32_t noise_value(int32_t M, int32_t D, uint64_t seed, uint32_t stream_id, int64_t idx,
                    int32_t lo, int32_t hi) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t ctr[4] = {(uint32_t)(uint64_t)idx, (uint32_t)((uint64_t)idx >> 32), stream_id, 0u};
    uint32_t r[4];
    philox4x32_10(ctr, key, r);
    int64_t sum_u = 0;
    for (int w = 0; w < 4; ++w) sum_u += (int64_t)(r[w] & 0xFFFFu) + (int64_t)(r[w] >> 16);
    const int64_t S2 = 2 * sum_u - 8 * 65535;           // zero mean, sd 107019.84
    const int64_t sigma_q16 = 97164LL * D;                // round(1.4826*65536) * D
    const int64_t num = S2 * sigma_q16;
    const int64_t den = 107020LL * 65536LL;
    const int64_t mag = ((num < 0 ? -num : num) + den / 2) / den;  // round half away from zero
    const int64_t off = num < 0 ? -mag : mag;
    return sat((int64_t)M + off, lo, hi);
}

int32_t lower_median(std::vector<int32_t> v) {
    std::sort(v.begin(), v.end());
    return v[(v.size() - 1) / 2];
}

struct Job {
    const void *x;
    void *z;
    int32_t bits;
    int64_t len;
    int32_t W;
    int64_t abs0;
    int64_t Kq;
    int32_t mode;
    int32_t const_value;
    uint64_t seed;
    uint32_t stream_id;
    uint32_t *mask;
    uint32_t *counts;
    int32_t *median;
    int32_t *mad;
};

int32_t load(const Job &j, int64_t i) {
    return j.bits == 8 ? (int32_t)((const int8_t *)j.x)[i] : (int32_t)((const int16_t *)j.x)[i];
}

void store(const Job &j, int64_t i, int32_t v) {
    if (j.bits == 8) ((int8_t *)j.z)[i] = (int8_t)v;
    else ((int16_t *)j.z)[i] = (int16_t)v;
}

// Samples of window w (samples [s0, s0+n) of the call); false if a 12-bit sample is out of range.
bool window_samples(const Job &j, int64_t w, std::vector<int32_t> &x) {
    const int32_t lo = j.bits == 8 ? -128 : -2048, hi = j.bits == 8 ? 127 : 2047;
    const int64_t s0 = w * (int64_t)j.W;
    const int64_t n = std::min<int64_t>(j.W, j.len - s0);
    x.resize(n);
    for (int64_t i = 0; i < n; ++i) {
        x[i] = load(j, s0 + i);
        if (x[i] < lo || x[i] > hi) return false;
    }
    return true;
}

// Robust estimation of one window (Section II-D): its median M and median absolute deviation D.
void window_stats(const std::vector<int32_t> &x, int32_t *M, int32_t *D) {
    const int32_t m = lower_median(x);
    std::vector<int32_t> dev(x.size());
    for (size_t i = 0; i < x.size(); ++i) dev[i] = x[i] > m ? x[i] - m : m - x[i];
    *M = m;
    *D = lower_median(dev);
}

// Threshold detection and filtering of window w (Eq. 1, Eq. 2) around centre M with dispersion D.
void apply_window(const Job &j, int64_t w, const std::vector<int32_t> &x, int32_t M, int32_t D);

// One data window: samples [s0, s0+n) of the call; window number w.
int excise_window(const Job &j, int64_t w) {
    std::vector<int32_t> x;
    if (!window_samples(j, w, x)) return ORACLE_SAMPLE_RANGE;
    int32_t M, D;
    window_stats(x, &M, &D);
    apply_window(j, w, x, M, D);
    if (j.median) j.median[w] = M;
    if (j.mad) j.mad[w] = D;
    return ORACLE_OK;
}

void apply_window(const Job &j, int64_t w, const std::vector<int32_t> &x, int32_t M, int32_t D) {
    const int32_t lo = j.bits == 8 ? -128 : -2048, hi = j.bits == 8 ? 127 : 2047;
    const int64_t s0 = w * (int64_t)j.W;
    const int64_t n = (int64_t)x.size();
    // Eq. 1 in Q16: tau_U = M + Kq*D/2^16, tau_L = M - Kq*D/2^16
    const int64_t tauU_q = (int64_t)M * 65536 + j.Kq * D;
    const int64_t tauL_q = (int64_t)M * 65536 - j.Kq * D;
    const int64_t words = (j.W + 31) / 32;
    uint32_t *mk = j.mask ? j.mask + w * words : nullptr;
    if (mk) std::memset(mk, 0, sizeof(uint32_t) * words);
    uint32_t flagged = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t xq = (int64_t)x[i] * 65536;
        // Eq. 2 (inclusive comparisons); D = 0 flags nothing
        const bool above = xq >= tauU_q, below = xq <= tauL_q;
        int32_t out = x[i];
        if (D > 0 && (above || below)) {
            ++flagged;
            if (mk) mk[i / 32] |= 1u << (i % 32);
            switch (j.mode) {
                case 0: out = 0; break;                                  // zero (blanking)
                case 1: out = sat(j.const_value, lo, hi); break;         // constant
                case 2:                                                  // threshold
                    out = above ? sat(floor_div(tauU_q, 65536), lo, hi)
                                : sat(-floor_div(-tauL_q, 65536), lo, hi);
                    break;
                default:                                                 // digital noise
                    out = noise_value(M, D, j.seed, j.stream_id, j.abs0 + s0 + i, lo, hi);
            }
        }
        store(j, s0 + i, out);
    }
    if (j.counts) j.counts[w] = flagged;
}

// Run f(w) for windows 0..nw-1 on nt threads (interleaved); returns the first non-OK status.
template <class F>
int for_windows(int64_t nw, int32_t nthreads, F f) {
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(nthreads, nw));
    std::vector<int> status(nt, ORACLE_OK);
    auto worker = [&](int t) {
        for (int64_t w = t; w < nw; w += nt) {
            const int s = f(w);
            if (s != ORACLE_OK) status[t] = s;
        }
    };
    if (nt == 1) {
        worker(0);
    } else {
        std::vector<std::thread> th;
        for (int t = 0; t < nt; ++t) th.emplace_back(worker, t);
        for (auto &t : th) t.join();
    }
    for (int s : status)
        if (s != ORACLE_OK) return s;
    return ORACLE_OK;
}

}  // namespace

extern "C" {

typedef struct {
    const void *x;        // input samples: int8 (bits 8) or int16 holding 12-bit values
    void *z;              // output samples, same type; may equal x
    int32_t bits;         // 8 or 12
    int64_t len;          // samples in x
    int32_t W;            // window length, 1..65536
    int64_t abs0;         // absolute stream index of x[0]; a multiple of W
    double n_sigma;       // threshold multiple (the paper's n)
    int32_t mode;         // 0 zero, 1 constant, 2 threshold, 3 digital noise
    int32_t const_value;  // constant replacement value (saturated)
    uint64_t seed;        // digital-noise seed
    uint32_t stream_id;   // digital-noise stream id
    uint32_t *mask;       // nullable: ceil(W/32) words per window, bit i = sample i of the window
    uint32_t *counts;     // nullable: flagged samples per window
    int32_t *median;      // nullable: M per window
    int32_t *mad;         // nullable: D per window
    int32_t nthreads;     // worker threads (>= 1)
} oracle_args;

int64_t oracle_k_q16(double n_sigma) { return k_q16(n_sigma); }

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    philox4x32_10(ctr, key, out);
}

int32_t oracle_noise_value(int32_t M, int32_t D, uint64_t seed, uint32_t stream_id, int64_t idx,
                           int32_t bits) {
    return noise_value(M, D, seed, stream_id, idx, bits == 8 ? -128 : -2048, bits == 8 ? 127 : 2047);
}

// Median and MAD of one window of int32 values (no range limit).
void oracle_median_mad(const int32_t *x, int64_t n, int32_t *M, int32_t *D) {
    std::vector<int32_t> v(x, x + n);
    const int32_t m = lower_median(v);
    for (auto &e : v) e = e > m ? e - m : m - e;
    *M = m;
    *D = lower_median(v);
}

int oracle_excise(const oracle_args *a) {
    if (!a || !a->x || !a->z || (a->bits != 8 && a->bits != 12) || a->len < 1 || a->W < 1 ||
        a->W > 65536 || a->abs0 < 0 || (a->abs0 % a->W) != 0 || !(a->n_sigma > 0.0) ||
        a->mode < 0 || a->mode > 3)
        return ORACLE_BAD_ARG;
    Job j{a->x, a->z, a->bits, a->len, a->W, a->abs0, k_q16(a->n_sigma), a->mode, a->const_value,
          a->seed, a->stream_id, a->mask, a->counts, a->median, a->mad};
    if (j.Kq < 1) return ORACLE_BAD_ARG;
    const int64_t nw = (a->len + a->W - 1) / a->W;
    return for_windows(nw, a->nthreads, [&](int64_t w) { return excise_window(j, w); });
}

// Median of MAD (Eq. 3): the dispersion of window j is the lower median of the MADs of the
// k_mom successive windows ending at j, D_{j-k_mom+1} .. D_j; windows before the first one of
// the stream do not exist, so early windows take the median of the MADs there are. The
// thresholds (Eq. 1) are then set around the window's own median M_j with that dispersion, and
// Eq. 2 and the replacement options apply unchanged. history holds the MADs of the n_history
// windows just before x (oldest first, n_history <= k_mom - 1), so a stream excised in slices
// equals the whole stream; mom (nullable) receives the dispersion used per window.
int oracle_excise_mom(const oracle_args *a, int32_t k_mom, const int32_t *history, int64_t n_history,
                      int32_t *mom) {
    if (!a || !a->x || !a->z || (a->bits != 8 && a->bits != 12) || a->len < 1 || a->W < 1 ||
        a->W > 65536 || a->abs0 < 0 || (a->abs0 % a->W) != 0 || !(a->n_sigma > 0.0) ||
        a->mode < 0 || a->mode > 3 || k_mom < 1 || n_history < 0 || n_history > k_mom - 1 ||
        (n_history > 0 && !history))
        return ORACLE_BAD_ARG;
    Job j{a->x, a->z, a->bits, a->len, a->W, a->abs0, k_q16(a->n_sigma), a->mode, a->const_value,
          a->seed, a->stream_id, a->mask, a->counts, a->median, a->mad};
    if (j.Kq < 1) return ORACLE_BAD_ARG;
    const int64_t nw = (a->len + a->W - 1) / a->W;
    // 1. M_j and D_j of every window
    std::vector<int32_t> M(nw), D(n_history + nw);
    for (int64_t i = 0; i < n_history; ++i) D[i] = history[i];
    int st = for_windows(nw, a->nthreads, [&](int64_t w) {
        std::vector<int32_t> x;
        if (!window_samples(j, w, x)) return ORACLE_SAMPLE_RANGE;
        window_stats(x, &M[w], &D[n_history + w]);
        return ORACLE_OK;
    });
    if (st != ORACLE_OK) return st;
    // 2. Eq. 3: M_m = M(D_{j-k+1}, ..., D_j), lower median, over the windows that exist
    std::vector<int32_t> Mm(nw);
    for_windows(nw, a->nthreads, [&](int64_t w) {
        const int64_t end = n_history + w + 1;
        const int64_t begin = std::max<int64_t>(0, end - k_mom);
        Mm[w] = lower_median(std::vector<int32_t>(D.begin() + begin, D.begin() + end));
        return ORACLE_OK;
    });
    // 3. Eq. 1 and Eq. 2 around M_j with dispersion M_m
    return for_windows(nw, a->nthreads, [&](int64_t w) {
        std::vector<int32_t> x;
        window_samples(j, w, x);
        apply_window(j, w, x, M[w], Mm[w]);
        if (j.median) j.median[w] = M[w];
        if (j.mad) j.mad[w] = D[n_history + w];
        if (mom) mom[w] = Mm[w];
        return ORACLE_OK;
    });
}

}  // extern "C"
