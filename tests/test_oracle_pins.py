"""Pins for the CPU oracle: checks against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: the rank definition of the median
(brute force), library order statistics, hand-derived worked windows and thresholds
(tests/golden), invariants of the definition, the closed-form flag probability of a rounded
Gaussian, the 50 % breakdown point of the MAD, and cuRAND's Philox4_32_10 generator.
"""
import ctypes
import ctypes.util
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODES = {"zero": oracle.ZERO, "const": oracle.CONST, "clip": oracle.CLIP, "noise": oracle.NOISE}


# ---------------------------------------------------------------- median and MAD
def rank_lower_median(vals):
    """Smallest v with #{x <= v} >= ceil(n/2): the lower median by its rank definition."""
    need = (len(vals) + 1) // 2
    v = min(vals)
    while sum(1 for x in vals if x <= v) < need:
        v += 1
    return v


def brute_median_mad(vals):
    M = rank_lower_median(vals)
    return M, rank_lower_median([abs(x - M) for x in vals])


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_median_mad_exhaustive_small_alphabet(n):
    # every window of length n over {-3..3} (Section II-D robust estimation, by rank counting)
    for w in itertools.product(range(-3, 4), repeat=n):
        assert oracle.median_mad(w) == brute_median_mad(list(w)), w


def test_median_mad_against_library_order_statistics():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    for trial in range(400):
        n = int(rng.integers(1, 65))
        lo, hi = (-128, 127) if trial % 2 == 0 else (-2048, 2047)
        x = rng.integers(lo, hi + 1, size=n)
        if trial % 5 == 0:  # heavy ties
            x = rng.integers(-2, 3, size=n)
        M, D = oracle.median_mad(x)
        r = (n - 1) // 2
        assert M == int(np.partition(x, r)[r])
        assert M == int(torch.median(torch.from_numpy(x)).item())  # torch: lower median
        dev = np.abs(x - M)
        assert D == int(np.partition(dev, r)[r])
        assert D == int(torch.median(torch.from_numpy(dev)).item())


def test_median_mad_invariants():
    rng = np.random.default_rng(12)
    for _ in range(200):
        n = int(rng.integers(1, 200)) | 1  # odd n for the negation invariant
        x = rng.integers(-60, 61, size=n)
        M, D = oracle.median_mad(x)
        assert oracle.median_mad(rng.permutation(x)) == (M, D)          # permutation
        c = int(rng.integers(-40, 41))
        assert oracle.median_mad(x + c) == (M + c, D)                    # shift by c
        assert oracle.median_mad(-x) == (-M, D)                          # negation (odd n)


# ---------------------------------------------------------------- threshold (Eq. 1)
def load_threshold_golden():
    rows = []
    for line in open(os.path.join(GOLDEN, "threshold_q16.txt")):
        if line.strip() and not line.startswith("#"):
            k, kq, d, t, c = line.split()
            rows.append((float(k), int(kq), int(d), int(t), int(c)))
    return rows


@pytest.mark.parametrize("row", load_threshold_golden())
def test_threshold_golden(row):
    k, kq, D, t, c = row
    assert oracle.k_q16(k) == kq
    # a window with median 0 and MAD exactly D: 5 zeros, 2 samples at +-D, then probes at
    # distances t-1 and t above and below; probes are a minority so M and D stay put
    M0 = 0
    bits = 12 if t > 120 else 8
    base = [0] * 9 + [D, -D, D, -D, D, -D, D, -D]
    probes = [t - 1, -(t - 1), t, -t]
    x = np.array(base + probes, dtype=np.int8 if bits == 8 else np.int16)
    assert oracle.median_mad(x) == (M0, D)
    r = oracle.excise(x, x.size, k, oracle.CLIP, bits=bits)
    assert r["status"] == 0 and r["median"][0] == M0 and r["mad"][0] == D
    z = r["z"].astype(int)
    nb = len(base)
    # |x - M| = t-1 is inside the thresholds, |x - M| = t is outside (Eq. 2, inclusive)
    assert list(z[nb:]) == [t - 1, -(t - 1), c, -c]
    assert r["counts"][0] == 2


def load_windows_golden():
    rows = []
    for line in open(os.path.join(GOLDEN, "windows.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        f = [s.strip() for s in line.split("|")]
        rows.append(dict(name=f[0], bits=int(f[1]), k=float(f[2]), mode=MODES[f[3]],
                         const=int(f[4]), x=[int(v) for v in f[5].split()], M=int(f[6]),
                         D=int(f[7]), flags=[int(v) for v in f[8].split()],
                         z=[int(v) for v in f[9].split()]))
    return rows


@pytest.mark.parametrize("g", load_windows_golden(), ids=lambda g: g["name"])
def test_worked_windows(g):
    x = np.array(g["x"], dtype=np.int8 if g["bits"] == 8 else np.int16)
    r = oracle.excise(x, x.size, g["k"], g["mode"], const=g["const"], bits=g["bits"])
    assert r["status"] == 0
    assert (r["median"][0], r["mad"][0]) == (g["M"], g["D"])
    assert list(r["z"].astype(int)) == g["z"]
    bits = [i for i in range(x.size) if (int(r["mask"][i // 32]) >> (i % 32)) & 1]
    assert bits == g["flags"]
    assert r["counts"][0] == len(g["flags"])


def test_eq2_against_real_valued_threshold():
    # Eq. 1 and Eq. 2 evaluated with the real multiple k*1.4826 (no fixed point), on windows
    # where no threshold lies within 1e-3 of an integer; the Q16 reading must flag the same.
    rng = np.random.default_rng(13)
    checked = 0
    for _ in range(300):
        n = int(rng.integers(8, 300))
        x = np.clip(np.rint(rng.normal(0, rng.uniform(2, 30), size=n)), -128, 127).astype(np.int8)
        x[rng.integers(0, n, size=max(1, n // 20))] = rng.integers(-128, 128)
        k = float(rng.choice([2.0, 2.5, 3.0, 3.5, 5.0]))
        r = oracle.excise(x, n, k, oracle.ZERO)
        M, D = int(r["median"][0]), int(r["mad"][0])
        if D == 0:
            assert r["counts"][0] == 0
            continue
        off = k * 1.4826 * D
        if abs(off - round(off)) < 1e-3:
            continue
        tauU, tauL = M + off, M - off
        flags = [(v >= tauU or v <= tauL) for v in x.astype(int)]
        got = [bool((int(r["mask"][i // 32]) >> (i % 32)) & 1) for i in range(n)]
        assert got == flags
        checked += 1
    assert checked > 200


def test_shift_and_permutation_invariance_of_flags():
    rng = np.random.default_rng(14)
    for _ in range(100):
        n = int(rng.integers(16, 400))
        x = np.clip(np.rint(rng.normal(0, 8, size=n)), -60, 60).astype(np.int8)
        x[rng.integers(0, n, size=n // 10)] = rng.integers(-60, 61)
        r = oracle.excise(x, n, 3.0, oracle.ZERO)
        flag = np.array([(int(r["mask"][i // 32]) >> (i % 32)) & 1 for i in range(n)])
        c = int(rng.integers(-50, 51))
        rs = oracle.excise((x.astype(int) + c).astype(np.int8), n, 3.0, oracle.ZERO)
        assert rs["median"][0] == r["median"][0] + c and rs["mad"][0] == r["mad"][0]
        flag_s = np.array([(int(rs["mask"][i // 32]) >> (i % 32)) & 1 for i in range(n)])
        assert (flag_s == flag).all()
        p = rng.permutation(n)
        rp = oracle.excise(x[p], n, 3.0, oracle.ZERO)
        flag_p = np.array([(int(rp["mask"][i // 32]) >> (i % 32)) & 1 for i in range(n)])
        assert (flag_p == flag[p]).all() and (rp["z"] == r["z"][p]).all()
        assert rp["counts"][0] == r["counts"][0]


def test_constant_window_flags_nothing():
    for v in (-128, -1, 0, 77, 127):
        for n in (1, 2, 31, 4096):
            x = np.full(n, v, np.int8)
            r = oracle.excise(x, n, 3.0, oracle.ZERO)
            assert r["counts"][0] == 0 and (r["z"] == x).all() and r["mad"][0] == 0


# ---------------------------------------------------------------- flag statistics
def _phi(z):
    return 0.5 * math.erfc(-z / math.sqrt(2.0))


def test_gaussian_flag_fraction_matches_discretised_closed_form():
    """Clean rounded Gaussian (sigma 16, int8): the flag count agrees with the exact
    expectation for each window's (M, D) within 5 binomial standard deviations."""
    sigma, W, k = 16.0, 4096, 3.0
    p = synth.params(seed=101, sigma=sigma, burst_rate=0.0, burst_len_max=1, bits=8)
    x = synth.fill(p, 0, 1 << 20)
    r = oracle.excise(x, W, k, oracle.ZERO, threads=os.cpu_count() or 1)
    vals = np.arange(-128, 128)
    pmf = np.array([_phi((v + 0.5) / sigma) - _phi((v - 0.5) / sigma) for v in vals])
    pmf[0] = _phi(-127.5 / sigma)
    pmf[-1] = 1.0 - _phi(126.5 / sigma)
    E = V = 0.0
    for w in range(len(r["counts"])):
        M, D = int(r["median"][w]), int(r["mad"][w])
        off = k * 1.4826 * D          # Eq. 1 with the real multiple
        pw = pmf[(vals >= M + off) | (vals <= M - off)].sum()
        E += W * pw
        V += W * pw * (1 - pw)
    flags = int(r["counts"].sum())
    assert abs(flags - E) <= 5 * math.sqrt(V), (flags, E, math.sqrt(V))
    # the raw fraction sits about 10 % under 2Q(k) because the samples are integers
    frac, two_q = flags / x.size, 2 * (1 - _phi(k))
    assert 0.80 * two_q < frac < 0.98 * two_q


@pytest.mark.parametrize("f,flagged", [(0.1, True), (0.25, True), (0.4, True),
                                       (0.6, False), (0.75, False)])
def test_mad_breakdown_point(f, flagged):
    """Section II-D: the MAD is robust up to 50 % RFI in a window. A contiguous burst covering
    a fraction f < 0.5 is excised in full; beyond 0.5 the median moves into the burst and the
    burst is kept."""
    W = 4096
    p = synth.params(seed=102, sigma=4.0, burst_rate=0.0, burst_len_max=1, bits=8)
    x = synth.fill(p, 0, W).astype(np.int16)
    nb = int(f * W)
    x[100:100 + nb] += 100
    x = np.clip(x, -128, 127).astype(np.int8)
    r = oracle.excise(x, W, 3.0, oracle.ZERO)
    burst_flags = [(int(r["mask"][i // 32]) >> (i % 32)) & 1 for i in range(100, 100 + nb)]
    if flagged:
        assert all(burst_flags) and abs(int(r["median"][0])) < 10
    else:
        # the median sits inside the burst; the burst is kept (only its own noise tail can
        # cross the narrow threshold) and the clean samples are excised instead
        assert int(r["median"][0]) > 80
        assert sum(burst_flags) <= 0.01 * nb
        assert int(r["counts"][0]) - sum(burst_flags) >= 0.9 * (W - nb)


# ---------------------------------------------------------------- layout, tails, errors
def test_mask_layout_partial_words_and_tail():
    rng = np.random.default_rng(15)
    W, n = 40, 40 * 5 + 17
    x = np.clip(np.rint(rng.normal(0, 5, size=n)), -128, 127).astype(np.int8)
    x[rng.integers(0, n, size=20)] = 120
    r = oracle.excise(x, W, 3.0, oracle.ZERO)
    assert r["mask"].size == 6 * 2 and r["counts"].size == 6
    for w in range(6):
        n_w = min(W, n - w * W)
        seg = x[w * W: w * W + n_w]
        M, D = oracle.median_mad(seg)
        assert (r["median"][w], r["mad"][w]) == (M, D)
        words = r["mask"][2 * w: 2 * w + 2]
        bits = [(int(words[i // 32]) >> (i % 32)) & 1 for i in range(64)]
        assert not any(bits[n_w:])     # padding bits stay clear
        zw = r["z"][w * W: w * W + n_w]
        for i in range(n_w):
            assert zw[i] == (0 if bits[i] else seg[i])
        assert r["counts"][w] == sum(bits)


def test_window_aligned_slice_equals_whole_stream():
    p = synth.params(seed=103, sigma=16.0, burst_rate=5e-3, burst_len_max=64, bits=8)
    x = synth.fill(p, 3, 9 * 256 + 100)
    full = oracle.excise(x, 256, 3.0, oracle.NOISE, seed=7, stream_id=3)
    a = 4 * 256
    part = oracle.excise(x[a:], 256, 3.0, oracle.NOISE, seed=7, stream_id=3, abs0=a)
    assert (part["z"] == full["z"][a:]).all()
    assert (part["counts"] == full["counts"][4:]).all()
    assert (part["mask"] == full["mask"][4 * 8:]).all()


def test_twelve_bit_range_error():
    x = np.zeros(64, np.int16)
    x[5] = 2048
    assert oracle.excise(x, 32, 3.0, oracle.ZERO, bits=12)["status"] == oracle.STATUS_SAMPLE_RANGE
    x[5] = -2049
    assert oracle.excise(x, 32, 3.0, oracle.ZERO, bits=12)["status"] == oracle.STATUS_SAMPLE_RANGE
    x[5] = -2048
    assert oracle.excise(x, 32, 3.0, oracle.ZERO, bits=12)["status"] == 0


def test_bad_arguments():
    x = np.zeros(8, np.int8)
    assert oracle.excise(x, 0, 3.0, oracle.ZERO)["status"] == oracle.STATUS_BAD_ARG
    assert oracle.excise(x, 65537, 3.0, oracle.ZERO)["status"] == oracle.STATUS_BAD_ARG
    assert oracle.excise(x, 8, 0.0, oracle.ZERO)["status"] == oracle.STATUS_BAD_ARG
    assert oracle.excise(x, 8, 3.0, 9)["status"] == oracle.STATUS_BAD_ARG
    assert oracle.excise(x, 8, 3.0, oracle.ZERO, abs0=3)["status"] == oracle.STATUS_BAD_ARG


# ---------------------------------------------------------------- digital noise
def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if path:
            try:
                return ctypes.CDLL(path)
            except OSError:
                pass
    return None


def test_philox_against_curand_host_generator():
    """cuRAND's host Philox4_32_10 generator emits block (x, j) = Philox(ctr=(x,0,j,0), key=seed)
    at output offset 4*(65536*x + j) (observed layout of its 65536 subsequences)."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not found")
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        for seed in (0, 7, 0x0123456789ABCDEF, 0xFFFFFFFF00000001):
            assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_uint64(seed)) == 0
            assert cr.curandSetGeneratorOffset(gen, ctypes.c_uint64(0)) == 0
            n = 4 * 65536 * 3
            buf = (ctypes.c_uint32 * n)()
            assert cr.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
            key = (seed & 0xFFFFFFFF, seed >> 32)
            for x in (0, 1, 2):
                for j in (0, 1, 2, 59, 1000, 65535):
                    o = 4 * (65536 * x + j)
                    assert oracle.philox4x32_10((x, 0, j, 0), key) == list(buf[o:o + 4]), (seed, x, j)
            # counter word 1 (idx_hi): offset 4*65536*2^32 carries into it
            assert cr.curandSetGeneratorOffset(gen, ctypes.c_uint64(4 * 65536 * (1 << 32))) == 0
            buf4 = (ctypes.c_uint32 * 4)()
            assert cr.curandGenerate(gen, buf4, ctypes.c_size_t(4)) == 0
            assert oracle.philox4x32_10((0, 1, 0, 0), key) == list(buf4)
    finally:
        cr.curandDestroyGenerator(gen)


def test_noise_distribution_moments_and_range():
    """The noise replacement is M + round(S2*1.4826*D/107020) with S2 a sum of 8 independent
    uniform 16-bit words, rescaled: mean 0, variance 8*(2^32-1)/3 (sd 107019.84), |S2| <= 524280."""
    D, N = 200, 100000
    vals = np.array([oracle.noise_value(0, D, 0x5EED, 9, i, bits=12) for i in range(N)], float)
    sd_expected = 1.4826 * D * math.sqrt(8 * (2 ** 32 - 1) / 3) / 107020
    assert abs(vals.mean()) < 5 * sd_expected / math.sqrt(N)
    assert abs(vals.std() / sd_expected - 1) < 0.015
    bound = math.floor(524280 * 97164 * D / (107020 * 65536) + 0.5)
    assert np.abs(vals).max() <= bound
    # symmetric, and lighter tails than a Gaussian (Irwin-Hall excess kurtosis -1.2/8)
    kurt = ((vals - vals.mean()) ** 4).mean() / vals.var() ** 2
    assert abs(kurt - (3 - 1.2 / 8)) < 0.06
    # keyed by (seed, stream, absolute index)
    assert oracle.noise_value(0, D, 0x5EED, 9, 5, 12) == oracle.noise_value(0, D, 0x5EED, 9, 5, 12)
    diff = sum(oracle.noise_value(0, D, 0x5EED, 9, i, 12) != oracle.noise_value(0, D, 0x5EED, 10, i, 12)
               for i in range(200))
    assert diff > 150


def test_noise_mode_uses_absolute_index_and_saturates():
    x = np.zeros(512, np.int8)
    x[::7] = 127
    x[3::11] = -128
    r = oracle.excise(x, 128, 2.0, oracle.NOISE, seed=42, stream_id=5, abs0=1024)
    for i in range(512):
        if (int(r["mask"][i // 32]) >> (i % 32)) & 1:
            w = i // 128
            want = oracle.noise_value(int(r["median"][w]), int(r["mad"][w]), 42, 5, 1024 + i, 8)
            assert int(r["z"][i]) == want
    # noise around a median near the top of the range saturates at 127: the int8 value is
    # the 12-bit (unsaturated here) value clamped to the int8 range
    y = (100 + (np.arange(256) % 28)).astype(np.int8)
    r2 = oracle.excise(y, 256, 0.01, oracle.NOISE, seed=1, stream_id=2)
    M, D = int(r2["median"][0]), int(r2["mad"][0])
    assert D > 0 and r2["counts"][0] > 200
    clamped = 0
    for i in range(256):
        if (int(r2["mask"][i // 32]) >> (i % 32)) & 1:
            raw = oracle.noise_value(M, D, 1, 2, i, 12)
            assert int(r2["z"][i]) == max(-128, min(127, raw))
            clamped += raw > 127
    assert clamped > 0


# ---------------------------------------------------------------- digital noise: worked values
def load_noise_golden():
    rows = []
    for line in open(os.path.join(GOLDEN, "noise.txt")):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows.append(dict(name=f[0], seed=int(f[1], 0), idx=int(f[2]), stream=int(f[3]), M=int(f[4]),
                             D=int(f[5]), bits=int(f[6]), r=[int(v, 0) for v in f[7:11]], sum_u=int(f[11]),
                             S2=int(f[12]), num=int(f[13]), q=int(f[14]), rem=int(f[15]), off=int(f[16]),
                             value=int(f[17])))
    return rows


NOISE_DEN = 107020 * 65536


@pytest.mark.parametrize("g", load_noise_golden(), ids=lambda g: g["name"])
def test_noise_golden(g):
    """Each row's worked steps hold together, its Philox words are cuRAND's (when the library is
    present) and the oracle's, and the oracle's replacement value is the worked value."""
    key = (g["seed"] & 0xFFFFFFFF, g["seed"] >> 32)
    ctr = (g["idx"] & 0xFFFFFFFF, g["idx"] >> 32, g["stream"], 0)
    assert oracle.philox4x32_10(ctr, key) == g["r"]
    cr = _curand()
    if cr is not None:
        gen = ctypes.c_void_p()
        assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0
        try:
            assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_uint64(g["seed"])) == 0
            block = 65536 * ctr[0] + g["stream"] + (65536 << 32) * ctr[1]
            assert cr.curandSetGeneratorOffset(gen, ctypes.c_uint64(4 * block)) == 0
            buf = (ctypes.c_uint32 * 4)()
            assert cr.curandGenerate(gen, buf, ctypes.c_size_t(4)) == 0
            assert list(buf) == g["r"]
        finally:
            cr.curandDestroyGenerator(gen)
    # the row's own arithmetic (steps 2-5 of the fixture header)
    assert sum((w & 0xFFFF) + (w >> 16) for w in g["r"]) == g["sum_u"]
    assert g["S2"] == 2 * g["sum_u"] - 8 * 65535
    assert g["num"] == g["S2"] * 97164 * g["D"]
    assert abs(g["num"]) == g["q"] * NOISE_DEN + g["rem"] and 0 <= g["rem"] < NOISE_DEN
    assert abs(g["off"]) == g["q"] + (1 if 2 * g["rem"] >= NOISE_DEN else 0)
    lo, hi = (-128, 127) if g["bits"] == 8 else (-2048, 2047)
    assert g["value"] == max(lo, min(hi, g["M"] + g["off"]))
    # the oracle
    assert oracle.noise_value(g["M"], g["D"], g["seed"], g["stream"], g["idx"], g["bits"]) == g["value"]


def _count_le(t):
    """#{(h_1..h_8) in [0, 65535]^8 : sum <= t}, by inclusion-exclusion over the halves that
    exceed their range (the distribution function of a sum of uniform 16-bit integers)."""
    if t < 0:
        return 0
    return sum((-1) ** j * math.comb(8, j) * math.comb(t - 65536 * j + 8, 8)
               for j in range(9) if t - 65536 * j >= 0)


def _exact_noise_pmf(D):
    """P(off = v) for a sample's noise offset at dispersion D, exactly, with S2 = 2*sum_u - 524280
    (sum_u a sum of eight uniform 16-bit halves) and off the value S2*97164*D/(107020*2^16)
    rounded half away from zero. Computed by locating where the offset steps in sum_u."""
    from fractions import Fraction

    def off(s):
        x = Fraction((2 * s - 524280) * 97164 * D, NOISE_DEN)
        m = abs(x)
        r = math.floor(m + Fraction(1, 2))
        return r if x >= 0 else -r

    lo_v, hi_v = off(0), off(524280)

    def first_s(v):  # smallest s with off(s) >= v (off is nondecreasing in s)
        a, b = 0, 524281
        while a < b:
            mid = (a + b) // 2
            if off(mid) >= v:
                b = mid
            else:
                a = mid + 1
        return a

    total = 65536 ** 8
    pmf = {}
    for v in range(lo_v, hi_v + 1):
        pmf[v] = Fraction(_count_le(first_s(v + 1) - 1) - _count_le(first_s(v) - 1), total)
    assert sum(pmf.values()) == 1
    return pmf


@pytest.mark.parametrize("D,N", [(1, 400000), (2, 200000), (3, 200000)])
def test_noise_exact_distribution_at_small_dispersion(D, N):
    """At D = 1..3 the noise offset takes a handful of values whose probabilities follow exactly
    from the Philox halves being uniform; the oracle's frequencies over N consecutive indices
    must match each within 5 binomial sd. Rounding down instead of to nearest moves P(0) from
    about 0.26 to about 0.5 at D = 1."""
    pmf = _exact_noise_pmf(D)
    vals = np.fromiter((oracle.noise_value(0, D, 0xD1CE, 3, i, 12) for i in range(N)), np.int64, N)
    seen = {int(v): int(c) for v, c in zip(*np.unique(vals, return_counts=True))}
    assert set(seen) <= set(pmf)
    for v, p in pmf.items():
        p = float(p)
        assert abs(seen.get(v, 0) - N * p) <= 5 * math.sqrt(N * p * (1 - p)) + 1, (D, v, seen.get(v, 0), N * p)
    # mean zero to within 0.01 LSB here; a one-sided rounding bias of 0.5 LSB would fail
    assert abs(vals.mean()) < 5 * vals.std() / math.sqrt(N)
