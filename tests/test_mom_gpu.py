"""Median-of-MAD plans (Eq. 3) on the GPU against the oracle, bit for bit.

A MoM plan runs three kernels per call: the persistent kernel in its estimation-only mode (M and
D of every window), the sliding lower median of the last k_mom MADs of each stream, and the
persistent kernel in its apply mode (Eq. 1 and Eq. 2 around each window's M with its MoM). Every
output is compared with oracle.excise_mom: samples, mask, counts, M, D and the MoM itself.
"""
import os
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _streams(bits, lens, seed):
    if bits == 8:
        p = synth.params(seed=seed, sigma=16.0, burst_rate=3e-3, burst_len_max=4096, bits=8, amp=(2.0, 6.0))
    else:
        p = synth.params(seed=seed, sigma=120.0, burst_rate=3e-3, burst_len_max=2048, bits=12,
                         amp=(2.0, 8.0), drift_amp=50.0)
    return [synth.fill(p, s, n) for s, n in enumerate(lens)]


def _gpu(rfi, xs, windows, bits, k, mode, kmom, const=0, seed=0, flags=0, sids=None):
    import torch
    plan = rfi.Plan(bits, [x.size for x in xs], windows, k, mode, const, seed, flags, sids, mom_windows=kmom)
    try:
        nwin = plan.num_windows
        ins = [torch.from_numpy(x).cuda() for x in xs]
        outs = [torch.full_like(t, 55) for t in ins]
        masks = [torch.full((plan.mask_words(i),), -1, dtype=torch.int32, device="cuda") for i in range(len(xs))]
        counts = [torch.full((n,), -1, dtype=torch.int32, device="cuda") for n in nwin]
        plan.excise(ins, outs, masks, counts)
        meds = [torch.full((n,), -99, dtype=torch.int32, device="cuda") for n in nwin]
        mads = [torch.full((n,), -99, dtype=torch.int32, device="cuda") for n in nwin]
        moms = [torch.full((n,), -99, dtype=torch.int32, device="cuda") for n in nwin]
        st, totals = plan.stats(meds, mads)
        plan.stats_mom(moms)
        torch.cuda.synchronize()
        noise_pass = bool(flags & rfi.RFI_PLAN_NOISE_PASS) and mode == 3
        # windows that span more than one stage class (at most 16 KiB, at most 32 KiB, larger; by
        # the window's bytes, or the stream's when it is shorter) make one internal plan per class
        esz = 1 if bits == 8 else 2
        parts = len({0 if b <= 16384 else (1 if b <= 32768 else 2)
                     for b in (min(W, x.size) * esz for W, x in zip(windows, xs))})
        assert plan.info().kernels_per_call == parts * (4 if noise_pass else 3)
        res = [dict(z=outs[i].cpu().numpy(), mask=masks[i].cpu().numpy().view(np.uint32),
                    counts=counts[i].cpu().numpy().view(np.uint32), median=meds[i].cpu().numpy(),
                    mad=mads[i].cpu().numpy(), mom=moms[i].cpu().numpy()) for i in range(len(xs))]
        return st, totals, res
    finally:
        plan.close()


def _check(got, ref, what):
    for key in ("mom", "median", "mad", "counts", "mask", "z"):
        a, b = got[key], ref[key]
        assert a.shape == b.shape, (what, key)
        if not np.array_equal(a, b):
            bad = np.flatnonzero(a != b)
            raise AssertionError("%s %s differs at %d positions, first %s" % (what, key, bad.size, bad[:8]))


CASES = [
    # bits, windows, lengths (ragged tails, a non-16-byte window), k_mom, mode
    (8, [512, 4096, 1000], [300 * 512 + 77, 40 * 4096, 120 * 1000 + 999], 7, 0),
    (8, [512, 4096, 1000], [300 * 512 + 77, 40 * 4096, 120 * 1000 + 999], 64, 3),
    (8, [1024, 1024], [500 * 1024, 130 * 1024 + 5], 2, 2),
    (8, [2048], [90 * 2048 + 100], 5000, 1),   # k_mom beyond the stream: running prefix median
    (8, [256, 8192], [2000 * 256 + 1, 33 * 8192], 300, 3),  # more windows than one MoM chunk
    (12, [1024, 2000], [200 * 1024 + 3, 80 * 2000 + 1999], 16, 3),
    (12, [4096], [70 * 4096], 4096, 2),
    (12, [512, 1001], [400 * 512, 150 * 1001 + 7], 3, 0),
]


@pytest.mark.parametrize("bits,windows,lens,kmom,mode", CASES)
def test_mom_plan_matches_oracle(cuda, rfi, bits, windows, lens, kmom, mode):
    xs = _streams(bits, lens, 40 + kmom)
    sids = [3 + 10 * i for i in range(len(xs))]
    k = 3.0 if bits == 8 else 3.5
    st, totals, got = _gpu(rfi, xs, windows, bits, k, mode, kmom, const=-2, seed=77, sids=sids)
    assert st == rfi.RFI_OK and totals.device_status == rfi.RFI_OK
    flagged = 0
    for i, x in enumerate(xs):
        ref = oracle.excise_mom(x, windows[i], k, mode, kmom, const=-2, seed=77, stream_id=sids[i], bits=bits,
                                threads=8)
        assert ref["status"] == 0
        _check(got[i], ref, "stream %d" % i)
        flagged += int(ref["counts"].sum())
    assert totals.flagged == flagged


@pytest.mark.parametrize("bits,windows,lens,kmom,mode", [c for c in CASES if c[4] == 3])
def test_mom_noise_pass_matches_oracle(cuda, rfi, bits, windows, lens, kmom, mode):
    """RFI_PLAN_NOISE_PASS: the apply pass replaces with 0 and a fourth kernel writes the noise
    from each window's M and MoM; every output equals the oracle's."""
    xs = _streams(bits, lens, 40 + kmom)
    k = 3.0 if bits == 8 else 3.5
    st, totals, got = _gpu(rfi, xs, windows, bits, k, mode, kmom, const=-2, seed=77,
                           flags=rfi.RFI_PLAN_NOISE_PASS | rfi.RFI_PLAN_GRAPH)
    assert st == rfi.RFI_OK and totals.device_status == rfi.RFI_OK
    for i, x in enumerate(xs):
        ref = oracle.excise_mom(x, windows[i], k, mode, kmom, const=-2, seed=77, stream_id=i, bits=bits, threads=8)
        _check(got[i], ref, "stream %d" % i)


@pytest.mark.parametrize("bits", [8, 12])
def test_mom_many_streams(cuda, rfi, bits):
    """120 streams of mixed window lengths (16 to 16384 samples) and lengths (one sample to a few
    hundred windows): the estimation pass, the sliding median over each stream's own MADs and the
    apply pass (and the noise pass) keep every stream's windows apart."""
    rng = np.random.default_rng(6060 + bits)
    S = 120
    wins = [int(rng.choice([16, 100, 256, 1000, 1024, 4096, 16384])) for _ in range(S)]
    lens = [int(rng.integers(1, min(300 * W, 1 << 18))) for W in wins]
    sids = [int(v) for v in rng.integers(0, 2 ** 32, size=S)]
    xs = _streams(bits, lens, 60 + bits)
    k = 3.0 if bits == 8 else 3.5
    for kmom, mode, flags in ((7, 3, rfi.RFI_PLAN_GRAPH), (64, 3, rfi.RFI_PLAN_NOISE_PASS), (2, 2, 0)):
        st, totals, got = _gpu(rfi, xs, wins, bits, k, mode, kmom, const=4, seed=21, flags=flags, sids=sids)
        assert st == rfi.RFI_OK and totals.device_status == rfi.RFI_OK
        flagged = 0
        for i, x in enumerate(xs):
            ref = oracle.excise_mom(x, wins[i], k, mode, kmom, const=4, seed=21, stream_id=sids[i], bits=bits,
                                    threads=8)
            _check(got[i], ref, "stream %d (W %d, kmom %d, flags %#x)" % (i, wins[i], kmom, flags))
            flagged += int(ref["counts"].sum())
        assert totals.flagged == flagged


def test_mom_graph_and_repeated_calls(cuda, rfi):
    """The CUDA-graph form gives the same bits, call after call."""
    lens = [200 * 4096 + 11, 150 * 4096]
    xs = _streams(8, lens, 5)
    W = [4096, 4096]
    a = _gpu(rfi, xs, W, 8, 3.0, 3, 32, seed=7, flags=rfi.RFI_PLAN_GRAPH)[2]
    for i, x in enumerate(xs):
        ref = oracle.excise_mom(x, 4096, 3.0, 3, 32, seed=7, stream_id=i, threads=8)
        _check(a[i], ref, "graph stream %d" % i)


def test_mom_of_one_window_is_the_mad_plan(cuda, rfi):
    """mom_windows 0 or 1 is the plain per-window plan (one kernel per call)."""
    import torch
    xs = _streams(8, [64 * 1024 + 9], 9)
    for kmom in (0, 1):
        plan = rfi.Plan(8, [xs[0].size], [1024], 3.0, 0, mom_windows=kmom)
        try:
            assert plan.info().kernels_per_call == 1
            d = torch.from_numpy(xs[0]).cuda()
            o = torch.empty_like(d)
            plan.excise([d], [o])
            torch.cuda.synchronize()
            ref = oracle.excise(xs[0], 1024, 3.0, 0)
            assert np.array_equal(o.cpu().numpy(), ref["z"])
            with pytest.raises(rfi.RfiError):
                plan.stats_mom([torch.empty(65, dtype=torch.int32, device="cuda")])
        finally:
            plan.close()


def test_mom_unsupported_forms(cuda, rfi):
    import torch
    xs = _streams(8, [8 * 1024], 1)
    with pytest.raises(rfi.RfiError):
        rfi.Plan(8, [xs[0].size], [1024], 3.0, 0, flags=rfi.RFI_PLAN_PER_STREAM, mom_windows=4)
    plan = rfi.Plan(8, [xs[0].size], [1024], 3.0, 0, mom_windows=4)
    try:
        h = [xs[0].copy()]
        o = [np.empty_like(xs[0])]
        assert rfi.rfi_excise_host(plan.handle, h, o) == rfi.RFI_ERR_UNSUPPORTED
    finally:
        plan.close()
    d = rfi.make_desc(8, [xs[0].size], [1024], 3.0, 0, mom_windows=4)
    t = torch.from_numpy(xs[0]).cuda()
    st, _ = rfi.rfi_excise_noalloc(d, [t], [torch.empty_like(t)])
    assert st == rfi.RFI_ERR_UNSUPPORTED


def test_mom_full_size_paper_configuration(cuda, rfi):
    """The GWB MoM configuration (4096-sample windows, median of 4096 MADs) on 60 streams of
    2^25 samples (8192 windows each, so the median slides over full histories), in the
    benchmark's launch form. Windows sampled across the streams are checked
    against the oracle run on the slice of k_mom windows that ends at them; every output is
    checked for consistency."""
    import torch
    S, N, W, K = 60, 1 << 25, 4096, 4096
    p = synth.params(seed=2, sigma=16.0, burst_rate=2e-3, burst_len_max=64, bits=8, amp=(5.0, 15.0))
    xs = [synth.fill(p, s, N) for s in range(S)]
    st, totals, got = _gpu(rfi, xs, [W] * S, 8, 3.0, 3, K, seed=7, flags=rfi.RFI_PLAN_GRAPH)
    assert st == rfi.RFI_OK
    nw = N // W
    rng = np.random.default_rng(0)
    picks = [(0, 0), (1, K - 2), (7, K - 1), (13, K), (21, K + 1000), (59, nw - 1)] + \
        [(int(rng.integers(S)), int(rng.integers(nw))) for _ in range(3)]
    for s, j in picks:
        j0 = max(0, j - K + 1)
        hist = oracle.excise(xs[s][j0 * W:j * W], W, 3.0, 0, threads=8, want=("z", "mad"))["mad"] if j > j0 \
            else np.zeros(0, np.int32)
        ref = oracle.excise_mom(xs[s][j * W:(j + 1) * W], W, 3.0, 3, K, seed=7, stream_id=s, abs0=j * W,
                                history=hist)
        g = got[s]
        assert g["mom"][j] == ref["mom"][0] and g["median"][j] == ref["median"][0] and g["mad"][j] == ref["mad"][0]
        assert g["counts"][j] == ref["counts"][0]
        assert np.array_equal(g["mask"][j * (W // 32):(j + 1) * (W // 32)], ref["mask"])
        assert np.array_equal(g["z"][j * W:(j + 1) * W], ref["z"])
    total = 0
    for s in range(S):
        g = got[s]
        bits = np.unpackbits(g["mask"].view(np.uint8), bitorder="little").reshape(nw, W).sum(axis=1)
        assert np.array_equal(bits, g["counts"])
        total += int(g["counts"].sum())
        changed = g["z"] != xs[s]
        flagged = np.unpackbits(g["mask"].view(np.uint8), bitorder="little").astype(bool)
        assert not np.any(changed & ~flagged)  # only flagged samples change
    assert totals.flagged == total
    # whole streams against the oracle, every window, in both digital-noise forms (the benchmark
    # runs the MoM plan with RFI_PLAN_NOISE_PASS)
    st2, totals2, got2 = _gpu(rfi, xs, [W] * S, 8, 3.0, 3, K, seed=7,
                              flags=rfi.RFI_PLAN_GRAPH | rfi.RFI_PLAN_NOISE_PASS)
    assert st2 == rfi.RFI_OK and totals2.flagged == totals.flagged
    threads = os.cpu_count() or 1
    t0 = time.time()
    for s in (0, 13, 37, 59):
        ref = oracle.excise_mom(xs[s], W, 3.0, 3, K, seed=7, stream_id=s, threads=threads)
        assert ref["status"] == 0
        _check(got[s], ref, "stream %d one-pass" % s)
        _check(got2[s], ref, "stream %d noise pass" % s)
    print("\nMoM whole-stream comparison: 4 streams in %.1f s on %d threads" % (time.time() - t0, threads))
