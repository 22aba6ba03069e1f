"""Pins of the improvement-metric oracle (Section III-A) to closed forms and to the behaviour
the paper reports for the replacement options.

The metric is 10 log10 of the ratio of the average mean-to-RMS ratios of the filtered and the
unfiltered detected-power series. The closed forms below fix each step: the per-window power,
the grouping into points and blocks, the mean-to-RMS ratio of a block, the average over blocks
and the logarithm; the last test is the paper's qualitative result on synthetic bursts.
"""
import numpy as np
import pytest

import oracle
import synth


def test_window_power_is_the_sum_of_squares():
    x = np.array([3, -4, 0, 1, 127, -128, 2], np.int8)
    assert list(oracle.window_power(x, 3)) == [9 + 16, 1 + 127 ** 2 + 128 ** 2, 4]
    y = np.array([-2048, 2047, 5], np.int16)
    assert list(oracle.window_power(y, 2)) == [2048 ** 2 + 2047 ** 2, 25]


def test_two_valued_block_ratio():
    # a block alternating a, b has mean (a+b)/2 and RMS deviation |a-b|/2
    a, b = 30.0, 10.0
    blk = np.array([a, b] * 32)
    assert oracle.mean_to_rms(blk, 1, 64) == pytest.approx((a + b) / abs(a - b), rel=1e-12)


def test_points_blocks_and_average():
    # two blocks with ratios 2 and 4 average to 3; points sum windows_per_point windows
    blk1 = np.array([3.0, 1.0] * 2)      # mean 2, rms 1 -> 2
    blk2 = np.array([5.0, 3.0] * 2)      # mean 4, rms 1 -> 4
    series = np.concatenate([blk1, blk2, [100.0]])  # trailing partial block dropped
    assert oracle.mean_to_rms(series, 1, 4) == pytest.approx(3.0, rel=1e-12)
    per_window = np.repeat(series / 2, 2)  # each point split over two windows
    assert oracle.mean_to_rms(per_window, 2, 4) == pytest.approx(3.0, rel=1e-12)
    # a block of zero deviation is left out
    flat = np.concatenate([np.full(4, 7.0), blk1])
    assert oracle.mean_to_rms(flat, 1, 4) == pytest.approx(2.0, rel=1e-12)


def test_improvement_closed_forms():
    rng = np.random.default_rng(1)
    p = rng.uniform(100, 200, size=640)
    db, su, sf = oracle.improvement_db(p, p)
    assert db == pytest.approx(0.0, abs=1e-12) and su == sf
    # scale invariance of each ratio
    assert oracle.improvement_db(p, 7.5 * p)[0] == pytest.approx(0.0, abs=1e-12)
    # halving every block's deviation about its mean doubles the ratio: +3.0103 dB
    blocks = p.reshape(-1, 64)
    m = blocks.mean(axis=1, keepdims=True)
    q = (m + 0.5 * (blocks - m)).ravel()
    assert oracle.improvement_db(p, q)[0] == pytest.approx(10 * np.log10(2.0), rel=1e-9)


def test_replacement_options_rank_as_reported():
    """Section III-B: replacement by zero gives the best improvement, digital noise a similar
    one, and the threshold (clipping) a clearly smaller one. Checked on a synthetic stream of
    short strong bursts (the impulsive RFI the per-window MAD is meant for)."""
    W = 4096
    p = synth.params(seed=3, sigma=16.0, burst_rate=1e-3, burst_len_max=64, bits=8, amp=(5.0, 15.0))
    x = synth.fill(p, 0, 1 << 23)
    pu = oracle.window_power(x, W)
    imp = {}
    for mode in (oracle.ZERO, oracle.NOISE, oracle.CLIP):
        z = oracle.excise(x, W, 3.0, mode, seed=7, threads=8, want=("z",))["z"]
        imp[mode] = oracle.improvement_db(pu, oracle.window_power(z, W))[0]
    assert imp[oracle.ZERO] > 3.0
    assert abs(imp[oracle.ZERO] - imp[oracle.NOISE]) < 1.5
    assert imp[oracle.NOISE] > imp[oracle.CLIP] + 3.0


def test_library_metric_matches_the_oracle():
    """rfi_improvement_db (host code of the library, no GPU) against the oracle's metric on
    interleaved per-window powers: same grouping, same blocks, equal to rounding."""
    import paper_1710_08576_gb300 as rfi
    rng = np.random.default_rng(7)
    nwin = 64 * 37 + 5
    pu = rng.integers(10 ** 6, 10 ** 7, size=nwin)
    pf = pu - rng.integers(0, 10 ** 6, size=nwin)
    pu[100:130] *= 30  # bursts
    inter = np.empty(2 * nwin, np.uint64)
    inter[0::2] = pu
    inter[1::2] = pf
    for wpp, ppb in ((1, 64), (4, 16), (3, 7)):
        st, db, su, sf = rfi.rfi_improvement_db(inter, wpp, ppb)
        assert st == rfi.RFI_OK
        ref = oracle.improvement_db(pu, pf, wpp, ppb)
        assert db == pytest.approx(ref[0], rel=1e-9, abs=1e-12)
        assert su == pytest.approx(ref[1], rel=1e-12) and sf == pytest.approx(ref[2], rel=1e-12)
    assert rfi.rfi_improvement_db(inter[:20], 1, 64)[0] == rfi.RFI_ERR_INVALID_ARG
