"""The multi-window form of the int8 kernel against the CPU oracle, bit for bit.

Plans with windows of 2^l = 512..8192 samples run the instantiation that histograms several
windows of a tile at once in the lane-striped table: eight for windows of at most 2048 samples
and for tiles of eight or more larger windows (window slot g in lanes 4g..4g+3), otherwise four
(lanes 8g..8g+7). It reduces them in
one pass that also clears the table and searches them on several warps in parallel. These cases
pin down what that adds to the per-window path: tiles of every remainder of the slot count
(sub-tiles of 1 to 7 windows), the switch between multi-window tiles and per-window tiles
(16384-sample windows, ragged tails, windows that are not a power of two, unaligned buffers) in
one kernel, whose table then has to be cleared or its running sums reset, every replacement
mode, both noise forms and every consumer-group size.
"""
import numpy as np
import pytest

import synth

from .parity import assert_same, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _streams(lens, seed, burst_rate=4e-3):
    p = synth.params(seed=seed, sigma=16.0, burst_rate=burst_rate, burst_len_max=96, bits=8, amp=(4.0, 15.0))
    return [synth.fill(p, s, n) for s, n in enumerate(lens)]


@pytest.mark.parametrize("W", [512, 1024, 2048, 4096, 8192])
@pytest.mark.parametrize("cw", [4, 8, 16])
def test_every_tile_remainder(cuda, rfi, W, cw):
    """16 KiB stages hold 16384 / W windows; streams of 1 .. 16384 / W + 5 full windows (and one
    ragged tail each) make tiles of every size, so the last sub-tile holds fewer windows than
    there are slots, and a tail window takes the per-window path right after."""
    per = 16384 // W
    counts = sorted(set([1, 2, 3, 4, 5, 6, 7, per, per + 1, per + 3, per + 5]))
    lens = [n * W for n in counts] + [n * W + 77 for n in counts[:4]]
    xs = _streams(lens, 100 + W + cw)
    shape = dict(consumer_warps=cw, stages=2, ctas_per_sm=1, dynamic_tiles=1, groups=1, stage_bytes=16384)
    wins = [W] * len(xs)
    for mode in (0, 1, 2, 3):
        ref = oracle_run(xs, wins, 8, 3.0, mode, 1 if mode == 1 else 0, 7)
        got, st, totals, _ = gpu_run(rfi, xs, wins, 8, 3.0, mode, 1 if mode == 1 else 0, 7, shape=shape)
        assert st == 0
        assert_same(got, ref, "W %d cw %d mode %d" % (W, cw, mode))
        assert totals.flagged == sum(int(r["counts"].sum()) for r in ref)


@pytest.mark.parametrize("form", [0, 0x40])  # noise in the excision kernel, or RFI_PLAN_NOISE_PASS
@pytest.mark.parametrize("dynamic", [1, 2])
def test_multi_and_per_window_tiles_in_one_kernel(cuda, rfi, form, dynamic):
    """Streams whose tiles take the multi-window path (4096, 512, 2048) and streams whose tiles
    take the per-window path (16384; 1000, not a power of two; 4096 with a ragged tail) in one
    plan and one kernel, the CTAs taking tiles from an atomic cursor or round robin: the table
    moves between running sums and cleared-after-use in both directions, many times over."""
    wins = [4096, 16384, 512, 1000, 2048, 16384, 4096, 8192]
    lens = [37 * 4096, 9 * 16384 + 5, 300 * 512, 61 * 1000 + 999, 90 * 2048, 7 * 16384, 29 * 4096 + 4095,
            13 * 8192]
    xs = _streams(lens, 321, burst_rate=6e-3)
    shape = dict(consumer_warps=8, stages=2, ctas_per_sm=1, dynamic_tiles=dynamic, groups=1, stage_bytes=16384)
    for mode in (2, 3):
        ref = oracle_run(xs, wins, 8, 3.0, mode, 0, 9)
        got, st, totals, _ = gpu_run(rfi, xs, wins, 8, 3.0, mode, 0, 9, flags=form | 0x20, shape=shape)
        assert st == 0
        assert_same(got, ref, "mode %d form %#x dynamic %d" % (mode, form, dynamic))


@pytest.mark.parametrize("W,sb", [(4096, 32768), (8192, 65536), (4096, 65536)])
@pytest.mark.parametrize("mode", [0, 2, 3])
def test_eight_slots_for_large_windows(cuda, rfi, W, sb, mode):
    """Stages of eight or more 4096- or 8192-sample windows take eight window slots (four lanes
    each) per tile instead of four; tiles of fewer (a stream's last) take four."""
    per = sb // W
    lens = [n * W for n in (1, 3, 7, 8, 9, per, per + 3, 2 * per + 5)] + [5 * W + 99]
    xs = _streams(lens, 700 + W + sb + mode)
    shape = dict(consumer_warps=8, stages=1, ctas_per_sm=1, dynamic_tiles=1, groups=1, stage_bytes=sb)
    wins = [W] * len(xs)
    ref = oracle_run(xs, wins, 8, 3.0, mode, 0, 7)
    got, st, totals, _ = gpu_run(rfi, xs, wins, 8, 3.0, mode, 0, 7, shape=shape)
    assert st == 0
    assert_same(got, ref, "W %d stage %d mode %d" % (W, sb, mode))


def test_multi_window_with_unaligned_buffers_falls_back(cuda, rfi):
    """Buffers one byte off a 16-byte boundary cannot be staged by bulk copies: every tile of the
    plan takes the per-window path of the multi-window kernel; the same data aligned takes the
    multi-window path. Both equal the oracle."""
    wins = [1024, 4096, 2048]
    lens = [40 * 1024, 11 * 4096 + 100, 25 * 2048]
    xs = _streams(lens, 55)
    ref = oracle_run(xs, wins, 8, 2.5, 3, 0, 5)
    for offset in (0, 1):
        got, st, _, _ = gpu_run(rfi, xs, wins, 8, 2.5, 3, 0, 5, offset=offset)
        assert st == 0
        assert_same(got, ref, "offset %d" % offset)


def test_degenerate_windows_in_multi_tiles(cuda, rfi):
    """Constant windows (D = 0: nothing flagged), windows of one value and a burst filling more
    than half a window, side by side in the four slots of a tile."""
    W = 1024
    x = np.zeros(16 * W, np.int8)
    x[W:2 * W] = 5                                   # constant
    x[2 * W:3 * W] = np.tile([-3, 4], W // 2)        # two values
    x[3 * W:4 * W] = 0
    x[3 * W + 100:3 * W + 700] = 120                 # a burst over 60 % of the window
    rng = np.random.default_rng(3)
    x[4 * W:] = np.clip(np.rint(rng.normal(0, 16, 12 * W)), -128, 127).astype(np.int8)
    x[5 * W + 10] = 127
    x[6 * W + 20] = -128
    for mode in (0, 1, 2, 3):
        ref = oracle_run([x], [W], 8, 3.0, mode, 1, 3)
        got, st, _, _ = gpu_run(rfi, [x], [W], 8, 3.0, mode, 1, 3)
        assert st == 0
        assert_same(got, ref, "mode %d" % mode)
