"""The split-warp form of the int8 kernel against the CPU oracle, bit for bit.

With `warp_split = 2` in the launch shape, four consumer warps histogram, reduce and search each
window while the other four replace the window before it; the thresholds go from one to the
other through a ring of hand-over slots. These cases cover what that adds to the joint form:
the zero, constant and threshold modes, every stage count and tile order, tiles of several
windows, ragged tails, windows that fill the largest stages, unaligned buffers (the histogram
warps copy the stage), the write-flagged in-place form, the CUDA graph, the test hook that
delays a CTA, and the plans the form does not serve.
"""
import numpy as np
import pytest

import synth
from synth import workloads

from .parity import assert_same, gen_streams, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _shape(**kw):
    s = dict(consumer_warps=8, groups=1, warp_split=2)
    s.update(kw)
    return s


GWB_LENS = [5 * 16384 + 1234, 3 * 16384, 2 * 16384 + 16, 777]


@pytest.mark.parametrize("stages,ctas,dyn", [(2, 3, 1), (2, 3, 2), (1, 2, 1), (3, 2, 2), (4, 1, 1)])
@pytest.mark.parametrize("vi", [0, 1, 2, 4, 5, 6])  # k 3 and 5; zero, constant, threshold
def test_gwb_variants(cuda, rfi, stages, ctas, dyn, vi):
    w = workloads.gwb60(nstreams=4)
    v = w.variants[vi]
    xs = gen_streams(w, GWB_LENS)
    shape = _shape(stages=stages, ctas_per_sm=ctas, dynamic_tiles=dyn, stage_bytes=16384)
    got, st, totals, info = gpu_run(rfi, xs, [16384] * 4, 8, v.k, v.mode, v.const, v.seed, shape=shape)
    assert st == 0 and info.shape.warp_split == 2
    ref = oracle_run(xs, [16384] * 4, 8, v.k, v.mode, v.const, v.seed)
    assert_same(got, ref, "%s stages %d" % (v.name, stages))
    assert totals.flagged == sum(int(r["counts"].sum()) for r in ref)


@pytest.mark.parametrize("W", [7, 40, 1000, 2000, 4000, 16000, 65536])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_tiles_of_several_windows_and_large_windows(cuda, rfi, W, mode):
    """16-byte multiples that are not powers of two (2000, 4000) go several to a 16 KiB stage,
    each a hand-over of its own, the stage released after the tile's last; other lengths (7, 40,
    1000) go one to a stage, copied in by the histogram warps; 65536-sample windows need 64 KiB
    stages."""
    p = synth.params(seed=41, sigma=16.0, burst_rate=2e-2, burst_len_max=64, bits=8)
    lens = [9 * W + W // 3 + 1, 3 * W, W + 5]
    xs = [synth.fill(p, s, n) for s, n in enumerate(lens)]
    sb = max(16384, (W + 127) // 128 * 128)
    shape = _shape(stages=2, ctas_per_sm=1, stage_bytes=sb)
    got, st, _, _ = gpu_run(rfi, xs, [W] * 3, 8, 3.0, mode, 1 if mode == 1 else 0, shape=shape)
    assert st == 0
    assert_same(got, oracle_run(xs, [W] * 3, 8, 3.0, mode, 1 if mode == 1 else 0), "W %d mode %d" % (W, mode))


@pytest.mark.parametrize("offset", [1, 8])
def test_unaligned_buffers(cuda, rfi, offset):
    w = workloads.gwb60(nstreams=3)
    xs = gen_streams(w, [4 * 16384 + 99, 16384, 2 * 16384 + 1])
    for mode in (0, 2):
        got, st, _, _ = gpu_run(rfi, xs, [16384] * 3, 8, 3.0, mode, offset=offset, shape=_shape(stages=2))
        assert st == 0
        assert_same(got, oracle_run(xs, [16384] * 3, 8, 3.0, mode), "offset %d mode %d" % (offset, mode))


def test_graph_and_repeated_calls(cuda, rfi):
    w = workloads.gwb60(nstreams=4)
    xs = gen_streams(w, GWB_LENS)
    got, st, _, _ = gpu_run(rfi, xs, [16384] * 4, 8, 5.0, 2, flags=rfi.RFI_PLAN_GRAPH, calls=3,
                            shape=_shape(stages=2, ctas_per_sm=3))
    assert st == 0
    assert_same(got, oracle_run(xs, [16384] * 4, 8, 5.0, 2), "graph")


def test_injected_timeout_is_reported_and_context_survives(cuda, rfi):
    w = workloads.gwb60(nstreams=2)
    xs = gen_streams(w, [4 * 16384, 16384 + 3])
    got, st, totals, _ = gpu_run(rfi, xs, [16384] * 2, 8, 3.0, 0, flags=rfi.RFI_PLAN_INJECT_TIMEOUT,
                                 shape=_shape(stages=2))
    assert st == rfi.RFI_ERR_TIMEOUT and totals.device_status == rfi.RFI_ERR_TIMEOUT
    assert_same(got, oracle_run(xs, [16384] * 2, 8, 3.0, 0), "after injected timeout")
    got, st, _, _ = gpu_run(rfi, xs, [16384] * 2, 8, 3.0, 0, shape=_shape(stages=2))
    assert st == 0


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_write_flagged_in_place(cuda, rfi, mode):
    """RFI_PLAN_WRITE_FLAGGED in the split-warp form: in place, only the chunks that change are
    stored, so the buffer ends equal to the oracle's output."""
    w = workloads.gwb60(nstreams=4)
    xs = gen_streams(w, GWB_LENS)
    got, st, _, info = gpu_run(rfi, xs, [16384] * 4, 8, 3.0, mode, 1 if mode == 1 else 0,
                               flags=rfi.RFI_PLAN_WRITE_FLAGGED, in_place=True, shape=_shape(stages=2))
    assert st == 0 and info.shape.warp_split == 2
    assert_same(got, oracle_run(xs, [16384] * 4, 8, 3.0, mode, 1 if mode == 1 else 0), "write-flagged mode %d" % mode)


@pytest.mark.parametrize("what", ["noise", "twelve_bit", "four_warps", "two_groups", "pow2_small"])
def test_plans_the_form_does_not_serve(cuda, rfi, what):
    args = dict(bits=8, lens=[3 * 16384], wins=[16384], mode=0, shape=_shape())
    if what == "noise":
        args["mode"] = 3
    elif what == "twelve_bit":
        args["bits"] = 12
    elif what == "four_warps":
        args["shape"] = _shape(consumer_warps=4)
    elif what == "two_groups":
        args["shape"] = _shape(groups=2)
    else:
        args["wins"] = [4096]  # the multi-window form serves this plan
    with pytest.raises(rfi.RfiError) as e:
        rfi.Plan(args["bits"], args["lens"], args["wins"], 3.0, args["mode"], 0, 7, 0, None, args["shape"])
    assert e.value.status == rfi.RFI_ERR_UNSUPPORTED


def test_autotuned_plan_may_take_either_form(cuda, rfi):
    w = workloads.gwb60(nstreams=4)
    xs = gen_streams(w, GWB_LENS)
    got, st, _, info = gpu_run(rfi, xs, [16384] * 4, 8, 3.0, 1, 1, flags=rfi.RFI_PLAN_AUTOTUNE)
    assert st == 0 and info.shape.warp_split in (1, 2)
    assert_same(got, oracle_run(xs, [16384] * 4, 8, 3.0, 1, 1), "autotuned")
