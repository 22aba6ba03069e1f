"""GPU path vs the CPU oracle, bit for bit, through the C ABI (small and ragged cases)."""
import numpy as np
import pytest

import oracle
import synth
from synth import workloads

from .parity import assert_same, gen_streams, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

# "noise_pass": batched noise plans write the digital noise in a second kernel
# (RFI_PLAN_NOISE_PASS); in the other forms it stays in the excision kernel
FORMS = {"batched": 0, "per_stream": 0x1, "graph": 0x4, "noise_pass": 0x40}


def _run_both(rfi, xs, windows, bits, k, mode, const=0, seed=0, **kw):
    got, st, totals, info = gpu_run(rfi, xs, windows, bits, k, mode, const, seed, **kw)
    ref = oracle_run(xs, windows, bits, k, mode, const, seed, kw.get("stream_ids"))
    return got, ref, st, totals, info


@pytest.mark.parametrize("form", list(FORMS))
def test_single_stream_workload(cuda, rfi, form):
    w = workloads.single()
    xs = gen_streams(w)
    v = w.variants[0]
    got, ref, st, totals, info = _run_both(rfi, xs, [w.streams[0].window], 8, v.k, v.mode,
                                           flags=FORMS[form])
    assert st == 0
    assert_same(got, ref, form)
    assert totals.windows == 256 and totals.flagged == int(ref[0]["counts"].sum())


GWB_LENS = [5 * 16384 + 1234, 3 * 16384, 2 * 16384 + 16, 777]


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("vi", range(8))
def test_gwb_variants_small(cuda, rfi, form, vi):
    w = workloads.gwb60(nstreams=4)
    v = w.variants[vi]
    xs = gen_streams(w, GWB_LENS)
    got, ref, st, totals, _ = _run_both(rfi, xs, [16384] * 4, 8, v.k, v.mode, v.const, v.seed,
                                        flags=FORMS[form])
    assert st == 0
    assert_same(got, ref, "%s %s" % (form, v.name))
    assert totals.flagged == sum(int(r["counts"].sum()) for r in ref)


@pytest.mark.parametrize("form", ["batched", "per_stream", "noise_pass"])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_twelve_bit_small(cuda, rfi, form, mode):
    w = workloads.twelve60(nstreams=3)
    xs = gen_streams(w, [6 * 8192 + 777, 8192, 3001])
    got, ref, st, _, _ = _run_both(rfi, xs, [8192] * 3, 12, 3.5, mode, const=-1000, seed=7,
                                   flags=FORMS[form])
    assert st == 0
    assert_same(got, ref, "12-bit mode %d" % mode)


def test_uneven_windows_small(cuda, rfi):
    w = workloads.uneven60(nstreams=8)
    rng = np.random.default_rng(5)
    wins = [1024, 2048, 4096, 8192, 16384, 32768, 65536, 1024]
    lens = [int(W * rng.integers(1, 4) + rng.integers(0, W)) for W in wins]
    xs = gen_streams(w, lens)
    for flags in (0, 0x1, 0x4, 0x40):
        got, ref, st, _, _ = _run_both(rfi, xs, wins, 8, 3.0, 3, seed=7, flags=flags)
        assert st == 0
        assert_same(got, ref, "uneven flags %d" % flags)


SHAPES = [
    dict(consumer_warps=4, stages=2, ctas_per_sm=1, dynamic_tiles=1, groups=1),
    dict(consumer_warps=4, stages=4, ctas_per_sm=2, dynamic_tiles=2, groups=1),
    dict(consumer_warps=8, stages=1, ctas_per_sm=2, dynamic_tiles=1, groups=1),
    dict(consumer_warps=8, stages=2, ctas_per_sm=1, dynamic_tiles=2, stage_bytes=65536, groups=1),
    dict(consumer_warps=16, stages=2, ctas_per_sm=1, dynamic_tiles=1, groups=1),
    dict(consumer_warps=16, stages=4, ctas_per_sm=1, dynamic_tiles=2, stage_bytes=32768, groups=1),
    dict(consumer_warps=4, stages=3, ctas_per_sm=1, dynamic_tiles=1, groups=2),
    dict(consumer_warps=8, stages=4, ctas_per_sm=1, dynamic_tiles=2, groups=2),
    dict(consumer_warps=8, stages=1, ctas_per_sm=1, dynamic_tiles=1, groups=2, stage_bytes=32768),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "cw%d-st%d-c%d-d%d-g%d" % (
    s["consumer_warps"], s["stages"], s["ctas_per_sm"], s["dynamic_tiles"], s["groups"]))
def test_launch_shapes(cuda, rfi, shape):
    w = workloads.gwb60(nstreams=4)
    xs = gen_streams(w, GWB_LENS)
    got, ref, st, _, info = _run_both(rfi, xs, [16384] * 4, 8, 3.0, 3, seed=7, shape=shape)
    assert st == 0 and info.shape.consumer_warps == shape["consumer_warps"]
    assert_same(got, ref, str(shape))


@pytest.mark.parametrize("groups", [1, 2])
@pytest.mark.parametrize("hc", [1, 2, 4])
def test_twelve_bit_histogram_copies(cuda, rfi, hc, groups):
    w = workloads.twelve60(nstreams=2)
    xs = gen_streams(w, [3 * 8192 + 5, 8192 * 2])
    got, ref, st, _, info = _run_both(rfi, xs, [8192] * 2, 12, 3.5, 3, seed=7,
                                      shape=dict(hist_copies=hc, consumer_warps=8, groups=groups,
                                                 stages=1 if hc * groups == 8 else 2))
    assert st == 0 and info.shape.hist_copies == hc and info.shape.groups == groups
    assert_same(got, ref, "hc %d" % hc)


@pytest.mark.parametrize("W", [1, 2, 7, 16, 33, 40, 48, 100, 1000, 65536])
@pytest.mark.parametrize("form", ["batched", "per_stream", "noise_pass"])
def test_odd_window_lengths(cuda, rfi, W, form):
    p = synth.params(seed=21, sigma=16.0, burst_rate=2e-2, burst_len_max=64, bits=8)
    n = 3 * W + (W // 3) + 1 if W > 1 else 50
    xs = [synth.fill(p, 0, n), synth.fill(p, 1, W)]
    for mode in (0, 2, 3):
        got, ref, st, _, _ = _run_both(rfi, xs, [W, W], 8, 3.0, mode, seed=3, flags=FORMS[form])
        assert st == 0
        assert_same(got, ref, "W %d mode %d" % (W, mode))


@pytest.mark.parametrize("bits", [8, 12])
@pytest.mark.parametrize("offset,in_place", [(0, True), (1, False), (2, False), (8, True), (4, False)])
def test_misaligned_and_in_place_buffers(cuda, rfi, bits, offset, in_place):
    if bits == 12 and offset % 2:
        pytest.skip("int16 buffers are 2-byte aligned")
    p = synth.params(seed=22, sigma=16.0 if bits == 8 else 120.0, burst_rate=1e-2, burst_len_max=64, bits=bits)
    xs = [synth.fill(p, s, 4 * 4096 + 99) for s in range(3)]
    for flags in (0, 1, 0x40):
        got, ref, st, _, _ = _run_both(rfi, xs, [4096] * 3, bits, 3.0, 3, seed=9, flags=flags,
                                       offset=offset, in_place=in_place)
        assert st == 0
        assert_same(got, ref, "offset %d in_place %s" % (offset, in_place))


@pytest.mark.parametrize("bits", [8, 12])
@pytest.mark.parametrize("split", [False, True])
def test_noise_pass_packed_units(cuda, rfi, bits, split):
    """RFI_PLAN_NOISE_PASS where the second pass packs several windows into one unit of mask
    words (windows of a multiple of 128 samples up to 2048, powers of two or not) beside windows
    that keep units of their own, in one launch and split into window classes; ragged, short and
    one-sample streams."""
    p = synth.params(seed=33, sigma=16.0 if bits == 8 else 120.0, burst_rate=2e-2, burst_len_max=64, bits=bits)
    wins = [128, 256, 384, 640, 1024, 1920, 2048, 1000, 4096, 16384, 2048, 128]
    lens = [37 * 128 + 5, 21 * 256, 9 * 384 + 383, 13 * 640 + 1, 11 * 1024 + 700, 4 * 1920 + 64, 2048 - 7,
            6 * 1000 + 3, 3 * 4096 + 9, 16384 + 100, 1, 31]
    xs = [synth.fill(p, s, n) for s, n in enumerate(lens)]
    flags = rfi.RFI_PLAN_NOISE_PASS | (0 if split else rfi.RFI_PLAN_NO_SPLIT)
    for k in (2.0, 3.0):
        got, st, totals, info = gpu_run(rfi, xs, wins, bits, k, 3, seed=5, flags=flags)
        assert st == 0
        if not split:
            assert info.kernels_per_call == 2
        ref = oracle_run(xs, wins, bits, k, 3, 0, 5)
        assert_same(got, ref, "bits %d k %g" % (bits, k))
        assert totals.flagged == sum(int(r["counts"].sum()) for r in ref)


@pytest.mark.parametrize("bits", [8, 12])
def test_noise_pass_without_caller_masks(cuda, rfi, bits):
    """A RFI_PLAN_NOISE_PASS plan called without masks (or counts) flags into the plan's own masks
    for its second pass: the samples equal the oracle's; a later call with masks gives the masks
    too. Windows divisible by 32, by 2048 and by neither."""
    import torch
    p = synth.params(seed=31, sigma=16.0 if bits == 8 else 120.0, burst_rate=1e-2, burst_len_max=64, bits=bits)
    wins = [4096, 1000, 64, 65536]
    lens = [5 * 4096 + 17, 7 * 1000 + 999, 300 * 64 + 5, 65536 + 11]
    xs = [synth.fill(p, s, n) for s, n in enumerate(lens)]
    ref = oracle_run(xs, wins, bits, 3.0, 3, 0, 12)
    plan = rfi.Plan(bits, lens, wins, 3.0, 3, 0, 12, rfi.RFI_PLAN_NO_SPLIT | rfi.RFI_PLAN_NOISE_PASS)
    try:
        assert plan.info().kernels_per_call == 2
        ins = [torch.from_numpy(x).cuda() for x in xs]
        outs = [torch.zeros_like(t) for t in ins]
        plan.excise(ins, outs)
        torch.cuda.synchronize()
        for i, x in enumerate(xs):
            assert np.array_equal(outs[i].cpu().numpy(), ref[i]["z"]), "stream %d" % i
        masks = [torch.zeros(plan.mask_words(i), dtype=torch.int32, device="cuda") for i in range(len(xs))]
        outs2 = [torch.zeros_like(t) for t in ins]
        plan.excise(ins, outs2, masks, None)
        torch.cuda.synchronize()
        for i, x in enumerate(xs):
            assert np.array_equal(outs2[i].cpu().numpy(), ref[i]["z"]), "stream %d" % i
            assert np.array_equal(masks[i].cpu().numpy().view(np.uint32), ref[i]["mask"]), "mask %d" % i
    finally:
        plan.close()


@pytest.mark.parametrize("bits", [8, 12])
def test_many_streams_of_mixed_lengths_and_windows(cuda, rfi, bits):
    """300 streams, lengths from 1 sample to a few windows, windows from 1 to 65536 samples: the
    work list, the segment tables, the split by window class and the noise pass's per-segment
    mask blocks all span hundreds of segments. Every form against one oracle run per mode."""
    rng = np.random.default_rng(4242 + bits)
    S = 300
    wins = [min(65536, int(rng.choice([1, 7, 32, 100, 1024, 4096, 16384, 65536, int(rng.integers(1, 70000))])))
            for _ in range(S)]
    lens = [int(rng.integers(1, 3 * min(W, 20000) + 2)) for W in wins]
    sids = [int(v) for v in rng.integers(0, 2 ** 32, size=S)]
    p = synth.params(seed=77 + bits, sigma=16.0 if bits == 8 else 120.0, burst_rate=5e-3, burst_len_max=200,
                     bits=bits)
    xs = [synth.fill(p, s, n) for s, n in enumerate(lens)]
    for mode in (2, 3):
        ref = oracle_run(xs, wins, bits, 3.0, mode, 0, 11, sids)
        flagged = sum(int(r["counts"].sum()) for r in ref)
        for form, flags in FORMS.items():
            got, st, totals, _ = gpu_run(rfi, xs, wins, bits, 3.0, mode, 0, 11, flags=flags, stream_ids=sids)
            assert st == 0
            assert_same(got, ref, "%d streams, bits %d mode %d form %s" % (S, bits, mode, form))
            assert totals.flagged == flagged
            assert totals.windows == sum(-(-n // W) for n, W in zip(lens, wins))


def test_degenerate_windows(cuda, rfi):
    W = 4096
    a = np.zeros(W, np.int8)                         # constant: D = 0
    b = np.full(W, 127, np.int8)                     # saturated high
    c = np.where(np.arange(W) % 2 == 0, -128, 127).astype(np.int8)   # two-valued, saturated
    d = np.zeros(W, np.int8)
    d[: W // 2 + 1] = 5                              # majority equal: D = 0 despite outliers
    d[-10:] = -100
    e = np.full(65536, -7, np.int8)                  # 65536 identical values: counter width
    f = np.arange(W, dtype=np.int64).astype(np.int8)  # uniform over all 256 values
    xs = [a, b, c, d, e, f]
    wins = [W, W, W, W, 65536, W]
    for mode in range(4):
        got, ref, st, _, _ = _run_both(rfi, xs, wins, 8, 3.0, mode, const=55, seed=1)
        assert st == 0
        assert_same(got, ref, "degenerate mode %d" % mode)
        assert got[0]["counts"].sum() == 0 and got[3]["mad"][0] == 0


def test_twelve_bit_extremes_and_range_error(cuda, rfi):
    x = np.tile(np.array([-2048, 2047, 0, 1, 2, 3, 4], np.int16), 1000)
    got, ref, st, _, _ = _run_both(rfi, [x], [7 * 16], 12, 3.0, 2)
    assert st == 0
    assert_same(got, ref, "12-bit extremes")
    bad = x.copy()
    bad[5000] = 2048
    got, st, totals, _ = gpu_run(rfi, [bad], [7 * 16], 12, 3.0, 2)
    assert st == rfi.RFI_ERR_SAMPLE_RANGE and totals.device_status == rfi.RFI_ERR_SAMPLE_RANGE
    # the next call on valid data is clean again
    got, st, _, _ = gpu_run(rfi, [x], [7 * 16], 12, 3.0, 2)
    assert st == 0


def test_injected_timeout_is_reported_and_context_survives(cuda, rfi):
    w = workloads.gwb60(nstreams=2)
    xs = gen_streams(w, [4 * 16384, 16384 + 3])
    got, st, totals, _ = gpu_run(rfi, xs, [16384] * 2, 8, 3.0, 0, flags=rfi.RFI_PLAN_INJECT_TIMEOUT)
    assert st == rfi.RFI_ERR_TIMEOUT and totals.device_status == rfi.RFI_ERR_TIMEOUT
    ref = oracle_run(xs, [16384] * 2, 8, 3.0, 0)
    assert_same(got, ref, "after injected timeout")   # the hook delays, it does not abort
    got, st, _, _ = gpu_run(rfi, xs, [16384] * 2, 8, 3.0, 0)
    assert st == 0


@pytest.mark.parametrize("bits", [8, 12])
def test_host_pipeline(cuda, rfi, bits):
    if bits == 8:
        w = workloads.gwb60(nstreams=3)
        lens, wins, k = [40 * 16384 + 321, 16384, 3000], [16384] * 3, 3.0
    else:
        w = workloads.twelve60(nstreams=2)
        lens, wins, k = [2200 * 8192 + 5, 100], [8192] * 2, 3.5
    xs = gen_streams(w, lens)
    got, ref, st, totals, _ = _run_both(rfi, xs, wins, bits, k, 3, seed=7, host=True, calls=2)
    assert st == 0
    assert_same(got, ref, "host pipeline %d-bit" % bits)
    assert totals.flagged == sum(int(r["counts"].sum()) for r in ref)
    # a noise-pass plan keeps the noise in the chunk kernel on host buffers: the same bits
    got, st, _, _ = gpu_run(rfi, xs, wins, bits, k, 3, seed=7, host=True, flags=rfi.RFI_PLAN_NOISE_PASS)
    assert st == 0
    assert_same(got, ref, "host pipeline, noise-pass plan, %d-bit" % bits)


def test_repeated_calls_and_stream_ids(cuda, rfi):
    w = workloads.gwb60(nstreams=3)
    xs = gen_streams(w, [3 * 16384, 2 * 16384 + 7, 16384])
    sids = [1000, 7, 0xFFFFFFFF]
    got, ref, st, _, _ = _run_both(rfi, xs, [16384] * 3, 8, 3.0, 3, seed=0xFEEDFACECAFEBEEF,
                                   stream_ids=sids, calls=3)
    assert st == 0
    assert_same(got, ref, "repeat")


def test_autotuned_plan(cuda, rfi):
    w = workloads.gwb60(nstreams=4)
    xs = gen_streams(w, GWB_LENS)
    got, ref, st, _, info = _run_both(rfi, xs, [16384] * 4, 8, 5.0, 2, flags=rfi.RFI_PLAN_AUTOTUNE | 0x4)
    assert st == 0 and info.grid >= 1
    assert_same(got, ref, "autotuned")


@pytest.mark.parametrize("bits", [8, 12])
@pytest.mark.parametrize("form", ["batched", "per_stream", "noise_pass"])
def test_noise_list_overflow(cuda, rfi, bits, form):
    """Windows whose flagged samples outnumber the digital-noise list (4096 entries): 55 % of
    each window sits in a narrow core (small D) and 45 % far outside it, so 7000+ of 16384
    samples take noise; the ones past the list are replaced by the lane that found them. A
    65536-sample window (listed by no entry) and windows just under the capacity too."""
    rng = np.random.default_rng(bits)
    dt = np.int8 if bits == 8 else np.int16
    far = 100 if bits == 8 else 1500

    def window(n, frac):
        core = rng.integers(-2, 3, size=n)
        out = rng.choice([-far, far], size=n) + rng.integers(-3, 4, size=n)
        pick = rng.random(n) < frac
        return np.where(pick, out, core).astype(dt)

    W = 16384
    xs = [np.concatenate([window(W, 0.45) for _ in range(6)]),
          np.concatenate([window(W, 4000 / W) for _ in range(4)] + [window(123, 0.4)]),
          window(65536, 0.3)]
    wins = [W, W, 65536]
    got, ref, st, totals, _ = _run_both(rfi, xs, wins, bits, 3.0, 3, seed=99, flags=FORMS[form])
    assert st == 0
    assert_same(got, ref, "noise overflow %s" % form)
    assert got[0]["counts"].min() > 4096


@pytest.mark.parametrize("mode", [0, 3])
def test_split_plan_by_window_class(cuda, rfi, mode):
    """Streams whose windows span the three stage classes (<= 16 KiB, <= 32 KiB, larger) run as
    one internal plan per class: outputs, per-stream M and D and the totals equal the single
    work list and the oracle; the graph, host-buffer and MoM forms route the same way."""
    import torch
    windows = [1024, 65536, 4096, 32768, 16384, 20000, 60000]
    lens = [40 * w + (w // 3) for w in windows]
    p = synth.params(seed=11, sigma=16.0, burst_rate=2e-3, burst_len_max=64, bits=8)
    xs = [synth.fill(p, s, n) for s, n in enumerate(lens)]
    sids = [100 + i for i in range(len(xs))]
    ref = oracle_run(xs, windows, 8, 3.0, mode, 0, 5, sids)
    for flags in (0, rfi.RFI_PLAN_GRAPH, rfi.RFI_PLAN_NO_SPLIT):
        got, st, totals, info = gpu_run(rfi, xs, windows, 8, 3.0, mode, 0, 5, flags=flags, stream_ids=sids)
        assert st == 0
        assert_same(got, ref, "split flags %d" % flags)
        assert totals.flagged == sum(int(r["counts"].sum()) for r in ref)
        assert totals.windows == sum(-(-n // w) for n, w in zip(lens, windows))
        assert info.kernels_per_call == (1 if flags & rfi.RFI_PLAN_NO_SPLIT else 3)
    got, st, _, _ = gpu_run(rfi, xs, windows, 8, 3.0, mode, 0, 5, stream_ids=sids, host=True)
    assert st == 0
    assert_same(got, ref, "split host pipeline")
    # a MoM plan splits the same way (the median of MADs stays within each stream)
    plan = rfi.Plan(8, lens, windows, 3.0, mode, 0, 5, 0, sids, mom_windows=5)
    try:
        ins = [torch.from_numpy(x).cuda() for x in xs]
        outs = [torch.empty_like(t) for t in ins]
        plan.excise(ins, outs)
        moms = [torch.zeros(n, dtype=torch.int32, device="cuda") for n in plan.num_windows]
        plan.stats_mom(moms)
        torch.cuda.synchronize()
        for i, x in enumerate(xs):
            r = oracle.excise_mom(x, windows[i], 3.0, mode, 5, seed=5, stream_id=sids[i], threads=8)
            assert np.array_equal(outs[i].cpu().numpy(), r["z"]) and np.array_equal(moms[i].cpu().numpy(), r["mom"])
    finally:
        plan.close()
