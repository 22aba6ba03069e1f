"""Streams past 2^31 and 2^32 samples against the CPU oracle, every window.

One int8 stream of 2^32 + 3 * 16384 + 100 samples: window indices and sample offsets beyond 32
bits, the last windows' digital noise keyed with a nonzero high counter word (the absolute
sample index passes 2^32), and a plan asked for the noise as a second kernel, which routes
segments of 2^31 samples or more through the one-pass form. One 12-bit stream of
2^31 + 8192 + 17 samples: byte offsets past 2^32 in the int16 container. Each GPU result is
compared with one oracle run over the whole stream.
"""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


def _gpu(rfi, x, W, bits, k, mode, seed, flags):
    import torch
    plan = rfi.Plan(bits, [x.size], [W], k, mode, 0, seed, flags, [3])
    try:
        nw = plan.num_windows[0]
        d_in = torch.from_numpy(x).cuda()
        d_out = torch.empty_like(d_in)
        d_mask = torch.empty(plan.mask_words(0), dtype=torch.int32, device="cuda")
        d_cnt = torch.empty(nw, dtype=torch.int32, device="cuda")
        d_med = torch.empty(nw, dtype=torch.int32, device="cuda")
        d_mad = torch.empty(nw, dtype=torch.int32, device="cuda")
        plan.excise([d_in], [d_out], [d_mask], [d_cnt])
        st, totals = plan.stats([d_med], [d_mad])
        torch.cuda.synchronize()
        assert st == 0, rfi.rfi_status_string(st)
        del d_in
        got = dict(z=d_out.cpu().numpy(), mask=d_mask.cpu().numpy().view(np.uint32),
                   counts=d_cnt.cpu().numpy().view(np.uint32), median=d_med.cpu().numpy(),
                   mad=d_mad.cpu().numpy())
        info = plan.info()
        del d_out, d_mask, d_cnt, d_med, d_mad
        torch.cuda.empty_cache()
        return got, totals, info
    finally:
        plan.close()


def _compare(got, ref, what):
    for key in ("median", "mad", "counts", "mask", "z"):
        a, b = got[key], ref[key]
        assert a.shape == b.shape, (what, key)
        if not np.array_equal(a, b):
            bad = np.flatnonzero(a != b)
            raise AssertionError("%s: %s differs at %d positions, first %s" % (what, key, bad.size, bad[:8]))


def test_int8_stream_past_two_to_the_32(cuda, rfi):
    W = 16384
    n = (1 << 32) + 3 * W + 100
    p = synth.params(seed=31, sigma=16.0, burst_rate=2e-3, burst_len_max=64, bits=8, amp=(5.0, 15.0))
    x = synth.fill(p, 3, n)
    ref = oracle.excise(x, W, 3.0, oracle.NOISE, seed=7, stream_id=3, bits=8, threads=THREADS)
    assert ref["status"] == 0
    # the last window's samples are keyed past 2^32: the high counter word is 1 there
    assert (n - 1) >> 32 == 1
    for flags in (rfi.RFI_PLAN_GRAPH, rfi.RFI_PLAN_GRAPH | rfi.RFI_PLAN_NOISE_PASS):
        got, totals, info = _gpu(rfi, x, W, 8, 3.0, 3, 7, flags)
        # a segment of 2^31 samples or more keeps the noise in the excision kernel
        assert info.kernels_per_call == 1
        assert totals.windows == -(-n // W) and totals.flagged == int(ref["counts"].sum())
        _compare(got, ref, "int8 n = 2^32 + %d, flags %#x" % (n - (1 << 32), flags))
        del got


def test_twelve_bit_stream_past_two_to_the_31(cuda, rfi):
    W = 8192
    n = (1 << 31) + W + 17
    p = synth.params(seed=32, sigma=120.0, burst_rate=5e-3, burst_len_max=256, bits=12, amp=(4.0, 30.0),
                     drift_amp=50.0)
    x = synth.fill(p, 3, n)
    ref = oracle.excise(x, W, 3.5, oracle.CLIP, seed=0, stream_id=3, bits=12, threads=THREADS)
    assert ref["status"] == 0
    got, totals, _ = _gpu(rfi, x, W, 12, 3.5, 2, 0, rfi.RFI_PLAN_GRAPH)
    assert totals.flagged == int(ref["counts"].sum())
    _compare(got, ref, "12-bit n = 2^31 + %d" % (n - (1 << 31)))
