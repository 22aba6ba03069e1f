"""The allocation-free entry point rfi_excise_noalloc against the plan-based path.

rfi_excise_noalloc serves callers that must not allocate device memory while they excise (a
receiver loop whose memory is set aside at start-up, a host whose budget belongs to another
allocator): its work list, segment table and counters sit in a fixed device array inside the
library. This file is collected last so that a failure here does not hide the other tests.
Both calls below must match the plan path (rfi_plan_create / rfi_excise / rfi_stats) bit for
bit, the second one after the first has left its contents in the shared array.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from synth import workloads

pytestmark = pytest.mark.gpu


def _streams(bits, lens, seed):
    if bits == 8:
        p = synth.params(seed=seed, sigma=16.0, burst_rate=5e-3, burst_len_max=64, bits=8)
    else:
        p = synth.params(seed=seed, sigma=120.0, burst_rate=5e-3, burst_len_max=256, bits=12,
                         amp=(4.0, 30.0), drift_amp=50.0)
    return [synth.fill(p, s, n) for s, n in enumerate(lens)]


def _run(rfi, xs, W, bits, k, mode, const, seed, noalloc):
    import torch
    dt = torch.int8 if bits == 8 else torch.int16
    dev_in = [torch.from_numpy(x).cuda() for x in xs]
    out = [torch.full_like(t, 77) for t in dev_in]
    nwin = [-(-x.size // W) for x in xs]
    mw = (W + 31) // 32
    masks = [torch.full((n * mw,), -1, dtype=torch.int32, device="cuda") for n in nwin]
    counts = [torch.full((n,), -1, dtype=torch.int32, device="cuda") for n in nwin]
    meds = [torch.full((n,), -99, dtype=torch.int32, device="cuda") for n in nwin]
    mads = [torch.full((n,), -99, dtype=torch.int32, device="cuda") for n in nwin]
    lens = [x.size for x in xs]
    if noalloc:
        d = rfi.make_desc(bits, lens, [W] * len(xs), k, mode, const, seed)
        st, totals = rfi.rfi_excise_noalloc(d, dev_in, out, masks, counts, meds, mads)
    else:
        plan = rfi.Plan(bits, lens, [W] * len(xs), k, mode, const, seed)
        try:
            plan.excise(dev_in, out, masks, counts)
            st, totals = plan.stats(meds, mads)
        finally:
            plan.close()
    torch.cuda.synchronize()
    res = dict(z=[t.cpu().numpy() for t in out], mask=[t.cpu().numpy() for t in masks],
               counts=[t.cpu().numpy() for t in counts], med=[t.cpu().numpy() for t in meds],
               mad=[t.cpu().numpy() for t in mads])
    return st, (totals.windows, totals.flagged, totals.device_status), res


def test_noalloc_matches_plan_path_on_two_calls_in_a_row(cuda, rfi):
    calls = [
        # 8-bit, digital noise, ragged streams
        (8, [5 * 16384 + 1234, 3 * 16384, 2 * 16384 + 16, 777], 16384, 3.0, 3, 0, 7, 11),
        # 12-bit, threshold replacement, different shapes (the shared array keeps call 1's data)
        (12, [6 * 8192 + 5, 8192, 3001], 8192, 3.5, 2, 0, 0, 12),
    ]
    for bits, lens, W, k, mode, const, seed, gseed in calls:
        xs = _streams(bits, lens, gseed)
        st_a, tot_a, a = _run(rfi, xs, W, bits, k, mode, const, seed, noalloc=True)
        st_b, tot_b, b = _run(rfi, xs, W, bits, k, mode, const, seed, noalloc=False)
        assert st_a == 0 and st_b == 0
        assert tot_a == tot_b
        for key in a:
            for i in range(len(xs)):
                assert np.array_equal(a[key][i], b[key][i]), (bits, key, i)


def test_noalloc_rejects_requests_beyond_its_limits(rfi):
    n = rfi.LIB  # noqa: F841  (library loaded)
    d = rfi.make_desc(8, [1024] * 65, [1024] * 65, 3.0, 0)
    st, _ = rfi.rfi_excise_noalloc(d, [1] * 65, [1] * 65)
    assert st == rfi.RFI_ERR_UNSUPPORTED
    d = rfi.make_desc(8, [1024], [0], 3.0, 0)
    st, _ = rfi.rfi_excise_noalloc(d, [1], [1])
    assert st == rfi.RFI_ERR_INVALID_ARG


def _noalloc_vs_oracle(rfi, bits, xs, wins, k, mode, seed, sids=None):
    """rfi_excise_noalloc on device copies of xs, every output compared with the oracle run on
    each whole stream (windows from absolute sample 0, as the call takes them)."""
    import torch
    sids = list(range(len(xs))) if sids is None else sids
    dev_in = [torch.from_numpy(x).cuda() for x in xs]
    out = [torch.full_like(t, 77) for t in dev_in]
    nwin = [-(-x.size // W) for x, W in zip(xs, wins)]
    masks = [torch.full((n * ((W + 31) // 32),), -1, dtype=torch.int32, device="cuda") for n, W in zip(nwin, wins)]
    counts = [torch.full((n,), -1, dtype=torch.int32, device="cuda") for n in nwin]
    meds = [torch.full((n,), -99, dtype=torch.int32, device="cuda") for n in nwin]
    mads = [torch.full((n,), -99, dtype=torch.int32, device="cuda") for n in nwin]
    d = rfi.make_desc(bits, [x.size for x in xs], wins, k, mode, 0, seed, stream_id=sids)
    st, totals = rfi.rfi_excise_noalloc(d, dev_in, out, masks, counts, meds, mads)
    torch.cuda.synchronize()
    assert st == 0, rfi.rfi_status_string(st)
    assert totals.windows == sum(nwin)
    flagged = 0
    for i, x in enumerate(xs):
        r = oracle.excise(x, wins[i], k, mode, seed=seed, stream_id=sids[i], bits=bits,
                          threads=os.cpu_count() or 1)
        assert r["status"] == 0
        got = dict(z=out[i].cpu().numpy(), mask=masks[i].cpu().numpy().view(np.uint32),
                   counts=counts[i].cpu().numpy().view(np.uint32), median=meds[i].cpu().numpy(),
                   mad=mads[i].cpu().numpy())
        for key in got:
            if not np.array_equal(got[key], r[key]):
                bad = np.flatnonzero(got[key] != r[key])
                raise AssertionError("stream %d (W %d) %s differs at %d positions, first %s"
                                     % (i, wins[i], key, bad.size, bad[:8]))
        flagged += int(r["counts"].sum())
    assert totals.flagged == flagged


def test_noalloc_against_oracle_unaligned_mixed_and_largest_windows(cuda, rfi):
    """Windows that are not a multiple of 16 bytes (one window per tile, loaded by lanes), 12-bit
    windows of 1000 samples (8 per tile), a different window per stream, and the largest window
    (65536 samples, one per 64 KiB stage), against the oracle directly."""
    xs = _streams(8, [40 * 1000 + 999, 30 * 4096 + 5, 3 * 65536 + 4097, 200 * 512, 65536], 21)
    _noalloc_vs_oracle(rfi, 8, xs, [1000, 4096, 65536, 512, 65536], 3.0, 3, 7)
    xs = _streams(12, [50 * 1000 + 17, 40 * 1001 + 3], 22)
    _noalloc_vs_oracle(rfi, 12, xs, [1000, 1001], 3.5, 3, 9, sids=[5, 6])


def test_noalloc_doubles_the_stage_when_the_work_list_is_full(cuda, rfi):
    """16 streams of 2^26 + 4096 int8 samples in 4096-sample windows: at the first stage size
    (16 KiB, 4 windows per tile) the work list would need 16 * 4097 = 65552 entries, more than
    the fixed array holds, so the call doubles the stage (8 windows per tile, 32784 entries).
    Every output against the oracle."""
    W, n = 4096, (1 << 26) + 4096
    per = 16384 // W
    assert 16 * -(-(n // W) // per) > rfi.RFI_NOALLOC_MAX_TILES >= 16 * -(-(n // W) // (2 * per))
    xs = _streams(8, [n] * 16, 23)
    _noalloc_vs_oracle(rfi, 8, xs, [W] * 16, 3.0, 3, 7)


def test_noalloc_rejects_a_work_list_beyond_its_array(rfi):
    """70 000 windows of 1000 int8 samples need one work-list entry each (a window that is not a
    multiple of 16 bytes is a tile of its own) at every stage size: more than the fixed array
    holds, so the call returns RFI_ERR_UNSUPPORTED before it touches the (dummy) buffers."""
    d = rfi.make_desc(8, [70000 * 1000], [1000], 3.0, 0)
    st, _ = rfi.rfi_excise_noalloc(d, [16], [16])
    assert st == rfi.RFI_ERR_UNSUPPORTED
