"""Power-metered excision (RFI_PLAN_POWER) against the oracle.

The kernel sums x^2 over every window's input and z^2 over its output while it excises. These
sums are the points of the detected-power series behind the improvement metric (Section III-A);
they must equal the sums over the oracle's input and output exactly (integers), and the
excision outputs must be the same bits as without metering.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _streams(bits, lens, seed):
    if bits == 8:
        p = synth.params(seed=seed, sigma=16.0, burst_rate=2e-3, burst_len_max=64, bits=8, amp=(5.0, 15.0))
    else:
        p = synth.params(seed=seed, sigma=120.0, burst_rate=5e-3, burst_len_max=256, bits=12,
                         amp=(4.0, 30.0), drift_amp=50.0)
    return [synth.fill(p, s, n) for s, n in enumerate(lens)]


def _run(rfi, xs, windows, bits, mode, flags, seed=7, k=3.0):
    import torch
    plan = rfi.Plan(bits, [x.size for x in xs], windows, k, mode, 2, seed, flags)
    try:
        ins = [torch.from_numpy(x).cuda() for x in xs]
        outs = [torch.full_like(t, 3) for t in ins]
        masks = [torch.zeros(plan.mask_words(i), dtype=torch.int32, device="cuda") for i in range(len(xs))]
        counts = [torch.zeros(n, dtype=torch.int32, device="cuda") for n in plan.num_windows]
        plan.excise(ins, outs, masks, counts)
        pw = None
        if flags & rfi.RFI_PLAN_POWER:
            pw = [torch.full((2 * n,), -1, dtype=torch.int64, device="cuda") for n in plan.num_windows]
            plan.stats_power(pw)
        st, totals = plan.stats()
        torch.cuda.synchronize()
        assert st == rfi.RFI_OK
        return ([o.cpu().numpy() for o in outs], [m.cpu().numpy() for m in masks],
                [p.cpu().numpy() for p in pw] if pw is not None else None)
    finally:
        plan.close()


@pytest.mark.parametrize("bits,mode", [(8, 0), (8, 1), (8, 2), (8, 3), (12, 0), (12, 2), (12, 3)])
def test_power_sums_match_the_oracle(cuda, rfi, bits, mode):
    windows = [16384, 1000, 4096] if bits == 8 else [8192, 1001, 512]
    lens = [20 * windows[0] + 333, 300 * windows[1] + 7, 50 * windows[2]]
    xs = _streams(bits, lens, 30 + mode)
    z, m, pw = _run(rfi, xs, windows, bits, mode, rfi.RFI_PLAN_POWER)
    z0, m0, _ = _run(rfi, xs, windows, bits, mode, 0)
    for i, x in enumerate(xs):
        ref = oracle.excise(x, windows[i], 3.0, mode, const=2, seed=7, stream_id=i, bits=bits, threads=8)
        assert np.array_equal(z[i], ref["z"]) and np.array_equal(m[i].view(np.uint32), ref["mask"])
        assert np.array_equal(z[i], z0[i]) and np.array_equal(m[i], m0[i])
        assert np.array_equal(pw[i][0::2], oracle.window_power(x, windows[i])), "stream %d input power" % i
        assert np.array_equal(pw[i][1::2], oracle.window_power(ref["z"], windows[i])), "stream %d output power" % i


def test_metric_from_gpu_power_matches_the_oracle(cuda, rfi):
    """The improvement metric computed from the kernel's power equals the oracle's metric on
    the oracle's own outputs; zero and noise beat clipping (Section III-B)."""
    W = 4096
    p = synth.params(seed=3, sigma=16.0, burst_rate=1e-3, burst_len_max=64, bits=8, amp=(5.0, 15.0))
    xs = [synth.fill(p, 0, 1 << 23)]
    got = {}
    for mode in (0, 3, 2):
        _, _, pw = _run(rfi, xs, [W], 8, mode, rfi.RFI_PLAN_POWER | rfi.RFI_PLAN_GRAPH)
        st, db, su, sf = rfi.rfi_improvement_db(pw[0], 1, 64)
        assert st == rfi.RFI_OK
        ref_z = oracle.excise(xs[0], W, 3.0, mode, const=2, seed=7, threads=8, want=("z",))["z"]
        ref = oracle.improvement_db(oracle.window_power(xs[0], W), oracle.window_power(ref_z, W))
        assert db == pytest.approx(ref[0], rel=1e-9)
        got[mode] = db
    assert got[0] > got[2] + 3.0 and got[3] > got[2] + 3.0


def test_power_unsupported_forms(cuda, rfi):
    with pytest.raises(rfi.RfiError):
        rfi.Plan(8, [4096], [1024], 3.0, 0, flags=rfi.RFI_PLAN_POWER | rfi.RFI_PLAN_PER_STREAM)
    with pytest.raises(rfi.RfiError):
        rfi.Plan(8, [4096], [1024], 3.0, 0, flags=rfi.RFI_PLAN_POWER, mom_windows=4)
    plan = rfi.Plan(8, [4096], [1024], 3.0, 0)
    try:
        import torch
        with pytest.raises(rfi.RfiError):
            plan.stats_power([torch.empty(8, dtype=torch.int64, device="cuda")])
    finally:
        plan.close()
