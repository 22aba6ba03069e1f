"""Digital copy (rfi_plan_create_copies): one pass over the input, several (k, mode) variants.

Section III-A describes the FPGA's copy mode, in which one antenna input feeds several filters
with different thresholds and replacement options at once. Each variant's outputs must equal,
bit for bit, the oracle run with that variant's parameters alone; the window's median and MAD
are shared.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GWB_VARIANTS = [(k, m, 1 if m == 1 else 0, 7 if m == 3 else 0) for k in (3.0, 5.0) for m in (0, 1, 2, 3)]


def _streams(bits, lens, seed):
    if bits == 8:
        p = synth.params(seed=seed, sigma=16.0, burst_rate=3e-3, burst_len_max=64, bits=8, amp=(5.0, 15.0))
    else:
        p = synth.params(seed=seed, sigma=120.0, burst_rate=5e-3, burst_len_max=256, bits=12,
                         amp=(4.0, 30.0), drift_amp=50.0)
    return [synth.fill(p, s, n) for s, n in enumerate(lens)]


def _run(rfi, xs, windows, bits, variants, flags=0, sids=None, offsets=None, with_counts=True):
    import torch
    plan = rfi.CopiesPlan(bits, [x.size for x in xs], windows, variants, flags, sids)
    try:
        ins = [torch.from_numpy(x).cuda() for x in xs]
        esz = 1 if bits == 8 else 2
        raws, outs, masks, counts = [], [], [], []
        for v in range(len(variants)):
            off = offsets[v] if offsets else 0
            ro = [torch.full((x.size * esz + 64,), 0x33, dtype=torch.uint8, device="cuda") for x in xs]
            raws.append(ro)
            outs.append([t.data_ptr() + off for t in ro])
            masks.append([torch.full((plan.mask_words(i),), -1, dtype=torch.int32, device="cuda")
                          for i in range(len(xs))])
            counts.append([torch.full((n,), -1, dtype=torch.int32, device="cuda") for n in plan.num_windows]
                          if with_counts or v % 2 == 0 else [None] * len(xs))
        plan.excise(ins, outs, masks, counts)
        meds = [torch.zeros(n, dtype=torch.int32, device="cuda") for n in plan.num_windows]
        mads = [torch.zeros(n, dtype=torch.int32, device="cuda") for n in plan.num_windows]
        st, totals = plan.stats(meds, mads)
        torch.cuda.synchronize()
        assert plan.info().kernels_per_call == 1
        res = []
        for v in range(len(variants)):
            off = offsets[v] if offsets else 0
            res.append([dict(z=raws[v][i][off:off + xs[i].size * esz].cpu().numpy().view(xs[i].dtype),
                             mask=masks[v][i].cpu().numpy().view(np.uint32),
                             counts=None if counts[v][i] is None else counts[v][i].cpu().numpy().view(np.uint32))
                        for i in range(len(xs))])
        return st, totals, res, [m.cpu().numpy() for m in meds], [m.cpu().numpy() for m in mads]
    finally:
        plan.close()


def _check(xs, windows, bits, variants, res, meds, mads, sids=None):
    flagged = 0
    for v, (k, mode, const, seed) in enumerate(variants):
        for i, x in enumerate(xs):
            sid = sids[i] if sids else i
            ref = oracle.excise(x, windows[i], k, mode, const=const, seed=seed, stream_id=sid, bits=bits, threads=8)
            g = res[v][i]
            assert np.array_equal(g["z"], ref["z"]), "variant %d stream %d samples" % (v, i)
            assert np.array_equal(g["mask"], ref["mask"]), "variant %d stream %d mask" % (v, i)
            if g["counts"] is not None:
                assert np.array_equal(g["counts"], ref["counts"]), "variant %d stream %d counts" % (v, i)
            assert np.array_equal(meds[i], ref["median"]) and np.array_equal(mads[i], ref["mad"])
            flagged += int(ref["counts"].sum())
    return flagged


@pytest.mark.parametrize("flags", [0, 0x4])
def test_gwb_variant_set_in_one_pass(cuda, rfi, flags):
    windows = [16384, 16384, 4096, 1000]
    lens = [12 * 16384 + 77, 9 * 16384, 40 * 4096 + 3, 300 * 1000 + 999]
    xs = _streams(8, lens, 21)
    sids = [5, 6, 7, 8]
    st, totals, res, meds, mads = _run(rfi, xs, windows, 8, GWB_VARIANTS, flags, sids)
    assert st == rfi.RFI_OK
    flagged = _check(xs, windows, 8, GWB_VARIANTS, res, meds, mads, sids)
    assert totals.flagged == flagged


def test_twelve_bit_and_two_noise_variants(cuda, rfi):
    variants = [(3.5, 3, 0, 7), (2.0, 3, 0, 123456789012), (4.0, 2, 0, 0), (3.0, 1, -5, 0)]
    windows = [8192, 2048, 1001]
    lens = [10 * 8192 + 5, 50 * 2048, 70 * 1001 + 1]
    xs = _streams(12, lens, 4)
    st, totals, res, meds, mads = _run(rfi, xs, windows, 12, variants)
    assert st == rfi.RFI_OK
    assert totals.flagged == _check(xs, windows, 12, variants, res, meds, mads)


def test_misaligned_outputs_and_missing_counts(cuda, rfi):
    variants = [(3.0, 0, 0, 0), (3.0, 3, 0, 9), (5.0, 2, 0, 0)]
    windows = [4096]
    xs = _streams(8, [30 * 4096 + 17], 8)
    st, totals, res, meds, mads = _run(rfi, xs, windows, 8, variants, offsets=[0, 3, 8], with_counts=False)
    assert st == rfi.RFI_OK
    _check(xs, windows, 8, variants, res, meds, mads)


def test_copies_arguments(cuda, rfi):
    import torch
    with pytest.raises(rfi.RfiError):
        rfi.CopiesPlan(8, [4096], [1024], [(3.0, 0, 0, 0)] * 9)
    with pytest.raises(rfi.RfiError):
        rfi.CopiesPlan(8, [4096], [1024], [(3.0, 0, 0, 0)], flags=rfi.RFI_PLAN_PER_STREAM)
    plan = rfi.CopiesPlan(8, [4096], [1024], [(3.0, 0, 0, 0), (5.0, 1, 2, 0)])
    try:
        t = torch.zeros(4096, dtype=torch.int8, device="cuda")
        assert rfi.rfi_excise(plan.handle, [t], [t]) == rfi.RFI_ERR_INVALID_ARG
    finally:
        plan.close()
