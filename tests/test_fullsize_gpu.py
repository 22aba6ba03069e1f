"""Full-size workloads in the benchmark's launch configuration (batched, CUDA graph, autotuned
shape). Selected variants are compared with the oracle on every window of every stream (one
stream at a time, so host memory stays bounded); the others on sampled windows, with
properties checked over every output. A noise variant compared in full runs in both digital
noise forms the benchmark may choose between (in the excision kernel, or RFI_PLAN_NOISE_PASS)."""
import os
import time

import numpy as np
import pytest

import oracle
from synth import workloads

from .parity import gen_streams

pytestmark = pytest.mark.gpu

SAMPLES = 40
THREADS = os.cpu_count() or 1


def _bits_of(mask_words_t, n):
    import torch
    b = mask_words_t.view(torch.uint8)
    sh = torch.arange(8, device=b.device, dtype=torch.uint8)
    return ((b.unsqueeze(-1) >> sh) & 1).reshape(-1)[:n]


def _run_form(rfi, dev_in, lens, wins, bits, v, flags):
    """One plan call; returns its device outputs (out, mask, counts, M, D) per stream."""
    import torch
    plan = rfi.Plan(bits, lens, wins, v.k, v.mode, v.const, v.seed, flags)
    try:
        nwin = plan.num_windows
        outs = [torch.empty_like(t) for t in dev_in]
        masks = [torch.empty(plan.mask_words(i), dtype=torch.int32, device="cuda") for i in range(len(lens))]
        counts = [torch.empty(nwin[i], dtype=torch.int32, device="cuda") for i in range(len(lens))]
        meds = [torch.empty(nwin[i], dtype=torch.int32, device="cuda") for i in range(len(lens))]
        mads = [torch.empty(nwin[i], dtype=torch.int32, device="cuda") for i in range(len(lens))]
        plan.excise(dev_in, outs, masks, counts)
        st, totals = plan.stats(meds, mads)
        assert st == 0, rfi.rfi_status_string(st)
        assert totals.windows == sum(nwin)
        assert totals.flagged == sum(int(c.sum().item()) for c in counts)
        return dict(z=outs, mask=masks, counts=counts, median=meds, mad=mads, nwin=nwin)
    finally:
        plan.close()


def _check_properties(g, dev_in, lens, wins, v):
    """Every output: unflagged samples unchanged, counts = mask popcount, zero/const values."""
    import torch
    for i in range(len(lens)):
        W, nw = wins[i], g["nwin"][i]
        mw = (W + 31) // 32
        m = g["mask"][i].view(nw, mw)
        flags_i = _bits_of(m.contiguous(), nw * mw * 32).view(nw, mw * 32)[:, :W]
        flat = flags_i.reshape(-1)[:lens[i]].bool()
        assert torch.equal(flags_i.sum(dim=1, dtype=torch.int64), g["counts"][i].to(torch.int64))
        assert bool(((g["z"][i] == dev_in[i]) | flat).all())
        if v.mode in (0, 1):
            want = 0 if v.mode == 0 else v.const
            assert bool((g["z"][i][flat] == want).all())


def _check_sampled(g, xs, w, v, rng):
    lens = [x.size for x in xs]
    wins = [s.window for s in w.streams]
    for n in range(SAMPLES):
        i = int(rng.integers(0, len(xs)))
        wi = int(rng.integers(0, g["nwin"][i]))
        if n == 0:
            i = len(xs) - 1
            wi = g["nwin"][i] - 1  # always include a last window
        W = wins[i]
        s0 = wi * W
        s1 = min(lens[i], s0 + W)
        r = oracle.excise(xs[i][s0:s1], W, v.k, v.mode, const=v.const, seed=v.seed,
                          stream_id=w.streams[i].index, abs0=s0, bits=w.bits)
        assert r["status"] == 0
        mw = (W + 31) // 32
        assert np.array_equal(g["z"][i][s0:s1].cpu().numpy(), r["z"]), (v.name, i, wi)
        assert np.array_equal(g["mask"][i][wi * mw:(wi + 1) * mw].cpu().numpy().view(np.uint32), r["mask"])
        assert int(g["counts"][i][wi].item()) == int(r["counts"][0])
        assert int(g["median"][i][wi].item()) == int(r["median"][0])
        assert int(g["mad"][i][wi].item()) == int(r["mad"][0])


def _check_full(forms, xs, w, v):
    """Every window of every stream, all five outputs, against the oracle on the whole stream."""
    wins = [s.window for s in w.streams]
    for i, x in enumerate(xs):
        r = oracle.excise(x, wins[i], v.k, v.mode, const=v.const, seed=v.seed, stream_id=w.streams[i].index,
                          bits=w.bits, threads=THREADS)
        assert r["status"] == 0
        for fname, g in forms.items():
            for key in ("z", "mask", "counts", "median", "mad"):
                a = g[key][i].cpu().numpy()
                b = r[key]
                a = a.view(b.dtype) if a.dtype.itemsize == b.dtype.itemsize else a
                if not np.array_equal(a, b):
                    bad = np.flatnonzero(a != b)
                    raise AssertionError("%s %s (%s) stream %d %s differs at %d of %d positions, first %s"
                                         % (w.name, v.name, fname, i, key, bad.size, a.size, bad[:8]))


def _check_workload(rfi, w, flags, rng_seed, full=()):
    import torch
    xs = gen_streams(w)
    dev_in = [torch.from_numpy(x).cuda() for x in xs]
    lens = [x.size for x in xs]
    wins = [s.window for s in w.streams]
    rng = np.random.default_rng(rng_seed)
    timing = {}
    for v in w.variants:
        if v.name in full:
            forms = {"one-pass": flags}
            if v.mode == workloads.NOISE:
                forms["noise-pass"] = flags | rfi.RFI_PLAN_NOISE_PASS
            got = {name: _run_form(rfi, dev_in, lens, wins, w.bits, v, f) for name, f in forms.items()}
            for g in got.values():
                _check_properties(g, dev_in, lens, wins, v)
            t0 = time.time()
            _check_full(got, xs, w, v)
            timing[v.name] = time.time() - t0
            del got
        else:
            g = _run_form(rfi, dev_in, lens, wins, w.bits, v, flags)
            _check_properties(g, dev_in, lens, wins, v)
            _check_sampled(g, xs, w, v, rng)
            del g
        torch.cuda.empty_cache()
    print("\n%s full-data comparison seconds (oracle on %d threads): %s" % (w.name, THREADS, timing))


def test_gwb60_full_size(cuda, rfi):
    w = workloads.gwb60()
    _check_workload(rfi, w, rfi.RFI_PLAN_GRAPH | rfi.RFI_PLAN_AUTOTUNE, 1,
                    full=("k3-noise", "k5-noise", "k3-clip"))


def test_twelve60_full_size(cuda, rfi):
    w = workloads.twelve60()
    _check_workload(rfi, w, rfi.RFI_PLAN_GRAPH | rfi.RFI_PLAN_AUTOTUNE, 2, full=("k3.5-noise",))


def test_uneven60_full_size(cuda, rfi):
    w = workloads.uneven60()
    _check_workload(rfi, w, rfi.RFI_PLAN_GRAPH | rfi.RFI_PLAN_AUTOTUNE, 3, full=("k3-noise",))
