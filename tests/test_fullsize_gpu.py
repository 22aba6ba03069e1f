"""Full-size workloads in the benchmark's launch configuration (batched, CUDA graph, autotuned
shape): sampled windows against the oracle, and properties checked over every output."""
import numpy as np
import pytest

import oracle
from synth import workloads

from .parity import gen_streams

pytestmark = pytest.mark.gpu

SAMPLES = 40


def _bits_of(mask_words_t, n):
    import torch
    b = mask_words_t.view(torch.uint8)
    sh = torch.arange(8, device=b.device, dtype=torch.uint8)
    return ((b.unsqueeze(-1) >> sh) & 1).reshape(-1)[:n]


def _check_workload(rfi, w, variants, flags, rng_seed):
    import torch
    xs = gen_streams(w)
    bits = w.bits
    esz = 1 if bits == 8 else 2
    dev_in = [torch.from_numpy(x).cuda() for x in xs]
    outs = [torch.empty_like(t) for t in dev_in]
    lens = [x.size for x in xs]
    wins = [s.window for s in w.streams]
    rng = np.random.default_rng(rng_seed)
    for v in variants:
        plan = rfi.Plan(bits, lens, wins, v.k, v.mode, v.const, v.seed, flags)
        try:
            nwin = plan.num_windows
            masks = [torch.empty(plan.mask_words(i), dtype=torch.int32, device="cuda") for i in range(len(xs))]
            counts = [torch.empty(nwin[i], dtype=torch.int32, device="cuda") for i in range(len(xs))]
            meds = [torch.empty(nwin[i], dtype=torch.int32, device="cuda") for i in range(len(xs))]
            mads = [torch.empty(nwin[i], dtype=torch.int32, device="cuda") for i in range(len(xs))]
            plan.excise(dev_in, outs, masks, counts)
            st, totals = plan.stats(meds, mads)
            assert st == 0, rfi.rfi_status_string(st)
            assert totals.windows == sum(nwin)
            assert totals.flagged == sum(int(c.sum().item()) for c in counts)
            # every output: unflagged samples unchanged, counts = mask popcount, zero/const values
            for i in range(len(xs)):
                W = wins[i]
                mw = (W + 31) // 32
                m = masks[i].view(nwin[i], mw)
                flags_i = _bits_of(m.contiguous(), nwin[i] * mw * 32).view(nwin[i], mw * 32)[:, :W]
                flat = flags_i.reshape(-1)[:lens[i]].bool()
                assert torch.equal(flags_i.sum(dim=1, dtype=torch.int64), counts[i].to(torch.int64))
                assert bool(((outs[i] == dev_in[i]) | flat).all())
                if v.mode in (0, 1):
                    want = 0 if v.mode == 0 else v.const
                    assert bool((outs[i][flat] == want).all())
            # sampled windows against the oracle
            for _ in range(SAMPLES):
                i = int(rng.integers(0, len(xs)))
                W = wins[i]
                wi = int(rng.integers(0, nwin[i]))
                if _ == 0:
                    i, wi = len(xs) - 1, nwin[len(xs) - 1] - 1   # always include a last window
                    W = wins[i]
                s0 = wi * W
                s1 = min(lens[i], s0 + W)
                r = oracle.excise(xs[i][s0:s1], W, v.k, v.mode, const=v.const, seed=v.seed,
                                  stream_id=w.streams[i].index, abs0=s0, bits=bits)
                assert r["status"] == 0
                mw = (W + 31) // 32
                z = outs[i][s0:s1].cpu().numpy()
                assert np.array_equal(z, r["z"]), (v.name, i, wi)
                assert np.array_equal(masks[i][wi * mw:(wi + 1) * mw].cpu().numpy().view(np.uint32), r["mask"])
                assert int(counts[i][wi].item()) == int(r["counts"][0])
                assert int(meds[i][wi].item()) == int(r["median"][0])
                assert int(mads[i][wi].item()) == int(r["mad"][0])
        finally:
            plan.close()


def test_gwb60_full_size(cuda, rfi):
    w = workloads.gwb60()
    _check_workload(rfi, w, w.variants, rfi.RFI_PLAN_GRAPH | rfi.RFI_PLAN_AUTOTUNE, 1)


def test_twelve60_full_size(cuda, rfi):
    w = workloads.twelve60()
    _check_workload(rfi, w, w.variants, rfi.RFI_PLAN_GRAPH | rfi.RFI_PLAN_AUTOTUNE, 2)


def test_uneven60_full_size(cuda, rfi):
    w = workloads.uneven60()
    _check_workload(rfi, w, w.variants, rfi.RFI_PLAN_GRAPH | rfi.RFI_PLAN_AUTOTUNE, 3)
