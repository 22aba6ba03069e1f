"""Helpers for the GPU-vs-oracle parity tests: run a plan through the C ABI, run the oracle on
the same host buffers, and compare every output element by element (bit-exact)."""
from __future__ import annotations

import os

import numpy as np

import oracle
import synth

THREADS = os.cpu_count() or 1


def gen_streams(workload, lengths=None):
    """Host sample arrays for a workload's streams (optionally overriding the lengths)."""
    xs = []
    for i, s in enumerate(workload.streams):
        n = lengths[i] if lengths is not None else s.length
        xs.append(synth.fill(s.feed, s.index, n))
    return xs


def oracle_run(xs, windows, bits, k, mode, const=0, seed=0, stream_ids=None):
    res = []
    for i, x in enumerate(xs):
        sid = stream_ids[i] if stream_ids is not None else i
        r = oracle.excise(x, windows[i], k, mode, const=const, seed=seed, stream_id=sid, bits=bits,
                          threads=THREADS)
        res.append(r)
    return res


def gpu_run(rfi, xs, windows, bits, k, mode, const=0, seed=0, flags=0, shape=None, stream_ids=None,
            in_place=False, offset=0, host=False, calls=1):
    """Excise host arrays xs on the GPU; returns per-stream dicts like oracle.excise plus the
    rfi_stats status and totals. offset shifts every device buffer by that many bytes."""
    import torch
    dt = torch.int8 if bits == 8 else torch.int16
    esz = 1 if bits == 8 else 2
    plan = rfi.Plan(bits, [x.size for x in xs], windows, k, mode, const, seed, flags, stream_ids, shape)
    try:
        nwin = plan.num_windows
        if host:
            ins = [np.ascontiguousarray(x) for x in xs]
            outs = [np.empty_like(x) for x in xs]
            masks = [np.zeros(plan.mask_words(i), np.uint32) for i in range(len(xs))]
            counts = [np.zeros(nwin[i], np.uint32) for i in range(len(xs))]
            for _ in range(calls):
                plan.excise_host(ins, outs, masks, counts)
            z = outs
            m = masks
            c = counts
        else:
            bufs_in, bufs_out, ins, outs = [], [], [], []
            for x in xs:
                raw = torch.empty(x.size * esz + 64, dtype=torch.uint8, device="cuda")
                view_ptr = raw.data_ptr() + offset
                host_t = torch.from_numpy(x.view(np.uint8).copy())
                raw[offset:offset + x.size * esz].copy_(host_t)
                bufs_in.append(raw)
                ins.append(view_ptr)
                if in_place:
                    outs.append(view_ptr)
                    bufs_out.append(raw)
                else:
                    ro = torch.full((x.size * esz + 64,), 0x5A, dtype=torch.uint8, device="cuda")
                    bufs_out.append(ro)
                    outs.append(ro.data_ptr() + offset)
            masks = [torch.full((plan.mask_words(i),), 0xDEADBEEF - (1 << 32), dtype=torch.int32,
                                device="cuda") for i in range(len(xs))]
            counts = [torch.full((nwin[i],), -1, dtype=torch.int32, device="cuda") for i in range(len(xs))]
            for _ in range(calls):
                plan.excise(ins, outs, masks, counts)
            torch.cuda.synchronize()
            z = []
            for i, x in enumerate(xs):
                b = bufs_out[i][offset:offset + x.size * esz].cpu().numpy()
                z.append(b.view(np.int8 if bits == 8 else np.int16).copy())
            m = [t.cpu().numpy().view(np.uint32) for t in masks]
            c = [t.cpu().numpy().view(np.uint32) for t in counts]
        meds = [torch.zeros(nwin[i], dtype=torch.int32, device="cuda") for i in range(len(xs))]
        mads = [torch.zeros(nwin[i], dtype=torch.int32, device="cuda") for i in range(len(xs))]
        st, totals = plan.stats(meds, mads)
        torch.cuda.synchronize()
        out = []
        for i in range(len(xs)):
            out.append(dict(z=z[i], mask=m[i], counts=c[i], median=meds[i].cpu().numpy(),
                            mad=mads[i].cpu().numpy()))
        return out, st, totals, plan.info()
    finally:
        plan.close()


def assert_same(gpu, ref, what=""):
    for i, (g, r) in enumerate(zip(gpu, ref)):
        for key in ("median", "mad", "counts", "mask", "z"):
            a, b = g[key], r[key]
            if a.shape != b.shape or not np.array_equal(a, b):
                bad = np.flatnonzero(a != b) if a.shape == b.shape else []
                raise AssertionError("%s stream %d %s differs at %d positions, first %s" %
                                     (what, i, key, len(bad), bad[:8]))
