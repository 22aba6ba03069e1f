"""Fused output format (rfi_plan_desc.out_format): the excised samples written as fp16 or bf16,
the real-valued input of a channeliser FFT, by the excision kernel itself.

Every int8 value is exact in fp16 and in bf16, and every 12-bit value in fp16 (the CPU test
below pins that); so the GPU's fp16/bf16 output must equal the oracle's integer output
converted, exactly, sample for sample.
"""
import numpy as np
import pytest

import oracle
import synth


def test_the_conversions_are_exact():
    import torch
    v8 = np.arange(-128, 128)
    v12 = np.arange(-2048, 2048)
    assert np.array_equal(v8.astype(np.float16).astype(np.int64), v8)
    assert np.array_equal(v12.astype(np.float16).astype(np.int64), v12)
    assert torch.equal(torch.from_numpy(v8).to(torch.bfloat16).to(torch.int64), torch.from_numpy(v8))


def _streams(bits, lens, seed):
    if bits == 8:
        p = synth.params(seed=seed, sigma=16.0, burst_rate=3e-3, burst_len_max=64, bits=8, amp=(5.0, 15.0))
    else:
        p = synth.params(seed=seed, sigma=120.0, burst_rate=5e-3, burst_len_max=256, bits=12,
                         amp=(4.0, 30.0), drift_amp=50.0)
    return [synth.fill(p, s, n) for s, n in enumerate(lens)]


def _run(rfi, xs, windows, bits, k, mode, fmt, flags=0, offset=0):
    import torch
    plan = rfi.Plan(bits, [x.size for x in xs], windows, k, mode, -3, 17, flags, None, out_format=fmt)
    try:
        ins = [torch.from_numpy(x).cuda() for x in xs]
        raws = [torch.full((2 * x.size + 64,), 0x7E, dtype=torch.uint8, device="cuda") for x in xs]
        outs = [r.data_ptr() + offset for r in raws]
        masks = [torch.full((plan.mask_words(i),), -1, dtype=torch.int32, device="cuda") for i in range(len(xs))]
        counts = [torch.full((n,), -1, dtype=torch.int32, device="cuda") for n in plan.num_windows]
        plan.excise(ins, outs, masks, counts)
        st, _ = plan.stats()
        torch.cuda.synchronize()
        assert st == rfi.RFI_OK
        dt = torch.float16 if fmt == rfi.RFI_OUT_F16 else torch.bfloat16
        res = []
        for i, x in enumerate(xs):
            b = raws[i][offset:offset + 2 * x.size].contiguous().view(dt).float().cpu().numpy()
            res.append((b, masks[i].cpu().numpy().view(np.uint32), counts[i].cpu().numpy().view(np.uint32)))
        return res
    finally:
        plan.close()


def _check(xs, windows, bits, k, mode, res):
    for i, x in enumerate(xs):
        ref = oracle.excise(x, windows[i], k, mode, const=-3, seed=17, stream_id=i, bits=bits, threads=8)
        z, m, c = res[i]
        assert np.array_equal(z, ref["z"].astype(np.float32)), "stream %d samples" % i
        assert np.array_equal(m, ref["mask"]) and np.array_equal(c, ref["counts"])


@pytest.mark.gpu
@pytest.mark.parametrize("fmt", [1, 2])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_int8_to_half_formats(cuda, rfi, fmt, mode):
    windows = [16384, 1000, 4096]
    lens = [10 * 16384 + 123, 200 * 1000 + 7, 30 * 4096]
    xs = _streams(8, lens, 50 + mode)
    _check(xs, windows, 8, 3.0, mode, _run(rfi, xs, windows, 8, 3.0, mode, fmt))


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [0, 2, 3])
def test_twelve_bit_to_fp16(cuda, rfi, mode):
    windows = [8192, 1001]
    lens = [12 * 8192 + 9, 100 * 1001 + 1]
    xs = _streams(12, lens, 60 + mode)
    _check(xs, windows, 12, 3.5, mode, _run(rfi, xs, windows, 12, 3.5, mode, 1))


@pytest.mark.gpu
def test_formats_unaligned_split_and_graph(cuda, rfi):
    """A 2-byte (not 16-byte) aligned output, a plan split by window class, and the graph form."""
    windows = [2048, 65536, 32768]
    lens = [40 * 2048 + 5, 3 * 65536 + 77, 4 * 32768]
    xs = _streams(8, lens, 3)
    _check(xs, windows, 8, 3.0, 3, _run(rfi, xs, windows, 8, 3.0, 3, 1, flags=0x4, offset=2))
    _check(xs, windows, 8, 3.0, 0, _run(rfi, xs, windows, 8, 3.0, 0, 2, offset=0))


@pytest.mark.gpu
def test_noise_overflow_in_fp16(cuda, rfi):
    """12-bit windows whose flagged samples overflow the noise list take the per-warp path, which
    writes fp16 too."""
    rng = np.random.default_rng(2)
    n = 16384
    core = rng.integers(-2, 3, size=n)
    far = rng.choice([-1500, 1500], size=n) + rng.integers(-3, 4, size=n)
    x = np.where(rng.random(n) < 0.45, far, core).astype(np.int16)
    xs = [np.concatenate([x, x[::-1]])]
    _check(xs, [n], 12, 3.0, 3, _run(rfi, xs, [n], 12, 3.0, 3, 1))


@pytest.mark.gpu
def test_format_arguments(cuda, rfi):
    import torch
    with pytest.raises(rfi.RfiError):
        rfi.Plan(12, [4096], [1024], 3.0, 0, out_format=2)          # bf16 would round 12-bit values
    with pytest.raises(rfi.RfiError):
        rfi.Plan(8, [4096], [1024], 3.0, 0, flags=rfi.RFI_PLAN_PER_STREAM, out_format=1)
    with pytest.raises(rfi.RfiError):
        rfi.Plan(8, [4096], [1024], 3.0, 0, out_format=3)
    plan = rfi.Plan(8, [4096], [1024], 3.0, 0, out_format=1)
    try:
        t = torch.zeros(4096, dtype=torch.int8, device="cuda")
        o = torch.zeros(2 * 4096 + 2, dtype=torch.uint8, device="cuda")
        assert rfi.rfi_excise(plan.handle, [t], [o.data_ptr() + 1]) == rfi.RFI_ERR_ALIGNMENT
        h = [np.zeros(4096, np.int8)]
        assert rfi.rfi_excise_host(plan.handle, h, [np.zeros(4096, np.float16)]) == rfi.RFI_ERR_UNSUPPORTED
    finally:
        plan.close()
