"""The in-place form that writes back only what changes (RFI_PLAN_WRITE_FLAGGED), against the
CPU oracle, bit for bit.

rfi_excise then takes out == in; chunks of 16 samples without a flagged sample are not stored
(they already hold their value) and with digital noise only the flagged samples are. The
result in the buffer must equal the oracle's output on the original samples, with masks,
counts, M and D in full."""
import numpy as np
import pytest

import synth

from .parity import assert_same, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

LENS = [5 * 16384 + 1234, 3 * 16384, 2 * 16384 + 16, 777, 40 * 1024 + 3]
WINS = [16384, 16384, 16384, 16384, 1024]


def _streams(seed):
    p = synth.params(seed=seed, sigma=16.0, burst_rate=4e-3, burst_len_max=64, bits=8, amp=(5.0, 15.0))
    return [synth.fill(p, s, n) for s, n in enumerate(LENS)]


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("flags", [0x80, 0x80 | 0x4 | 0x8, 0x80 | 0x40])  # plain, graph + autotune, noise pass asked
def test_in_place_write_flagged(cuda, rfi, mode, flags):
    xs = _streams(900 + mode)
    const = 1 if mode == 1 else 0
    ref = oracle_run(xs, WINS, 8, 3.0, mode, const, 7)
    got, st, totals, _ = gpu_run(rfi, xs, WINS, 8, 3.0, mode, const, 7, flags=flags, in_place=True)
    assert st == 0
    assert_same(got, ref, "mode %d flags %#x" % (mode, flags))
    assert totals.flagged == sum(int(r["counts"].sum()) for r in ref)


@pytest.mark.parametrize("offset", [1, 8])
def test_in_place_write_flagged_unaligned(cuda, rfi, offset):
    """Buffers off a 16-byte boundary: the consumers stage the windows themselves and the
    ragged stores skip unflagged samples."""
    xs = _streams(950 + offset)
    for mode in (2, 3):
        ref = oracle_run(xs, WINS, 8, 3.0, mode, 0, 7)
        got, st, _, _ = gpu_run(rfi, xs, WINS, 8, 3.0, mode, 0, 7, flags=0x80, in_place=True, offset=offset)
        assert st == 0
        assert_same(got, ref, "mode %d offset %d" % (mode, offset))


def test_write_flagged_needs_in_place(cuda, rfi):
    import torch
    xs = _streams(970)
    plan = rfi.Plan(8, [x.size for x in xs], WINS, 3.0, 0, flags=rfi.RFI_PLAN_WRITE_FLAGGED)
    try:
        d_in = [torch.from_numpy(x).cuda() for x in xs]
        d_out = [torch.empty_like(t) for t in d_in]
        with pytest.raises(rfi.RfiError):
            plan.excise(d_in, d_out)
        plan.excise(d_in, d_in)  # in place is accepted
        torch.cuda.synchronize()
    finally:
        plan.close()
