"""The C ABI without a GPU: the library loads, exports what include/rfi.h declares, its structs
match the header's layout, and argument errors come back before any CUDA call."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1710_08576_gb300 as rfi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rfi.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"RFI_API\s+[\w\s\*]*?\b(rfi_\w+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("rfi_plan_create", "rfi_excise", "rfi_stats", "rfi_plan_destroy", "rfi_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(rfi.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_only_the_abi_is_exported():
    out = subprocess.run(["nm", "-D", "--defined-only", rfi.LIB_PATH], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nm unavailable")
    text_syms = {l.split()[-1] for l in out.stdout.splitlines() if " T " in l}
    assert text_syms == set(declared_functions())


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "rfi.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(rfi_launch_shape), sizeof(rfi_plan_desc),
         sizeof(rfi_totals), sizeof(rfi_plan_info), offsetof(rfi_plan_desc, shape));
  printf("%zu %zu %zu\n", offsetof(rfi_plan_desc, k), offsetof(rfi_plan_desc, seed),
         offsetof(rfi_plan_info, shape));
  printf("%zu %zu %zu %zu %zu\n", sizeof(rfi_variant), offsetof(rfi_variant, seed),
         offsetof(rfi_plan_desc, mom_windows), offsetof(rfi_plan_desc, out_format),
         offsetof(rfi_plan_info, kernels_per_call));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    a, b, c = subprocess.check_output([str(exe)], text=True).splitlines()
    C = ctypes
    assert [int(v) for v in a.split()] == [C.sizeof(rfi.RfiLaunchShape), C.sizeof(rfi.RfiPlanDesc),
                                          C.sizeof(rfi.RfiTotals), C.sizeof(rfi.RfiPlanInfo),
                                          rfi.RfiPlanDesc.shape.offset]
    assert [int(v) for v in b.split()] == [rfi.RfiPlanDesc.k.offset, rfi.RfiPlanDesc.seed.offset,
                                          rfi.RfiPlanInfo.shape.offset]
    assert [int(v) for v in c.split()] == [C.sizeof(rfi.RfiVariant), rfi.RfiVariant.seed.offset,
                                          rfi.RfiPlanDesc.mom_windows.offset, rfi.RfiPlanDesc.out_format.offset,
                                          rfi.RfiPlanInfo.kernels_per_call.offset]


def test_constants_match_header(tmp_path):
    """Every RFI_* enum value and flag of the header equals the binding's constant of that name."""
    text = open(HEADER).read()
    names = sorted(set(re.findall(r"#define\s+(RFI_(?:PLAN|MAX|NOALLOC)_\w+)\s", text)) |
                   set(re.findall(r"\b(RFI_(?:OK|ERR_\w+|REPLACE_\w+|OUT_\w+))\s*=", text)))
    assert "RFI_PLAN_NOISE_PASS" in names and "RFI_NOALLOC_SCRATCH_BYTES" in names and "RFI_ERR_BUSY" in names and "RFI_OUT_BF16" in names
    src = tmp_path / "consts.c"
    src.write_text("#include <stdio.h>\n#include \"rfi.h\"\nint main(void) {\n" +
                   "".join('  printf("%%s %%lld\\n", "%s", (long long)(%s));\n' % (n, n) for n in names) +
                   "  return 0;\n}\n")
    exe = tmp_path / "consts"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        name, value = line.split()
        assert hasattr(rfi, name), name
        assert getattr(rfi, name) == int(value), name


@pytest.mark.parametrize("kw", [
    dict(bits=7), dict(bits=16), dict(stream_len=[0]), dict(window_len=[0]),
    dict(window_len=[65537]), dict(k=0.0), dict(k=-3.0), dict(k=float("nan")), dict(k=1e-7),
    dict(mode=4), dict(mode=-1), dict(flags=0x80000000),
    dict(flags=rfi.RFI_PLAN_PER_STREAM | rfi.RFI_PLAN_GRAPH),
    dict(shape=dict(consumer_warps=5)), dict(shape=dict(stages=9)), dict(shape=dict(hist_copies=3)),
    dict(shape=dict(warp_split=3)), dict(shape=dict(warp_split=-1)),
])
def test_invalid_plan_arguments_fail_before_cuda(kw):
    args = dict(bits=8, stream_len=[4096], window_len=[1024], k=3.0, mode=0)
    args.update(kw)
    shape = args.pop("shape", None)
    d = rfi.make_desc(args["bits"], args["stream_len"], args["window_len"], args["k"], args["mode"],
                      flags=args.get("flags", 0), shape=shape)
    st, h = rfi.rfi_plan_create(d)
    assert st == rfi.RFI_ERR_INVALID_ARG and h is None


def test_null_arguments():
    assert rfi.LIB.rfi_plan_create(None, None) == rfi.RFI_ERR_INVALID_ARG
    assert rfi.LIB.rfi_excise(None, None, None, None, None, None) == rfi.RFI_ERR_INVALID_ARG
    assert rfi.LIB.rfi_stats(None, None, None, None, None) == rfi.RFI_ERR_INVALID_ARG
    assert rfi.LIB.rfi_plan_get_info(None, None) == rfi.RFI_ERR_INVALID_ARG
    assert rfi.LIB.rfi_plan_destroy(None) == rfi.RFI_OK


def test_status_strings():
    for s in range(9):
        assert rfi.rfi_status_string(s) and rfi.rfi_status_string(s) != "unknown status"
    assert rfi.rfi_status_string(99) == "unknown status"
    assert "sm_103a" in rfi.rfi_version()


def test_server_layouts_match_header(tmp_path):
    src = tmp_path / "srv.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "rfi.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(rfi_server_desc), sizeof(rfi_request_desc), sizeof(rfi_server_stats),
         offsetof(rfi_server_desc, memory_budget), offsetof(rfi_request_desc, abs0),
         offsetof(rfi_server_stats, device_status));
  return 0;
}''')
    exe = tmp_path / "srv"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)], text=True).split()]
    C = ctypes
    assert got == [C.sizeof(rfi.RfiServerDesc), C.sizeof(rfi.RfiRequestDesc), C.sizeof(rfi.RfiServerStats),
                   rfi.RfiServerDesc.memory_budget.offset, rfi.RfiRequestDesc.abs0.offset,
                   rfi.RfiServerStats.device_status.offset]


def test_server_invalid_arguments_fail_before_cuda():
    n = 2
    w = (ctypes.c_int32 * n)(1024, 0)
    d = rfi.RfiServerDesc(8, n, w, None, None, 4096, 3.0, 0, 0, 0, 1 << 30, 1, 0)
    assert rfi.rfi_server_create(d)[0] == rfi.RFI_ERR_INVALID_ARG
    w = (ctypes.c_int32 * n)(1024, 2048)
    d = rfi.RfiServerDesc(8, n, w, None, None, 1024, 3.0, 0, 0, 0, 1 << 30, 1, 0)  # ring < W
    assert rfi.rfi_server_create(d)[0] == rfi.RFI_ERR_INVALID_ARG
    starts = (ctypes.c_int64 * n)(0, 1000)  # not a multiple of W
    d = rfi.RfiServerDesc(8, n, w, None, starts, 1 << 16, 3.0, 0, 0, 0, 1 << 30, 1, 0)
    assert rfi.rfi_server_create(d)[0] == rfi.RFI_ERR_INVALID_ARG
    assert rfi.LIB.rfi_server_destroy(None) == rfi.RFI_OK


def test_mom_arguments_checked_before_cuda():
    lens = (ctypes.c_int64 * 1)(4096)
    wins = (ctypes.c_int32 * 1)(1024)
    h = ctypes.c_void_p()
    for kmom, flags, want in ((-1, 0, rfi.RFI_ERR_INVALID_ARG), ((1 << 20) + 1, 0, rfi.RFI_ERR_INVALID_ARG),
                              (4, rfi.RFI_PLAN_PER_STREAM, rfi.RFI_ERR_UNSUPPORTED)):
        d = rfi.RfiPlanDesc(8, 1, lens, wins, None, 3.0, 0, 0, 0, flags, None, kmom)
        assert rfi.LIB.rfi_plan_create(ctypes.byref(d), ctypes.byref(h)) == want
    assert rfi.LIB.rfi_stats_mom(None, None, None) == rfi.RFI_ERR_INVALID_ARG


@pytest.mark.parametrize("kw", [
    dict(bits=12), dict(flags=rfi.RFI_PLAN_PER_STREAM), dict(flags=rfi.RFI_PLAN_POWER), dict(mom_windows=16),
    dict(out_format=rfi.RFI_OUT_F16),
])
def test_write_flagged_unsupported_combinations_fail_before_cuda(kw):
    """The in-place form that writes back only changed chunks is 8-bit, batched, per-window MAD,
    without power metering or a fused output format."""
    args = dict(bits=8, stream_len=[4096], window_len=[1024], k=3.0, mode=0)
    flags = rfi.RFI_PLAN_WRITE_FLAGGED | kw.get("flags", 0)
    d = rfi.make_desc(kw.get("bits", 8), args["stream_len"], args["window_len"], args["k"], args["mode"],
                      flags=flags, mom_windows=kw.get("mom_windows", 0), out_format=kw.get("out_format", 0))
    st, h = rfi.rfi_plan_create(d)
    assert st == rfi.RFI_ERR_UNSUPPORTED and h is None
