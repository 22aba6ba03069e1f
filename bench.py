"""Benchmark: GSamples/s of bit-exact windowed median/MAD excision and its HBM roofline fraction.

Workload (one step): the 60-stream GWB-shaped batch, 60 streams x 2^26 int8 samples, window
16384, excised once for each of the 8 variants k in {3, 5} x {zero, constant 1, clip, noise
seed 7}: 8 calls, 32 Gi samples per step. Inputs (4 GiB) are larger than L2, so every call
streams from HBM.

Arms and keys of the JSON line:
  value       batched persistent kernel (CUDA graph, autotuned shape), device-resident buffers,
              CUDA events on the launching stream
  per_stream  the plain one-launch-per-stream form on the same data
  e2e         rfi_excise_host on pinned host buffers: host->device, kernel and device->host
              copies inside the timed region
  roofline    algorithmic bytes per launch / mean launch time of the persistent kernel, against
              the measured HBM copy bandwidth
  cpu_baseline  the CPU oracle on a bounded sample of the same workload (host cores)
--impl reference times the CPU oracle alone on the same workload (bounded sample per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GSamples/s excised (bit-exact) and % of HBM roofline, batched vs per-stream"
UNIT = "GSamples/s"
PROFILE = os.path.join(ROOT, "profiles", "persistent_kernel_gwb60.md")
KERNEL_SOURCES = ["core.cuh", "kernels_impl.cuh", "kernels8.cu"]


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def workload_desc(nstreams, length):
    return ("gwb60: %d streams x 2^%d int8 samples, window 16384, k {3,5} x {zero, const 1, clip, "
            "noise seed 7} (8 calls per step)" % (nstreams, length.bit_length() - 1))


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        loaded = [s for s in sm if mx and s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for n in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1710_08576_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken on these sources."""
    if not os.path.exists(PROFILE):
        return None, "no profile"
    text = open(PROFILE).read()
    m1 = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    m2 = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    if not (m1 and m2):
        return None, "profile without traffic"
    if m2.group(1) != kernel_source_hash():
        return None, "kernel changed since the profile"
    return int(m1.group(1)), "ncu"


def cpu_oracle_sample(xs, variants, windows_per_stream, W):
    """Run the oracle on the first windows_per_stream windows of every stream for every variant,
    one stream per host core at a time; returns (samples, seconds, threads)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    threads = os.cpu_count() or 1
    parts = [x[: windows_per_stream * W] for x in xs]

    def one(args):
        v, i = args
        oracle.excise(parts[i], W, v.k, v.mode, const=v.const, seed=v.seed, stream_id=i, threads=1,
                      want=("z", "mask", "counts"))
        return parts[i].size

    jobs = [(v, i) for v in variants for i in range(len(parts))]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        n = sum(ex.map(one, jobs))
    return n, time.perf_counter() - t0, threads


# ------------------------------------------------------------------ arms
def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    import synth
    from synth import workloads
    w = workloads.gwb60(length=args.length, nstreams=args.streams)
    wps = args.ref_windows
    xs = [synth.fill(s.feed, s.index, wps * 16384) for s in w.streams]
    for _ in range(args.warmup):
        cpu_oracle_sample(xs[:2], w.variants[:1], 1, 16384)
    tot_n, tot_t, threads = 0, 0.0, 1
    for _ in range(args.steps):
        n, t, threads = cpu_oracle_sample(xs, w.variants, wps, 16384)
        tot_n += n
        tot_t += t
    value = tot_n / tot_t / 1e9
    sample = ("oracle (std::sort median/MAD) on the first %d windows of each of the %d streams, all 8 "
              "variants per step" % (wps, len(xs)))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
            "data": "synthetic", "config": {"workload": workload_desc(len(xs), args.length)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_1710_08576_gb300 as rfi
    import synth
    from synth import workloads

    from paper_1710_08576_gb300 import dist as rdist

    rank, local, world = rdist.env_rank()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    group = rdist.Group("nccl" if world > 1 else None, device=dev)
    barrier, max_over_ranks, sum_over_ranks = group.barrier, group.max, group.sum

    W = 16384
    w = workloads.gwb60(length=args.length, nstreams=args.streams)
    # each rank excises its own 60-stream batch (a different antenna set): weak scaling
    sids = rdist.stream_ids(rank, len(w.streams))
    t_gen = time.perf_counter()
    xs = [synth.fill(s.feed, sid, s.length) for s, sid in zip(w.streams, sids)]
    t_gen = time.perf_counter() - t_gen
    S = len(xs)
    lens = [x.size for x in xs]
    dev_in = [torch.from_numpy(x).to(dev) for x in xs]
    out = [torch.empty_like(t) for t in dev_in]
    nwin = [-(-n // W) for n in lens]
    masks = [torch.empty(nw * (W // 32), dtype=torch.int32, device=dev) for nw in nwin]
    counts = [torch.empty(nw, dtype=torch.int32, device=dev) for nw in nwin]
    samples_per_call = sum(lens)
    windows_per_call = sum(nwin)
    stream = torch.cuda.Stream(device=dev)

    batched = [rfi.Plan(8, lens, [W] * S, v.k, v.mode, v.const, v.seed,
                        rfi.RFI_PLAN_GRAPH | rfi.RFI_PLAN_AUTOTUNE, sids)
               for v in w.variants]
    per_stream = [rfi.Plan(8, lens, [W] * S, v.k, v.mode, v.const, v.seed, rfi.RFI_PLAN_PER_STREAM, sids)
                  for v in w.variants]
    info = batched[0].info()

    def timed(plans, steps, warmup, per_call_events=True):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                for p in plans:
                    p.excise(dev_in, out, masks, counts, stream)
            stream.synchronize()
            barrier()
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps * len(plans))]
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            j = 0
            for _ in range(steps):
                for p in plans:
                    ev[j][0].record(stream)
                    p.excise(dev_in, out, masks, counts, stream)
                    ev[j][1].record(stream)
                    j += 1
            e1.record(stream)
            stream.synchronize()
        barrier()
        torch.cuda.synchronize()
        total_ms = e0.elapsed_time(e1)
        calls = [a.elapsed_time(b) for a, b in ev]
        for p in plans:
            st, _ = p.stats(stream=stream)
            if st != 0:
                raise RuntimeError("device status %s" % rfi.rfi_status_string(st))
        return total_ms, calls

    clocks = ClockSampler(local)
    clocks.start()
    total_ms, calls = timed(batched, args.steps, args.warmup)
    clocks_b = clocks.stop()
    total_ms = max_over_ranks(total_ms)
    ps_steps = max(1, args.steps // 4)
    ps_ms, ps_calls = timed(per_stream, ps_steps, min(args.warmup, 2))
    ps_ms = max_over_ranks(ps_ms)

    samples_all = sum_over_ranks(samples_per_call * len(batched) * args.steps)
    value = samples_all / (total_ms * 1e-3) / 1e9
    ps_value = sum_over_ranks(samples_per_call * len(per_stream) * ps_steps) / (ps_ms * 1e-3) / 1e9

    # roofline of the persistent kernel: algorithmic bytes per launch / mean launch time
    alg_bytes = samples_per_call * (2 + 1 / 8) + windows_per_call * 12
    mean_call_s = statistics.mean(calls) * 1e-3
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / mean_call_s / 1e9
    traffic, traffic_src = profiled_traffic()
    ps_mean_s = statistics.mean(ps_calls) * 1e-3 / S   # per launch (one stream)
    ps_achieved = (alg_bytes / S) / ps_mean_s / 1e9

    # end to end through rfi_excise_host with pinned host buffers
    e2e = None
    if not args.no_e2e:
        h_in = [torch.from_numpy(x).pin_memory() for x in xs]
        h_out = [torch.empty_like(t).pin_memory() for t in h_in]
        h_mask = [torch.empty(nw * (W // 32), dtype=torch.int32).pin_memory() for nw in nwin]
        h_cnt = [torch.empty(nw, dtype=torch.int32).pin_memory() for nw in nwin]
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        for p in batched[:1]:
            p.excise_host(h_in, h_out, h_mask, h_cnt, stream)
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for p in batched:
                p.excise_host(h_in, h_out, h_mask, h_cnt, stream)
        torch.cuda.synchronize()
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
        h2d = samples_per_call * len(batched)
        d2h = (samples_per_call + sum(m.numel() * 4 for m in h_mask) + windows_per_call * 4) * len(batched)
        e2e = {"value": sum_over_ranks(samples_per_call * len(batched) * e2e_steps) / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps,
               "path": "rfi_excise_host, pinned host buffers, 32 MiB chunks on 3 streams"}
        del h_in, h_out, h_mask, h_cnt

    # CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        n, t, threads = cpu_oracle_sample(xs, w.variants, args.cpu_windows, W)
        cpu = {"value": n / t / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "first %d windows of each of the %d streams, all 8 variants (%d samples, %.1f s)"
                         % (args.cpu_windows, S, n, t)}

    for p in batched + per_stream:
        p.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": {"workload": workload_desc(S, args.length), "streams": S, "samples_per_stream": args.length,
                       "window": W, "variants": len(batched),
                       "form": "batched persistent kernel, CUDA graph, autotuned launch shape",
                       "launch_shape": {"consumer_warps": info.shape.consumer_warps, "stages": info.shape.stages,
                                        "ctas_per_sm": info.shape.ctas_per_sm,
                                        "stage_bytes": info.shape.stage_bytes,
                                        "dynamic_tiles": info.shape.dynamic_tiles, "groups": info.shape.groups,
                                        "grid": info.grid},
                       "l2": "inputs (%d MiB per rank) larger than L2 (129 MB)" % (samples_per_call >> 20),
                       "parallelism": "replicas (one 60-stream batch per GPU)", "feed_gen_s": round(t_gen, 2)},
            "per_stream": {"value": ps_value, "unit": UNIT, "ms_per_step": ps_ms / ps_steps, "steps": ps_steps,
                           "achieved_gbs": ps_achieved, "frac": ps_achieved / peak,
                           "launches_per_call": S},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "traffic_source": traffic_src,
                         "algorithmic_bytes_per_launch": int(alg_bytes),
                         "bytes_rule": "per sample 1 read + 1 write + 1/8 mask; per window 4 count + 8 M/D",
                         "mean_launch_ms": statistics.mean(calls), "kernel": "persistent_kernel<8,mode,cw>"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": len(batched) * args.steps,
            "clocks": clocks_b,
        }
        print(json.dumps(line), flush=True)
    group.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--streams", type=int, default=60)
    ap.add_argument("--length", type=int, default=1 << 26)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--ref-windows", type=int, default=8)
    ap.add_argument("--cpu-windows", type=int, default=32)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
