#!/usr/bin/env python
"""Throughput of the PRUNE firing path on B300: graph Msamples/s.

One step fires the whole hot path (FIR with delay line, DET, SEL, HX_b,
SINK) over the whole synthetic stream of the workload (default: the plain
graph with 1000 frames of F = 4096 blocks x B = 1024 complex64 samples,
T = 64 taps, H 32 x 32, tau = 4B, burst fraction U(0.1, 0.9) per frame).
Inputs are resident in HBM (32 GiB per step, far above the 126 MB L2, so no
L2 flush is needed) and pushed into f0 by reference; results stay in the
result ring.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank fires its own graph instance (independent streams,
instance sharding with no collective: weak scaling); rank 0 prints the line
with the samples of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1802_06625_b300 import synth  # noqa: E402

METRIC = "graph Msamples/s + % HBM roofline on 1 B300, batched vs plain; p99 latency"
# DRAM bytes (read + write) per frame of the 4096 x 1024 workload, per kernel
# name, from one ncu capture of the kernel as it stands (48-frame launch of
# the warp-specialised loop: 1611.218 MB read + 813.758 MB written, divided
# by 48); scaled to a launch by the frames it fires.  Remove an entry when
# its kernel changes.
TRAFFIC_PER_FRAME = {"firing_loop_ws_kernel": (1611.218e6 + 813.758e6) / 48}
UNIT = "Msamples/s"
# FP32 FFMA peak from the unit counts and clock of the part: 148 SMs x 128
# FP32 lanes x 2 flop x 2.032 GHz.
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
KIND_NAMES = {0: "f0_push_kernel", 1: "fir_energy_kernel", 2: "det_sel_kernel", 3: "hx_cuda_kernel",
              4: "hx_tc_kernel", 5: "firing_loop_kernel", 6: "firing_loop_tc_kernel"}
NKINDS = 7


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_description():
    """The host the CPU baseline ran on: its logical CPUs and CPU model."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        torch.distributed.barrier()


def max_over_ranks(v, ws, dev):
    if ws == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, ws, dev):
    if ws == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t)
    return float(t.item())


# ------------------------------------------------------------------ oracle

def oracle_sample(w, frames, first=0, instance=0):
    """Time the FP64 oracle on `frames` frames of the workload (the delay
    token before the first frame comes from the input).  Returns
    (Msamples/s, seconds, frames)."""
    import oracle
    oracle.build()
    xs = w.frames_tensor(first, frames, instance=instance).numpy()
    hist = None
    if first > 0 and w.T > 1:
        hist = w.frame(first - 1, instance=instance).numpy().reshape(-1)[-(w.T - 1):].astype(np.complex128)
    taps, H = w.taps(instance=instance).numpy(), w.H(instance=instance).numpy()
    t0 = time.perf_counter()
    oracle.run(w.F, w.B, w.T, w.N, np.float32(w.tau), taps, H, xs, C=w.C, hist_in=hist)
    dt = time.perf_counter() - t0
    return frames * w.F * w.B / dt / 1e6, dt, frames


def run_reference(args, w):
    """--impl reference: the oracle, as it stands, timed on the host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    per_step = args.ref_frames
    for _ in range(args.warmup):
        oracle_sample(w, per_step, first=0)
    t = 0.0
    for s in range(args.steps):
        _, dt, _ = oracle_sample(w, per_step, first=1 + s)
        t += dt
    value = args.steps * per_step * w.F * w.B / t / 1e6
    sample = f"{per_step} frame(s) of {w.name} per step, single-threaded FP64 C oracle"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 + Box-Muller)",
            "config": {"workload": w.name, "F": w.F, "B": w.B, "T": w.T, "N": w.N, "frames_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_description()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours

def make_inputs(w, frames, dev, instance):
    x = torch.empty(frames, w.F, w.B, dtype=torch.complex64, device=dev)
    for k in range(frames):
        x[k] = w.frame(k, device=dev, instance=instance)
    return x


def run_ours(args, w):
    from paper_1802_06625_b300 import _lib
    from paper_1802_06625_b300.graph import Graph

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        torch.distributed.init_process_group("nccl", device_id=dev)

    frames = args.frames or w.frames
    C = args.C
    x = make_inputs(w, frames, dev, instance=rank)
    stream = torch.cuda.Stream(device=dev)
    g = Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(instance=rank), w.H(instance=rank), C=C, out_frames=frames,
              stream=stream, device=local)
    L = w.F * w.B

    actors, cuda_cores = args.path == "actors", args.path == "cuda_cores"

    def step():
        for k in range(0, frames, C):
            m = min(C, frames - k)
            g.push(x[k:k + m], mem=_lib.PRUNE_MEM_DEVICE_BORROW)
            g.run(actors=actors, cuda_cores=cuda_cores)
        g.discard()

    for _ in range(args.warmup):
        step()
    g.sync()
    # selected blocks per step (the same every step: the same frames)
    for k in range(0, frames, C):
        m = min(C, frames - k)
        g.push(x[k:k + m], mem=_lib.PRUNE_MEM_DEVICE_BORROW)
        g.run(actors=actors, cuda_cores=cuda_cores)
    recs = (_lib.prune_frame_out * frames)()
    nrec = ctypes.c_int32()
    _lib.check(_lib.lib().prune_pull(g.h, recs, frames, ctypes.byref(nrec), _lib.PRUNE_MEM_DISCARD), g.h)
    selected_blocks = sum(recs[i].c for i in range(nrec.value))
    g.profile(True)
    for kind in range(NKINDS):
        g.kernel_times(kind, reset=True)

    barrier(ws)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    barrier(ws)
    ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
    times = {k: g.kernel_times(k, reset=True) for k in range(NKINDS)}
    g.profile(False)
    launches = sum(n for _, n in times.values())
    samples = sum_over_ranks(float(args.steps * frames * L), ws, dev)
    value = samples / (ms / 1e3) / 1e6

    # dominant kernel and its roofline (algorithmic work per launch / avg duration)
    kind, (kms, kn) = max(times.items(), key=lambda kv: kv[1][0])
    # kind 6 is the warp-specialised loop when T <= 65 (at most 3 tap shifts)
    # unless PRUNE_TC_KERNEL=pipes selects the tile-pipeline loop
    ws_loop = os.environ.get("PRUNE_TC_KERNEL", "") != "pipes" and 1 + (w.T - 1 + 31) // 32 <= 3

    def kind_name(k):  # the kernel that ran for a timing kind
        return "firing_loop_ws_kernel" if k == 6 and ws_loop else KIND_NAMES[k]

    peaks = measured_peaks()
    runs = args.steps * ((frames + C - 1) // C)
    roof = None
    sel_frac = selected_blocks / float(frames * w.F)
    if kn:
        avg_s = kms / kn / 1e3
        frames_per_launch = args.steps * frames / kn
        samples = L * frames_per_launch
        if kind in (1, 5):  # CUDA-core FIR (+HX): 8T (+8N per selected sample) FP32 flop per sample
            work = (8.0 * w.T + (8.0 * w.N * sel_frac if kind == 5 else 0.0)) * samples
            roof = {"bound": "alu", "achieved": work / avg_s / 1e12, "peak": FP32_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 x 2.032 GHz"}
        else:               # bytes the path must move: frames in, selected blocks + indices out
            nbytes = 8.0 * samples + (8.0 * w.B + 4.0) * w.F * sel_frac * frames_per_launch
            if kind == 2:
                nbytes = 8.0 * w.F * frames_per_launch
            roof = {"bound": "hbm", "achieved": nbytes / avg_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "peak_source": "measured" if not peaks.get("fallback") else "fallback"}
            if kind == 6:   # tensor pipe: split-FP16 FIR (ns shifts) + HX
                ns = 1 + (w.T - 1 + 31) // 32
                if ws_loop:
                    # per 128-row tile: ns x 4 K steps x (128 x 128 x 16 + 128 x 64 x 16) (FIR), 3 passes
                    # x 4 K steps of 128 x 64 x 16 (HX on all rows): per sample (ns + 1) * 768 flop
                    per_sample, note = (ns + 1) * 768.0, ("FIR per K step as hi x [taps hi | lo] (N=128) and lo x taps hi "
                                                          "(N=64), HX 3 passes on all rows")
                else:
                    # 3 passes x 4 K steps of 128 x 64 x 16 per shift (FIR), HX on the selected rows
                    per_sample, note = (ns + sel_frac) * 768.0, "FIR and HX in 3 split passes, HX on the selected rows"
                tflop = samples * per_sample / 1e12
                peak_t = peaks.get("bf16_tflops_sustained", 1400.0)
                roof["tensor"] = {"achieved": tflop / avg_s, "peak": peak_t, "unit": "TFLOP/s",
                                  "frac": tflop / avg_s / peak_t,
                                  "note": "FP16 MMA work: " + note + "; peak = measured BF16 sustained "
                                          "(FP16 has the same nominal rate)"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        traffic = args.traffic
        if traffic is None and kind_name(kind) in TRAFFIC_PER_FRAME and w.name == synth.PLAIN_LARGE.name:
            traffic = TRAFFIC_PER_FRAME[kind_name(kind)] * frames_per_launch
        roof["traffic"] = traffic
        roof["kernel"] = kind_name(kind)
        roof["avg_launch_ms"] = kms / kn
        roof["share"] = kms / max(sum(t for t, _ in times.values()), 1e-12)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded SplitMix64 + Box-Muller, generated on device)",
            "config": {"workload": w.name, "F": w.F, "B": w.B, "T": w.T, "N": w.N, "tau": w.tau,
                       "frames_per_step": frames, "C": C, "path": args.path,
                       "selected_fraction": sel_frac,
                       "l2": "inputs larger than L2 (%.1f GiB per step), no flush" % (frames * L * 8 / 2**30),
                       "parallelism": f"instance-sharded x{ws}" if ws > 1 else "single instance"},
            "roofline": roof, "gpu_launches": launches,
            "kernel_ms_per_step": {kind_name(k): t / args.steps for k, (t, n) in times.items() if n},
            "clocks": clk.summary()}

    # the batched form: one frame of each of 512 uneven instances per step
    del g
    if not args.no_batched and ws == 1:
        line["batched"] = run_batched(args, dev)

    # the Dynamic Predistortion stream
    if not args.no_dpd and ws == 1:
        line["dpd"] = run_dpd(args, dev)

    # the 100-frame plain workload: throughput and per-frame latency
    if not args.no_small and ws == 1:
        line["plain_small"] = run_plain_small(args, dev)

    # differentiation over the control trace: forward / backward, store vs recompute
    if not args.no_diff and ws == 1:
        line["differentiation"] = run_differentiation(args, dev)

    # the request loop: Poisson stream arrivals, admission by HBM budget
    if not args.no_serving and ws == 1:
        line["serving"] = run_serving(args, dev)

    # end to end through the public API: host frames in, host records out
    line["e2e"] = run_e2e(args, w, dev, stream, rank, ws)

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, dt, nf = oracle_sample(w, args.cpu_frames, first=0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {nf} frame(s) of {w.name}, single-threaded FP64 C oracle, {dt:.1f} s",
                                "host": host_description()}
        if w.name == synth.PLAIN_LARGE.name:  # the plain-small stream, timed in full
            ws_ = synth.PLAIN_SMALL
            v1, dt1, nf1 = oracle_sample(ws_, ws_.frames, first=0)
            line["cpu_baseline"]["plain_small"] = {
                "value": v1, "unit": UNIT, "cores": 1,
                "sample": f"all {nf1} frames of {ws_.name}, single-threaded FP64 C oracle, {dt1:.2f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_batched(args, dev, compare_plain=True):
    """Batched (one launch sequence for all instances, replayed as a CUDA
    graph) against plain (one graph object per instance, fired one by one),
    same frames, wall clock over K steps with the device synchronized."""
    from paper_1802_06625_b300 import _lib
    from paper_1802_06625_b300.graph import Batch, Graph

    b = synth.BATCHED
    ws_ = [b.instance(i) for i in range(b.instances)]
    x = torch.cat([w.frame(0, device=dev).reshape(-1) for w in ws_])
    insts = [{"F": w.F, "T": w.T, "tau": w.tau, "taps": w.taps(), "H": w.H()} for w in ws_]
    samples = x.numel()
    stream = torch.cuda.Stream(device=dev)
    bt = Batch(b.B, b.N, insts, stream=stream, device=dev.index)
    tuned, candidates = bt.autotune(x, reps=3)   # launch shape picked by timing every candidate
    for _ in range(args.warmup):
        bt.fire(x, graph=True)
    bt.sync()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bt.fire(x, graph=True)
    bt.sync()
    t_batched = (time.perf_counter() - t0) / args.steps
    # algorithmic bytes of the step, as for the plain line: every input
    # sample read once (8 B), every selected block written once with its
    # index (8 B + 4 B per block); the bytes the three launches actually move
    # (the FIR output written and read back between launches, energies) are
    # reported beside them
    sel_blocks = sum(bt.pull(i)[1] for i in range(b.instances))
    sel_samples = sel_blocks * b.B
    blocks = sum(w.F for w in ws_)
    step_bytes = 8.0 * samples + (8.0 * b.B + 4.0) * sel_blocks
    moved_bytes = 16.0 * samples + 16.0 * sel_samples + 8.0 * blocks + 4.0 * sel_blocks
    peaks = measured_peaks()
    roof = {"bound": "hbm", "achieved": step_bytes / t_batched / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "peak_source": "measured" if not peaks.get("fallback") else "fallback",
            "frac": step_bytes / t_batched / 1e9 / peaks["hbm_gbs"], "bytes_per_step": step_bytes,
            "moved_bytes_per_step": moved_bytes, "moved_GBs": moved_bytes / t_batched / 1e9,
            "selected_fraction": sel_samples / float(samples),
            "note": "algorithmic bytes (8 B per input sample + (8B + 4) B per selected block) over the whole "
                    "step's time, against the HBM copy bandwidth; moved_* counts the FIR output's round trip "
                    "between the launches too"}
    bt_off = list(bt.offsets)
    bt.close()
    # blocks of the timed frame whose decision lies inside the parity guard
    # band (|E - tau| <= 1e-3 |tau|, where either decision is correct), by T,
    # from the FP32 block energies of the CUDA-core FIR (untimed)
    from paper_1802_06625_b300.graph import fir_energy
    band = {f"T={t}": 0 for t in sorted({w.T for w in ws_})}
    for i, w in enumerate(ws_):
        _, e, _ = fir_energy(x[bt_off[i]:bt_off[i] + w.F * w.B].reshape(1, -1), w.taps(), w.F, w.B, w.T,
                             want_y=False)
        band[f"T={w.T}"] += int((torch.abs(e.double() - w.tau) <= 1e-3 * abs(w.tau)).sum())
    in_band = {**band, "seed": b.seed, "blocks": blocks,
               "note": "blocks with |E - tau| <= 1e-3 |tau| by the FP32 energies of the CUDA-core FIR"}
    out = {"workload": b.name, "instances": b.instances, "samples_per_step": samples, "launches_per_step": 3,
           "batched_Msamples_s": samples / t_batched / 1e6, "batched_ms_per_step": 1e3 * t_batched,
           "roofline": roof, "in_band_blocks": in_band, "tuning": tuned,
           "candidates_ms": [round(c["ms"], 4) for c in candidates]}
    if not compare_plain:
        return out

    # plain with the same tensor-core kernels: one single-instance batch per
    # instance, (a) fired one by one from the host (each its own CUDA-graph
    # replay of its three launches), (b) all 512 x 3 launches captured in one
    # CUDA graph, so that the batching gain is measured apart from the host
    # launch cost
    offs = []
    for i in range(b.instances):
        offs.append(bt_off[i])
    cs = torch.cuda.Stream(device=dev)
    singles = [Batch(b.B, b.N, [insts[i]], stream=cs, device=dev.index) for i in range(b.instances)]
    xs = [x[offs[i]:offs[i] + ws_[i].F * ws_[i].B] for i in range(b.instances)]

    def single_launches():
        for sb, xi in zip(singles, xs):
            sb.fire(xi, graph=True)

    for _ in range(args.warmup):
        single_launches()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        single_launches()
    torch.cuda.synchronize(dev)
    t_single = (time.perf_counter() - t0) / args.steps
    for sb, xi in zip(singles, xs):       # one untimed pass outside the capture
        sb.fire(xi, graph=False)
    torch.cuda.synchronize(dev)
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=cs):
        for sb, xi in zip(singles, xs):
            sb.fire(xi, graph=False)
    for _ in range(args.warmup):
        cg.replay()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cg.replay()
    torch.cuda.synchronize(dev)
    t_one_graph = (time.perf_counter() - t0) / args.steps
    del cg
    for sb in singles:
        sb.close()
    out.update({"plain_tc_launches_ms_per_step": 1e3 * t_single, "plain_tc_one_graph_ms_per_step": 1e3 * t_one_graph,
                "speedup_vs_plain_tc_launches": t_single / t_batched,
                "speedup_vs_plain_tc_one_graph": t_one_graph / t_batched})

    graphs = [Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=1, out_frames=1, device=dev.index) for w in ws_]
    offs, o = [], 0
    for w in ws_:
        offs.append(o)
        o += w.F * w.B

    def plain_step():
        for g, w, off in zip(graphs, ws_, offs):
            g.push(x[off:off + w.F * w.B].view(1, w.F, w.B), mem=_lib.PRUNE_MEM_DEVICE_BORROW)
            g.run()
            g.discard()

    for _ in range(args.warmup):
        plain_step()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plain_step()
    torch.cuda.synchronize(dev)
    t_plain = (time.perf_counter() - t0) / args.steps
    for g in graphs:
        g.close()
    return {**out, "plain_Msamples_s": samples / t_plain / 1e6, "plain_ms_per_step": 1e3 * t_plain,
            "speedup": t_plain / t_batched,
            "timing": "wall clock over K steps, device synchronized; batched = 3 launches replayed as one CUDA "
                      "graph with the autotuned launch shape; plain = one graph object per instance (push, run, "
                      "drop per step; the actor path, FIR on CUDA cores at N = 64); plain_tc = the same "
                      "tensor-core kernels one instance per launch, fired from the host or captured as one graph"}


def run_dpd(args, dev):
    """The 67 M-sample DPD stream (1024 periods of 65536 samples, 10 branches
    of 10 taps, 2..10 active per period) fired in one call per step, the
    delay tokens carried in place; CUDA events on the current stream."""
    from paper_1802_06625_b300 import dpd

    w = synth.DPD
    masks = w.masks()
    taps = w.taps()
    x = w.x(device=dev)
    y = torch.empty_like(x)
    h = torch.zeros(w.K, w.T - 1, dtype=torch.complex64, device=dev)
    for _ in range(args.warmup):
        dpd.fire(x, masks, taps, w.period, hist=h, hist_out=h, y=y)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        dpd.fire(x, masks, taps, w.period, hist=h, hist_out=h, y=y)
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    active = sum(bin(int(m)).count("1") for m in masks)
    flops = active * w.period * 8.0 * w.T               # complex MACs of the active branches
    samples = w.periods * w.period
    return {"workload": w.name, "samples_per_step": samples, "Msamples_s": samples / (ms * 1e-3) / 1e6,
            "ms_per_step": ms, "mean_active_branches": active / w.periods,
            "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                         "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 x 2.032 GHz",
                         "hbm_GBs": 16.0 * samples / (ms * 1e-3) / 1e9},
            "paper": "PRUNE heterogeneous 106 Msamples/s on the RX platform (Table 4), other hardware: context only"}


def serve_once(args, dev, streams, lam, host_inputs=False):
    """Streams arrive on the host clock as a Poisson process of rate lam;
    each is admitted when a slot and room in the 40 GB budget are free, its
    frames queued as one request, and every step fires the next frames of
    all admitted streams.  Latency of a stream = observed completion of its
    last frame - arrival.  host_inputs: a request's distinct frames (its
    period of the pool) start in pinned host memory and are copied to the
    device at admission, on the server's stream, inside the latency."""
    from paper_1802_06625_b300.serve import Server

    sw = synth.ServingWorkload(**{**synth.SERVING.__dict__, "streams": streams, "lam": lam})
    specs = [sw.stream(i) for i in range(sw.streams)]
    arr = sw.arrivals()
    params = [(sw.taps(i).numpy(), sw.H(i).numpy()) for i in range(sw.streams)]
    pool = sw.pool_tensor(device=dev)
    pool_h = pool.cpu().pin_memory() if host_inputs else None
    fps = args.serve_fps
    sstream = torch.cuda.Stream(device=dev)
    srv = Server(sw.B, sw.N, F_max=sw.F_hi, T_max=sw.T, max_streams=args.serve_slots,
                 hbm_budget=int(args.serve_budget_gb * 2**30), frames_per_step=fps, ring=2 * fps,
                 max_inflight=args.serve_inflight, auto_release=True, stream=sstream, device=dev.index)

    def inputs(sp):
        L = sp["F"] * sw.B
        lo, hi = sp["offset"], sp["offset"] + sp["period"] * L
        if not host_inputs:
            return pool[lo:hi]
        buf = torch.empty(hi - lo, dtype=torch.complex64, device=dev)
        with torch.cuda.stream(sstream):
            buf.copy_(pool_h[lo:hi], non_blocking=True)
        return buf

    # warm-up: one short stream end to end
    sid = srv.open(specs[0]["F"], sw.T, specs[0]["tau"], *params[0])
    srv.submit(sid, inputs(specs[0])[:specs[0]["F"] * sw.B], n=2 * fps, period=1)
    while srv.step():
        pass
    srv.sync()
    srv.poll()
    srv.close(sid)
    srv.sync()

    h2d = 0
    t0 = time.monotonic_ns()
    due = [t0 + int(a * 1e9) for a in arr]
    waiting, nxt, done_at, admitted_at, sid_of = [], 0, {}, {}, {}
    peak_open, steps, entries = 0, 0, 0
    while len(done_at) < sw.streams:
        now = time.monotonic_ns()
        while nxt < sw.streams and due[nxt] <= now:
            waiting.append(nxt)
            nxt += 1
        while waiting:                                   # admission in arrival order
            i = waiting[0]
            sp = specs[i]
            sid = srv.open(sp["F"], sw.T, sp["tau"], *params[i])
            if sid is None:
                break
            waiting.pop(0)
            sid_of[sid] = i
            admitted_at[i] = time.monotonic_ns()
            xin = inputs(sp)
            if host_inputs:
                h2d += xin.numel() * 8
            srv.submit(sid, xin, n=sp["frames"], period=sp["period"])
        peak_open = max(peak_open, len(sid_of))
        n = srv.step()
        if n:
            steps += 1
            entries += n
        for sid, t_ns in srv.poll():
            done_at[sid_of.pop(sid)] = t_ns
            srv.close(sid)
        if n == 0:
            if sid_of:
                srv.sync()                               # only steps in flight: wait for them
            elif nxt < sw.streams:
                time.sleep(max(0.0, (due[nxt] - time.monotonic_ns()) * 1e-9))
    srv.sync()
    t1 = max(done_at.values())
    srv.close_server()
    lat = np.array([(done_at[i] - due[i]) * 1e-6 for i in range(sw.streams)])
    wait = np.array([(admitted_at[i] - due[i]) * 1e-6 for i in range(sw.streams)])
    samples = sum(sp["frames"] * sp["F"] * sw.B for sp in specs)
    out = {"streams": sw.streams, "lambda_per_s": sw.lam, "samples": samples,
           "offered_Msamples_s": samples / max(arr[-1], 1e-9) / 1e6,
           "Msamples_s": samples / ((t1 - t0) * 1e-9) / 1e6, "makespan_s": (t1 - t0) * 1e-9,
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())},
           "admission_wait_ms": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
           "steps": steps, "entries_per_step": entries / max(steps, 1), "peak_open_streams": peak_open}
    if host_inputs:
        out["h2d_bytes"] = h2d
    return out


def run_serving(args, dev):
    """The request loop on the serving workload: the fixed trace of the
    first second of arrivals at 2000 streams/s (offered load about twice what
    one GPU sustains, so latencies include queueing), then a run at 0.7 of
    the saturation rate measured on the trace, with inputs resident and with
    inputs copied from host memory per request."""
    trace = serve_once(args, dev, args.serve_streams, synth.SERVING.lam)
    sw = synth.ServingWorkload(**{**synth.SERVING.__dict__, "streams": args.serve_streams_07})
    mean_samples = np.mean([sp["frames"] * sp["F"] * sw.B for sp in (sw.stream(i) for i in range(sw.streams))])
    lam_sat = trace["Msamples_s"] * 1e6 / mean_samples          # streams/s the GPU sustains
    lam07 = 0.7 * lam_sat
    r07 = serve_once(args, dev, args.serve_streams_07, lam07)
    r07h = serve_once(args, dev, args.serve_streams_07, lam07, host_inputs=True)
    return {"workload": synth.SERVING.name, "trace_streams": trace["streams"],
            "frames_per_stream": "log-uniform [10, 10^4]", "F": "uniform [64, 2048]",
            **trace, "lambda_saturation_per_s": lam_sat,
            "lambda_0p7_sat": {**r07, "host_inputs": r07h},
            "frames_per_step": args.serve_fps, "hbm_budget_GB": args.serve_budget_gb, "slots": args.serve_slots,
            "steps_in_flight": args.serve_inflight,
            "timing": "host monotonic clock; arrival = scheduled Poisson time, completion = when the host saw "
                      "the stream's last step complete; saturation rate = trace throughput / mean samples per "
                      "stream of the 0.7 run's streams"}


def run_plain_small(args, dev):
    """The 100-frame plain workload (64 blocks x 256 samples, T = 16, H
    16 x 16; the CUDA-core fused loop, N < 32): throughput over the whole
    stream (frames resident on the device, pushed by reference, one launch,
    CUDA events on the graph's stream), and the latency of one frame from
    the host: pushed from pinned host memory, fired, its record pulled into
    pinned host memory, one frame at a time (host clock, device synchronized
    by the pull)."""
    from paper_1802_06625_b300 import _lib
    from paper_1802_06625_b300.graph import Graph

    w = synth.PLAIN_SMALL
    n = w.frames
    x = torch.stack([w.frame(k, device=dev) for k in range(n)])
    stream = torch.cuda.Stream(device=dev)
    g = Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=n, out_frames=n, stream=stream, device=dev.index)

    def step():
        g.push(x, mem=_lib.PRUNE_MEM_DEVICE_BORROW)
        g.run()
        g.discard()

    for _ in range(args.warmup):
        step()
    g.sync()
    reps = max(args.steps, 20)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    g.close()

    # one frame at a time from the host
    xh = x.cpu().pin_memory()
    g = Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=3, out_frames=3, stream=stream, device=dev.index)
    lib = _lib.lib()
    ih = torch.empty(w.F, dtype=torch.int32).pin_memory()
    yh = torch.empty(w.F, w.B, dtype=torch.complex64).pin_memory()
    rec = (_lib.prune_frame_out * 1)()
    rec[0].idx, rec[0].y = ih.data_ptr(), yh.data_ptr()
    cnt = ctypes.c_int32()
    lat = []
    for rep in range(3):
        for k in range(n):
            t0 = time.perf_counter()
            _lib.check(lib.prune_push_frames(g.h, xh[k].data_ptr(), 1, _lib.PRUNE_MEM_HOST), g.h)
            g.run()
            _lib.check(lib.prune_pull(g.h, rec, 1, ctypes.byref(cnt), _lib.PRUNE_MEM_HOST), g.h)
            if rep > 0:
                lat.append((time.perf_counter() - t0) * 1e3)
    g.close()
    lat = np.array(lat)
    samples = n * w.F * w.B
    return {"workload": w.name, "samples_per_step": samples, "Msamples_s": samples / (ms * 1e-3) / 1e6,
            "ms_per_step": ms, "kernel": "firing_loop_kernel<16> (CUDA cores, N = 16)",
            "frame_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                 "frames": int(lat.size)},
            "note": "throughput: 100 device-resident frames per step in one launch (CUDA events, "
                    f"{reps} steps); latency: host push (pinned) -> run -> host pull of one frame"}


def run_differentiation(args, dev):
    """Forward and backward of the differentiation workload (100 frames of
    64 x 256 samples, T = 64, H 32 x 32, L2 loss against the sink output of
    the graph with the seed-5 parameters) through torch.autograd over the
    recorded control trace, with the FIR output stored or recomputed: CUDA
    events per phase, peak device memory per mode."""
    from paper_1802_06625_b300 import autodiff as AD

    w = synth.DIFF
    n = w.frames
    x = torch.stack([w.frame(k, device=dev).reshape(-1) for k in range(n)])
    taps0, H0 = w.taps().to(dev), w.H().to(dev)
    tt, Ht = synth.taps(synth.DIFF_TARGET_SEED, w.T).to(dev), synth.hmat(synth.DIFF_TARGET_SEED, w.N).to(dev)
    with torch.no_grad():
        out_t, c_t, idx_t = AD.fire(tt, Ht, x, F=w.F, B=w.B, T=w.T, N=w.N, tau=w.tau)
        target = AD.scatter(out_t, c_t, idx_t, w.F, w.B)
    res = {}
    for store in (True, False):
        fwd, bwd = [], []
        torch.cuda.synchronize(dev)
        torch.cuda.reset_peak_memory_stats(dev)
        base = torch.cuda.memory_allocated(dev)
        for it in range(args.warmup + max(args.steps, 10)):
            t = taps0.clone().requires_grad_(True)
            h = H0.clone().requires_grad_(True)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            out, c, idx = AD.fire(t, h, x, F=w.F, B=w.B, T=w.T, N=w.N, tau=w.tau, store=store)
            d = AD.scatter(out, c, idx, w.F, w.B) - target
            loss = (d.real.square() + d.imag.square()).sum()
            e1.record()
            loss.backward()
            e2.record()
            torch.cuda.synchronize(dev)
            if it >= args.warmup:
                fwd.append(e0.elapsed_time(e1))
                bwd.append(e1.elapsed_time(e2))
        res["store" if store else "recompute"] = {
            "forward_ms": float(np.median(fwd)), "backward_ms": float(np.median(bwd)),
            "peak_device_MB": (torch.cuda.max_memory_allocated(dev) - base) / 2**20}
    samples = n * w.F * w.B
    return {"workload": w.name, "samples_per_step": samples, **res,
            "Msamples_s_fwd_bwd_store": samples / ((res["store"]["forward_ms"] + res["store"]["backward_ms"]) * 1e-3) / 1e6,
            "note": "forward = FIR + DET/SEL + HX + scatter + loss; backward = HX and FIR adjoints (+ FIR "
                    "recompute when not stored); medians over the timed iterations"}


def copy_ceiling(xh, yh, d2h_bytes, dev, reps=3):
    """Plain pinned copies of one e2e step's bytes: the step's input host to
    device on one stream while its output bytes go device to host on
    another (the link is full duplex but the host side shares it).  The e2e
    step time over this one is the share of the box's copy ceiling."""
    xb = xh.view(torch.uint8).reshape(-1)
    yb = yh.view(torch.uint8).reshape(-1)[:d2h_bytes]
    din = torch.empty(xb.numel(), dtype=torch.uint8, device=dev)
    dout = torch.empty(max(1, yb.numel()), dtype=torch.uint8, device=dev)[:yb.numel()]
    si, so = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def both():
        with torch.cuda.stream(si):
            din.copy_(xb, non_blocking=True)
        with torch.cuda.stream(so):
            yb.copy_(dout, non_blocking=True)

    def alone():
        with torch.cuda.stream(si):
            din.copy_(xb, non_blocking=True)

    out = {}
    for name, fn in (("s_per_step", both), ("h2d_alone_s", alone)):
        fn()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize(dev)
        out[name] = (time.perf_counter() - t0) / reps
    out["h2d_alone_GBs"] = xb.numel() / out.pop("h2d_alone_s") / 1e9
    out["in_and_out_GBs"] = (xb.numel() + yb.numel()) / out["s_per_step"] / 1e9
    del din, dout
    return out


def run_e2e(args, w, dev, stream, rank, ws):
    from paper_1802_06625_b300 import _lib
    from paper_1802_06625_b300.graph import Graph

    E = args.e2e_frames
    C = args.C
    L = w.F * w.B
    xh = torch.empty(E, w.F, w.B, dtype=torch.complex64).pin_memory()
    for k in range(E):
        xh[k] = w.frame(k, device=dev, instance=rank).cpu()
    yh = torch.empty(E, w.F, w.B, dtype=torch.complex64).pin_memory()
    ih = torch.empty(E, w.F, dtype=torch.int32).pin_memory()
    g = Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(instance=rank), w.H(instance=rank), C=C, out_frames=C,
              stream=stream, device=dev.index)
    recs = (_lib.prune_frame_out * C)()
    lib = _lib.lib()

    # chunks of the step's frames, pipelined: chunk k is pushed and fired
    # before chunk k-1 is pulled, so a pull (its own stream, after the run
    # that fired it) overlaps the next chunk's host-to-device copy.  The
    # pipeline runs on across steps, as a stream's would: a step's last
    # chunk is pulled during the next step's first push, and the timed
    # region ends with the one pull still outstanding.
    ch = max(1, min(C // 2, 8, E))
    chunks = [(k, min(ch, E - k)) for k in range(0, E, ch)]
    pending = []

    def pull_chunk(k, m):
        for i in range(m):
            recs[i].idx = ih[k + i].data_ptr()
            recs[i].y = yh[k + i].data_ptr()
        n = ctypes.c_int32()
        _lib.check(lib.prune_pull(g.h, recs, m, ctypes.byref(n), _lib.PRUNE_MEM_HOST), g.h)
        return sum(recs[i].c * (w.B * 8 + 4) + 12 for i in range(n.value))

    def step():
        d2h = 0
        for k, m in chunks:
            _lib.check(lib.prune_push_frames(g.h, xh[k].data_ptr(), m, _lib.PRUNE_MEM_HOST), g.h)
            g.run()
            if pending:
                d2h += pull_chunk(*pending.pop())
            pending.append((k, m))
        return d2h

    def drain():
        return pull_chunk(*pending.pop()) if pending else 0

    for _ in range(max(1, args.warmup)):
        step()
    drain()
    barrier(ws)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(args.steps):
        d2h += step()
    d2h += drain()
    torch.cuda.synchronize(dev)
    dt = max_over_ranks(time.perf_counter() - t0, ws, dev)
    g.close()
    samples = sum_over_ranks(float(args.steps * E * L), ws, dev)
    d2h_step = d2h // args.steps
    ceiling = copy_ceiling(xh, yh, d2h_step, dev)
    ceiling["frac"] = ceiling["s_per_step"] / (dt / args.steps)
    return {"value": samples / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": E * L * 8,
            "d2h_bytes_per_step": d2h_step, "frames_per_step": E,
            "chunk_frames": ch, "copy_ceiling": ceiling,
            "note": "pinned host frames pushed (H2D) and records pulled (D2H) through the C ABI, in chunks "
                    "pipelined so that a chunk's pull overlaps the next chunk's push (across steps too; the "
                    "timed region ends with the last pull)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain_large", choices=["plain_large", "plain_small"])
    ap.add_argument("--frames", type=int, default=0, help="frames per step (default: the workload's)")
    ap.add_argument("--C", type=int, default=336,
                    help="buffering constant of eq. (2): frames f0 holds, hence frames one launch can fire")
    ap.add_argument("--path", default="fused", choices=["fused", "cuda_cores", "actors"],
                    help="fused loop (tensor cores where the shape allows), fused loop on CUDA cores, "
                         "or one kernel per actor")
    ap.add_argument("--e2e-frames", type=int, default=48)
    ap.add_argument("--cpu-frames", type=int, default=8)
    ap.add_argument("--ref-frames", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-loop measurement")
    ap.add_argument("--no-dpd", action="store_true", help="skip the DPD stream measurement")
    ap.add_argument("--no-small", action="store_true", help="skip the 100-frame plain-small measurement")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiation measurement")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched step (no plain comparison): a small process for profiling it")
    ap.add_argument("--dpd-only", action="store_true",
                    help="only the DPD stream: a small process for profiling it")
    ap.add_argument("--serve-streams", type=int, default=2000,
                    help="streams of the fixed trace (2000 = the first second of arrivals at 2000/s)")
    ap.add_argument("--serve-streams-07", type=int, default=400,
                    help="streams of the runs at 0.7 of the saturation rate")
    ap.add_argument("--serve-slots", type=int, default=256)
    ap.add_argument("--serve-fps", type=int, default=16, help="frames a stream advances per step")
    ap.add_argument("--serve-budget-gb", type=float, default=40.0)
    ap.add_argument("--serve-inflight", type=int, default=2, help="request-loop steps in flight")
    ap.add_argument("--traffic", type=float, default=None, help="ncu dram bytes per launch of the top kernel")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    w = synth.PLAIN_LARGE if args.workload == "plain_large" else synth.PLAIN_SMALL
    if args.batched_only and args.impl == "ours":
        r = run_batched(args, torch.device("cuda:0"), compare_plain=False)
        print(json.dumps({"metric": "batched step Msamples/s", "value": r["batched_Msamples_s"], "unit": UNIT,
                          "batched": r}))
        return
    if args.dpd_only and args.impl == "ours":
        r = run_dpd(args, torch.device("cuda:0"))
        print(json.dumps({"metric": "DPD Msamples/s", "value": r["Msamples_s"], "unit": UNIT, "dpd": r}))
        return
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
