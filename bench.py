#!/usr/bin/env python
"""Throughput of list-mode TOF-MLEM on the full-body workload (one B300).

Workload (default): the synthetic full-body stand-in for the paper's NCAT
study — 146 M events (33% scatter), 150 x 150 x 600 voxels of 4 mm, 300 ps
FWHM TOF, 3 MLEM iterations per step, sensitivity from 50 M LORs.
A step is one reconstruction of all events (3 iterations through the fused
event pass, the update and the per-iteration conservation sums); the metric
is events x iterations / s.  The sensitivity image and the upload are done
once before the timed region and reported separately.

Prints one JSON line (rank 0).  --impl reference times the FP64 oracle on the
host cores on a bounded sample of the same workload instead.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TOF-MLEM events x iterations / s (full-body, 146M events, 150x150x600 @ 4 mm)"
UNIT = "events*iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--events", type=int, default=146_000_000)
    ap.add_argument("--lors", type=int, default=50_000_000)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--seed", type=int, default=1708)
    ap.add_argument("--cpu-sample", type=int, default=300_000, help="events in the oracle's timed sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--launch", default=None,
                    help="fix the event-pass launch: threads,blocks_per_sm,chunk,cached_pieces,tail_eval "
                         "(default: the library's autotuner)")
    ap.add_argument("--no-graphs", action="store_true", help="launch iterations directly instead of graph replay")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def measure_probes(n_vox, stream, dev):
    """Roofline denominators measured on this GPU (librecon_probe.so)."""
    import ctypes as C
    import torch
    from paper_1706_07075_b300 import build as lib_build
    lib = C.CDLL(lib_build.build_probe())
    for name in ("recon_probe_l2_red", "recon_probe_gather", "recon_probe_erfc"):
        getattr(lib, name).restype = C.c_int
    img = torch.zeros(n_vox, dtype=torch.float32, device=dev)
    sink = torch.zeros(148 * 64 * 256, dtype=torch.float32, device=dev)
    out = {}
    v = C.c_double()
    h = C.c_void_p(stream.cuda_stream)
    if lib.recon_probe_l2_red(C.c_void_p(img.data_ptr()), C.c_int64(n_vox), 1, h, C.byref(v)) == 0:
        out["l2_red_gops"] = v.value / 1e9
    if lib.recon_probe_l2_red(C.c_void_p(img.data_ptr()), C.c_int64(n_vox), 4, h, C.byref(v)) == 0:
        out["l2_red_runs4_gops"] = v.value / 1e9
    if lib.recon_probe_gather(C.c_void_p(img.data_ptr()), C.c_int64(n_vox), C.c_void_p(sink.data_ptr()), h,
                              C.byref(v)) == 0:
        out["gather_gops"] = v.value / 1e9
    if lib.recon_probe_erfc(C.c_void_p(sink.data_ptr()), h, C.byref(v)) == 0:
        out["erfc_gops"] = v.value / 1e9
    torch.cuda.synchronize(dev)
    return out


def mean_visits(ev, n_sample=200_000):
    """Exact mean Siddon pieces per event inside the TOF window (oracle count)."""
    import numpy as np
    import oracle
    from paper_1706_07075_b300 import synth
    g = oracle.Grid(*synth.grid_of("fullbody"))
    idx = np.linspace(0, ev.shape[1] - 1, min(n_sample, ev.shape[1])).astype(np.int64)
    sub = ev[:, idx].astype(np.float64)
    return oracle.count_visits(g, sub, oracle.tof_sigma_mm(300.0)) / sub.shape[1]


def cpu_baseline(ev, lors_for_sens, iters_unit, n_sample):
    """The FP64 oracle (as it stands) on a bounded sample of the workload: one MLEM
    iteration over n_sample events on the full-body grid, all host cores."""
    import numpy as np
    import oracle
    from paper_1706_07075_b300 import synth
    g = oracle.Grid(*synth.grid_of("fullbody"))
    sigma = oracle.tof_sigma_mm(300.0)
    idx = np.linspace(0, ev.shape[1] - 1, n_sample).astype(np.int64)
    sub = ev[:, idx].astype(np.float64)
    s = oracle.sensitivity(g, lors_for_sens)
    t = time.perf_counter()
    oracle.mlem(g, sub, s, 1, sigma)
    dt = time.perf_counter() - t
    return {"value": n_sample * 1 / dt, "unit": UNIT, "cores": oracle.threads_used(), "kind": "oracle",
            "sample": f"1 FP64 MLEM iteration over {n_sample} of the full-body events (evenly strided) on the "
                      f"150x150x600 grid, sensitivity from {lors_for_sens.shape[1]} LORs; {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_1706_07075_b300 import synth
    n_sample = args.cpu_sample
    ev = synth.events("fullbody", n_sample, args.seed)
    lors = synth.sensitivity_lors("fullbody", 200_000, args.seed)
    g = oracle.Grid(*synth.grid_of("fullbody"))
    sigma = oracle.tof_sigma_mm(300.0)
    s = oracle.sensitivity(g, lors)
    evd = ev.astype(np.float64)
    for _ in range(args.warmup):
        oracle.mlem(g, evd[:, : max(1, n_sample // 10)], s, 1, sigma)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.mlem(g, evd, s, 1, sigma)
        times.append(time.perf_counter() - t)
    T = sum(times)
    value = n_sample * args.steps / T
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fullbody-146M-150x150x600-4mm (oracle: bounded sample)", "events_per_step": n_sample,
                   "iters_per_step": 1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads_used(), "kind": "oracle",
                         "sample": f"1 FP64 MLEM iteration over {n_sample} full-body events per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    from paper_1706_07075_b300 import binding as B
    from paper_1706_07075_b300 import synth

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    n = args.events
    t_gen = time.perf_counter()
    ev = synth.events("fullbody", n, args.seed + rank)
    lors = synth.sensitivity_lors("fullbody", args.lors, args.seed)
    t_gen = time.perf_counter() - t_gen

    stream = torch.cuda.Stream(device=dev)
    ctx = B.Context((400.0, 2400.0, 45.0), synth.grid_of("fullbody"), 300.0)
    ctx.set_stream(stream.cuda_stream)
    t = time.perf_counter()
    ctx.sensitivity(lors)
    t_sens = time.perf_counter() - t
    pinned = torch.from_numpy(ev).pin_memory()
    t = time.perf_counter()
    ctx.load_events(B.make_events(pinned))
    t_load = time.perf_counter() - t

    if args.launch:
        ctx.set_launch(*[int(x) for x in args.launch.split(",")])
    if args.no_graphs:
        ctx.set_graphs(0)
    # warm-up (the first call also runs the launch autotuner)
    for _ in range(args.warmup):
        ctx.mlem(None, args.iters)
    cfg = ctx.get_launch()

    # timed region: events resident in HBM
    ctx.set_timing(1)
    ctx.reset_stats()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cons = np.zeros((args.iters, 2))
    for _ in range(args.steps):
        ctx.mlem(None, args.iters, None, None, cons)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    stats = ctx.get_stats()
    ctx.set_timing(0)
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())
    value = n * args.iters * args.steps * world / (ms / 1e3)

    # end to end through the public call: pinned host events in, host image out
    img = torch.empty(ctx.n_vox, dtype=torch.float32).pin_memory()
    e2e_times = []
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        ctx.mlem(B.make_events(pinned), args.iters, None, img, cons)
        e2e_times.append(time.perf_counter() - t)
    e2e_T = sum(e2e_times[1:]) / args.e2e_steps if args.e2e_steps > 0 else float("nan")
    h2d = ev.nbytes
    d2h = img.numel() * 4 + cons.nbytes

    # roofline of the dominant kernel (the fused event pass)
    passes = max(1, stats["pass_launches"])
    pass_ms = stats["pass_ms"] / passes
    upd_ms = stats["update_ms"] / passes
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "fullbody-146M-150x150x600-4mm", "events": n, "iters_per_step": args.iters,
                      "sensitivity_lors": args.lors, "tof_fwhm_ps": 300.0,
                      "launch": {"threads": cfg[0], "blocks_per_sm": cfg[1], "chunk": cfg[2]},
                      "l2": "inputs larger than L2 (events 32 B x 146M = 4.7 GB resident)",
                      "parallelism": f"replicas{world}" if world > 1 else "single"},
           "e2e": {"value": n * args.iters / e2e_T, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h)},
           "gpu_launches": int(stats["kernel_launches"]),
           "clocks": clocks,
           "extra": {"t_generate_s": t_gen, "t_sensitivity_s": t_sens, "t_load_s": t_load,
                     "pass_ms": pass_ms, "update_ms": upd_ms, "conservation_last": list(cons[-1])}}
    if rank == 0:
        peaks, src = measured_peaks()
        vbar = mean_visits(ev)
        visits = vbar * n
        out["extra"]["mean_visits_per_event"] = vbar
        probes = measure_probes(ctx.n_vox, stream, dev)
        out["extra"]["probes"] = probes
        # The event pass issues one FP32 reduction into the L2-resident image per
        # Siddon piece (visits per launch = mean pieces per event x events) and
        # reads each 32-byte event record once from HBM.
        red_rate = visits / (pass_ms / 1e3)
        hbm_gbs = 32.0 * n / (pass_ms / 1e3) / 1e9
        out["roofline"] = {
            "bound": "l2_red", "achieved": red_rate / 1e9, "peak": probes["l2_red_gops"], "unit": "Gop/s",
            "frac": red_rate / 1e9 / probes["l2_red_gops"], "traffic": None,
            "per_launch": {"events": n, "reductions": visits, "gathers": visits, "hbm_bytes": 32.0 * n,
                           "pass_ms": pass_ms},
            "peak_source": "live probe: scattered red.global.add.f32 into an L2-resident image of the grid's size",
            "secondary": {"hbm_gbs": hbm_gbs, "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_frac": hbm_gbs / peaks["hbm_gbs"],
                          "hbm_peak_source": src,
                          "gather_frac": red_rate / 1e9 / probes["gather_gops"]}}
        if not args.no_cpu_baseline:
            lsub = lors[:, :200_000]
            out["cpu_baseline"] = cpu_baseline(ev, lsub, args.iters, args.cpu_sample)
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
