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
# Per event of the fused pass, from one ncu capture each on 8 M full-body events (cell and
# direction order, 128 threads, series masses through h^4, walk in sigma units; the brick
# walk with tau_out clipped to the crossing budgets), by image
# layout (0 linear, 1 2x2x2-brick copies): DRAM bytes (dram__bytes_read.sum +
# dram__bytes_write.sum) and L2 requests (lts__t_requests_srcunit_tex_op_red.sum +
# lts__t_requests_srcunit_tex_op_read.sum)
NCU_PER_EVENT = {0: {"dram_bytes": 49.2, "l2_requests": 52.70},
                 1: {"dram_bytes": 47.78, "l2_requests": 39.71}}
# algorithmic FP32 operations per Siddon piece: ~25 for the step and the two
# accumulations plus ~20 for the Gaussian mass of the piece
ALU_OPS_PER_PIECE = 45.0
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
    ap.add_argument("--cpu-sample", type=int, default=15_000_000, help="events in the oracle's timed sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--launch", default=None,
                    help="fix the event-pass launch: threads,blocks_per_sm,chunk,cached_pieces,tail_eval "
                         "(default: the library's autotuner)")
    ap.add_argument("--no-graphs", action="store_true", help="launch iterations directly instead of graph replay")
    ap.add_argument("--tiles", action="store_true", help="shared-memory tiled event pass (off by default)")
    ap.add_argument("--cell-order", type=int, default=0,
                    help="events grouped by TOF-point cells of this edge (voxels), cells spread over blocks "
                         "(0: the library default)")
    ap.add_argument("--dir-bins", default="1,1", help="azimuth,polar direction bins within a cell")
    ap.add_argument("--tile-min", type=int, default=0, help="minimum events per tiled cell (0: the library default)")
    ap.add_argument("--tile-lanes", type=int, default=1, help="threads per event in the tiled pass (1 or 8)")
    ap.add_argument("--samples", type=int, default=0,
                    help="time the sampled TOF kernel with this many samples in the main measurement "
                         "(default 0: the exact Siddon x Phi projector)")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the region-divided and packed/BF16 legs that follow the main measurement")
    ap.add_argument("--serve", action="store_true",
                    help="run the served-reconstruction workload (Poisson stream of mixed jobs) instead")
    ap.add_argument("--serve-jobs", type=int, default=200)
    ap.add_argument("--smallfov-only", action="store_true",
                    help="time only the small field of view (128^3 voxels of 0.5 mm, 5 M events); with --launch "
                         "the launch is fixed instead of tuned")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "events", "regions"],
                    help="with N GPUs: replicas (each rank reconstructs its own 146M events, weak scaling), "
                         "events (one 146M-event job, each rank a shard of the events, one all-reduce of C per "
                         "iteration, strong scaling) or regions (one job divided into the nine TOF body regions, "
                         "each rank a consecutive block of regions, the stitched images summed once per job)")
    ap.add_argument("--serve-leg-jobs", type=int, default=60,
                    help="jobs of the bounded serving leg of the default line (0: no serving leg)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x):
    """Largest value over the ranks of the process group (x itself without one).
    Ranks run independent reconstructions (replicas, no data-path collective);
    the job's time is the slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world, ms):
    """Whole-job throughput: units processed by all ranks over the slowest rank's time."""
    return units_per_rank * world / (ms / 1e3)


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


def roofline(n, visits, pass_ms, probes, hbm_peak_gbs, sm_mhz, traffic, layout=0):
    """Roofline of the fused event pass as t_min / t_measured, t_min the largest of
    its algorithmic terms per launch: HBM (32 B per event), L2 reductions (one FP32
    reduction per Siddon piece at the live rate of scattered red.global.add.f32), L2
    gathers (one 4-byte gather per piece at the live gather rate) and FP32 ALU
    (ALU_OPS_PER_PIECE per piece on 148 SMs x 128 lanes at the sampled SM clock).
    A fifth term, two 32-byte L2 sectors per piece at the live L2 read bandwidth, is
    reported but kept out of the maximum: it charges an L2 sector to every gather,
    while about a third of the gathers hit L1, so it is not a lower bound on the
    time.  `achieved` and `peak` are in the unit of the largest term; `traffic` is
    the ncu DRAM bytes of the launch (or None).

    The reduction rate is that of scattered reductions, one L2 request each.  In the
    2x2x2-brick layout (layout 1) the lanes of a warp share sectors more often, so a
    reduction costs less than one request and the element rate can pass that rate
    (frac above 1).  `l2_requests` then reports the pass at the request level: the
    ncu-measured requests per event of the layout, scaled to the launch, against the
    same probe's request rate."""
    R, G, L2BW = probes.get("l2_red_gops"), probes.get("gather_gops"), probes.get("l2_stream_gbs")
    alu_peak = 148 * 128 * sm_mhz * 1e6                      # FP32 lane operations per second
    t = pass_ms / 1e3
    terms = {"hbm": (32.0 * n) / (hbm_peak_gbs * 1e9),
             "l2_reductions": visits / (R * 1e9) if R else 0.0,
             "l2_gathers": visits / (G * 1e9) if G else 0.0,
             "alu": visits * ALU_OPS_PER_PIECE / alu_peak}
    bound = max(terms, key=terms.get)
    rates = {"hbm": (32.0 * n / t / 1e9, hbm_peak_gbs, "GB/s"),
             "l2_reductions": (visits / t / 1e9, R, "Gred/s"),
             "l2_gathers": (visits / t / 1e9, G, "Ggather/s"),
             "alu": (visits * ALU_OPS_PER_PIECE / t / 1e12, alu_peak / 1e12, "Tops/s")}
    ach, pk, unit = rates[bound]
    hbm_gbs = 32.0 * n / t / 1e9
    sectors_ms = 1e3 * visits * 2 * 32.0 / (L2BW * 1e9) if L2BW else None
    return {
        "bound": bound, "achieved": ach, "peak": pk, "unit": unit, "frac": ach / pk if pk else None,
        "traffic": traffic,
        "traffic_source": f"ncu capture of the same kernel on 8 M full-body events, "
                          f"{NCU_PER_EVENT[layout]['dram_bytes']:.2f} B per event, scaled to the launch's events",
        "t_min_ms": 1e3 * terms[bound], "terms_ms": {k: 1e3 * v for k, v in terms.items()},
        "l2_sectors_ms_not_a_bound": sectors_ms,
        "per_launch": {"events": n, "pieces": visits, "gathers": visits, "reductions": visits,
                       "hbm_bytes": 32.0 * n, "pass_ms": pass_ms},
        "peak_source": "builder-measured live in this run (librecon_probe.so): scattered red.global.add.f32 "
                       "and 4-byte gathers into an L2-resident image of the grid's size, coalesced 16-byte "
                       "reads for the L2 bandwidth; HBM from MEASURED_PEAKS (driver-measured); ALU from "
                       "148 SMs x 128 lanes x the sampled SM clock",
        "mixed_probe_gsteps": probes.get("mixed_gsteps"),
        "image_layout": ["linear", "2x2x2-brick copies"][layout],
        "l2_requests": {"per_event": NCU_PER_EVENT[layout]["l2_requests"],
                        "achieved_greq_s": NCU_PER_EVENT[layout]["l2_requests"] * n / t / 1e9,
                        "ceiling_greq_s": R,
                        "frac": NCU_PER_EVENT[layout]["l2_requests"] * n / t / 1e9 / R if R else None,
                        "source": "reduction + read requests per event from ncu on 8 M full-body events "
                                  "(this layout), scaled to the launch; ceiling: the scattered-reduction "
                                  "probe, one request per reduction"},
        "note": ("frac above 1: in the brick layout a warp's lanes share L2 sectors, so the reductions "
                 "cost fewer requests than the scattered probe's one per reduction; see l2_requests"
                 if R and visits / t / 1e9 > R else None),
        "secondary": {"hbm_gbs": hbm_gbs, "hbm_peak_gbs": hbm_peak_gbs, "hbm_frac": hbm_gbs / hbm_peak_gbs}}


def measure_probes(n_vox, stream, dev):
    """Roofline denominators measured on this GPU (librecon_probe.so)."""
    import ctypes as C
    import torch
    from paper_1706_07075_b300 import build as lib_build
    lib = C.CDLL(lib_build.build_probe())
    for name in ("recon_probe_l2_red", "recon_probe_gather", "recon_probe_erfc", "recon_probe_mixed",
                 "recon_probe_l2_stream", "recon_probe_red_groups"):
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
    # element reductions per second when `group` lanes of a warp share one 32-byte sector
    groups = {}
    for group in (1, 2, 4, 8, 32):
        if lib.recon_probe_red_groups(C.c_void_p(img.data_ptr()), C.c_int64(n_vox), group, 1, h, C.byref(v)) == 0:
            groups[str(group)] = v.value / 1e9
    out["red_lanes_per_sector_gops"] = groups
    if lib.recon_probe_gather(C.c_void_p(img.data_ptr()), C.c_int64(n_vox), C.c_void_p(sink.data_ptr()), h,
                              C.byref(v)) == 0:
        out["gather_gops"] = v.value / 1e9
    img2 = torch.zeros(n_vox, dtype=torch.float32, device=dev)
    if lib.recon_probe_mixed(C.c_void_p(img2.data_ptr()), C.c_void_p(img.data_ptr()), C.c_int64(n_vox),
                             C.c_void_p(sink.data_ptr()), h, C.byref(v)) == 0:
        out["mixed_gsteps"] = v.value / 1e9
    if lib.recon_probe_erfc(C.c_void_p(sink.data_ptr()), h, C.byref(v)) == 0:
        out["erfc_gops"] = v.value / 1e9
    n4 = n_vox - n_vox % 4
    if n4 > 0 and lib.recon_probe_l2_stream(C.c_void_p(img.data_ptr()), C.c_int64(n4), 20,
                                            C.c_void_p(sink.data_ptr()), h, C.byref(v)) == 0:
        out["l2_stream_gbs"] = v.value / 1e9
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


def workload_config(args, n, world):
    """The workload both arms report: the same dictionary for the CUDA arm and the oracle."""
    return {"workload": "fullbody-146M-150x150x600-4mm", "events": n, "iters_per_step": args.iters,
            "sensitivity_lors": args.lors, "tof_fwhm_ps": 300.0,
            "timing": "events resident in HBM; each MLEM iteration a CUDA-graph replay of pass, update and "
                      "conservation sums",
            "projector": f"sampled TOF kernel, {args.samples} samples" if args.samples else
            "exact Siddon pieces x Gaussian mass",
            "l2": "inputs larger than L2 (events 32 B x 146M = 4.7 GB resident)",
            "parallelism": f"replicas{world}" if world > 1 else "single"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_1706_07075_b300 import synth
    # each step a bounded sample: the whole --steps K run stays near 1.5 min of FP64 work
    # on 16 cores (15 M events per step up to 10 steps, fewer per step beyond)
    n_sample = min(args.cpu_sample, max(2_000_000, 150_000_000 // max(1, args.steps)))
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
        "config": dict(workload_config(args, args.events, world), sampled_events=n_sample,
                       timing=f"host wall clock; each step one FP64 MLEM iteration over {n_sample} of the events"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads_used(), "kind": "oracle",
                         "sample": f"each step: 1 FP64 MLEM iteration over a bounded sample of {n_sample} full-body "
                                   f"events (the 150x150x600 grid, sensitivity from 200000 LORs); the metric counts "
                                   f"those sampled events x iterations per second"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0




def time_split_leg(ctx, B, n, args, stream):
    """MLEM through recon_event_pass + recon_update, the calls of the event-sharded
    form, on one rank: the cost of the split (C copied out and back, the stream
    synchronised twice per iteration) against recon_mlem's graph replay."""
    import torch
    from paper_1706_07075_b300.shard import sharded_mlem
    dev = torch.device("cuda", torch.cuda.current_device())
    c_buf = torch.zeros(ctx.n_vox, dtype=torch.float32, device=dev)
    one_rank = lambda c, n_eff: n_eff                                  # noqa: E731  (world of one: no exchange)
    sharded_mlem(ctx, args.iters, c_buf, one_rank)                     # warm-up
    ms = _timed_steps(stream, args.steps, lambda: sharded_mlem(ctx, args.iters, c_buf, one_rank))
    return {"workload": "fullbody, 3 iterations as recon_event_pass + recon_update (one rank)",
            "value": n * args.iters * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps}


def run_sharded(args, B, synth, rank, world, local, dev, stream, ctx, n_total):
    """One full-body job with its events sharded over the ranks (NCCL all-reduce
    of C per iteration); every rank holds n_total / world events."""
    import numpy as np
    import torch
    from paper_1706_07075_b300.shard import sharded_mlem, torch_allreduce_sum
    c_buf = torch.zeros(ctx.n_vox, dtype=torch.float32, device=dev)
    red = torch_allreduce_sum() if world > 1 else (lambda c, n_eff: n_eff)
    for _ in range(args.warmup):
        sharded_mlem(ctx, args.iters, c_buf, red)
    ctx.reset_stats()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hist = None
    for _ in range(args.steps):
        hist = sharded_mlem(ctx, args.iters, c_buf, red)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    host_ms = 1e3 * (time.perf_counter() - t0)
    clocks = sampler.stop()
    gpu_ms = e0.elapsed_time(e1)
    ms = max_over_ranks(max(gpu_ms, host_ms))
    value = n_total * args.iters * args.steps / (ms / 1e3)
    launches = int(ctx.get_stats()["kernel_launches"])
    launch = launch_record(ctx.get_launch(), ctx.get_layout())
    # the same GPU's recon_mlem on this rank's events, for comparison
    mlem_ms = _timed_steps(stream, args.steps, lambda: ctx.mlem(None, args.iters)) / args.steps
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args, n_total, world), parallelism=f"events{world}",
                           sharding="each rank a shard of the events; one all-reduce of C (54 MB) per iteration"),
            "gpu_launches": launches, "clocks": clocks, "gpu_event_ms_per_step": gpu_ms / args.steps,
            "launch": launch, "recon_mlem_ms_per_step_this_rank": mlem_ms,
            "conservation_last": [float(x) for x in hist[-1]]}


def run_region_sharded(args, B, synth, rank, world, local, dev, stream, ctx, n):
    """One full-body job divided into the nine TOF body regions (Sec. 2.5), each
    rank a consecutive block of regions; every rank holds all events, and the
    stitched images are summed once per job (NCCL)."""
    import numpy as np
    import torch
    from paper_1706_07075_b300.shard import region_block, regions_mlem_sharded
    from paper_1706_07075_b300.synth import FULLBODY_REGIONS
    sigma = ctx.get_info()["sigma_mm"]
    margin = 3.0 * sigma + 6.0
    codes = np.zeros(n, np.uint8)
    ctx.split_regions(None, FULLBODY_REGIONS, 0.0, 6.0, codes, None, None)
    n_in = int(np.count_nonzero(codes != 0xFF))
    del codes
    img = torch.zeros(ctx.n_vox, dtype=torch.float32, device=dev)
    red = (lambda t: torch.distributed.all_reduce(t)) if world > 1 else (lambda t: None)
    step = lambda: regions_mlem_sharded(ctx, FULLBODY_REGIONS, margin, 6.0, args.iters, img, rank, world, red)  # noqa
    for _ in range(args.warmup):
        step()
    ctx.reset_stats()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    host_ms = 1e3 * (time.perf_counter() - t0)
    clocks = sampler.stop()
    ms = max_over_ranks(host_ms)
    lo, hi = region_block(len(FULLBODY_REGIONS), rank, world)
    launches = int(ctx.get_stats()["kernel_launches"])
    launch = list(ctx.get_launch())
    # the whole division on this rank alone, for comparison
    whole_ms = _timed_steps(stream, args.steps, lambda: ctx.mlem_regions(None, FULLBODY_REGIONS, margin, 6.0,
                                                                          args.iters)) / args.steps
    return {"metric": METRIC, "value": n_in * args.iters * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args, n, world), parallelism=f"regions{world}",
                           sharding="nine TOF body regions in consecutive blocks over the ranks; stitched images "
                                    "summed once per job", events_in_regions=n_in,
                           timing="host wall clock over the steps (each synchronises)"),
            "regions_of_rank0": [lo, hi], "gpu_launches": launches, "clocks": clocks, "launch": launch,
            "all_regions_on_this_rank_ms_per_step": whole_ms}


def launch_record(ctx_cfg, layout):
    """The event-pass launch the library used, every tuned dimension named."""
    return {"threads": ctx_cfg[0], "blocks_per_sm": ctx_cfg[1], "chunk": ctx_cfg[2], "cached_pieces": ctx_cfg[3],
            "piece_mass": ["fitted erfc tails", "erfcf tails", "midpoint series through h^6", "midpoint series through h^4"][ctx_cfg[4]],
            "reduction": ["scalar, linear image", "scalar, 2x2x2-brick copies"][ctx_cfg[5]],
            "image_tiling": ["global image (L2-resident)", "shared-memory tiles"][layout[0]],
            "threads_per_event": layout[1]}


def time_smallfov_leg(B, synth, args, stream):
    """The small field of view of the served mix (128^3 voxels of 0.5 mm, R = 60 mm,
    5 M events, ~200 Siddon pieces per event) as a reconstruction of its own: the
    launch the autotuner picks for it and its rate, events resident."""
    import numpy as np
    ev = synth.events("smallfov", 5_000_000, args.seed)
    lors = synth.sensitivity_lors("smallfov", 10_000_000, args.seed)
    with B.Context((60.0, 100.0, 90.0), synth.grid_of("smallfov"), 300.0) as c:
        c.set_stream(stream.cuda_stream)
        c.sensitivity(lors)
        c.load_events(B.make_events(ev))
        if args.smallfov_only and args.launch:
            c.set_launch(*[int(x) for x in args.launch.split(",")])
        if args.smallfov_only and args.no_graphs:
            c.set_graphs(0)
        cons = np.zeros((args.iters, 2))
        c.mlem(None, args.iters, None, None, cons)          # warm-up (+ autotune for this key)
        ms = _timed_steps(stream, args.steps, lambda: c.mlem(None, args.iters, None, None, cons))
        rec = launch_record(c.get_launch(), c.get_layout())
    return {"workload": "small FOV 128^3 @ 0.5 mm, R = 60 mm scanner, 5 M events, 3 iterations",
            "value": ev.shape[1] * args.iters * args.steps / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / args.steps, "launch": rec, "conservation_last": [float(x) for x in cons[-1]]}


def _timed_steps(stream, k, fn):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def time_regions_leg(ctx, B, n, args, stream):
    """Region-divided form (Sec. 2.5): split by TOF z into nine body regions,
    all regions' events in one event-pass launch per iteration, stitch.  Counts
    the original events that join a region (not their duplicates) per iteration."""
    import numpy as np
    from paper_1706_07075_b300.synth import FULLBODY_REGIONS
    sigma = ctx.get_info()["sigma_mm"]
    codes = np.zeros(n, np.uint8)
    offs = np.zeros(len(FULLBODY_REGIONS) + 1, np.int64)
    ctx.split_regions(None, FULLBODY_REGIONS, 0.0, 6.0, codes, offs, None)
    n_in = int(np.count_nonzero(codes != 0xFF))
    del codes
    margin = 3.0 * sigma + 6.0
    cons = np.zeros((args.iters, 9, 2))
    ctx.mlem_regions(None, FULLBODY_REGIONS, margin, 6.0, args.iters, None, None, cons)   # warm-up (+ autotune)
    st0 = ctx.get_stats()
    ms = _timed_steps(stream, args.steps, lambda: ctx.mlem_regions(None, FULLBODY_REGIONS, margin, 6.0, args.iters,
                                                                     None, None, cons))
    st1 = ctx.get_stats()
    return {"workload": "fullbody 9 TOF body regions (cores of 50 slices from slice 42, the last of 68), shell 6 mm, "
                        "margin 3 sigma + shell", "value": n_in * args.iters * args.steps / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / args.steps, "events_in_regions": n_in,
            "events_per_region": [int(x) for x in np.diff(offs)],
            "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
            "launch": list(ctx.get_launch()), "n_eff_per_region_last": [float(x) for x in cons[-1, :, 0]],
            "steps": args.steps}


def time_packed_leg(ctx, B, synth, ev, n, args, stream, img_plain, bf16):
    """Precision-packed form: int16 endpoints on a 0.05 mm lattice + FP16 d
    (16 B per event), the forward gather from the FP32 image or from a BF16 copy
    of it.  Resident events and end to end (pinned packed records uploaded, the
    image read back per job); the image's distance to the plain FP32 form's after
    the same iterations from the same start is reported beside the rate."""
    import numpy as np
    import torch
    rec = torch.from_numpy(synth.pack_events(ev)).pin_memory()
    ctx.load_events(B.make_events(rec, packed=True, lattice_mm=synth.LATTICE_MM))
    ctx.set_gather_bf16(1 if bf16 else 0)
    cons = np.zeros((args.iters, 2))
    try:
        ctx.mlem(None, args.iters, None, None, cons)     # warm-up (+ autotune for the packed format)
        st0 = ctx.get_stats()
        ms = _timed_steps(stream, args.steps, lambda: ctx.mlem(None, args.iters, None, None, cons))
        st1 = ctx.get_stats()
        img = torch.empty(ctx.n_vox, dtype=torch.float32).pin_memory()
        times = []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t = time.perf_counter()
            ctx.mlem(B.make_events(rec, packed=True, lattice_mm=synth.LATTICE_MM), args.iters, None, img, cons)
            times.append(time.perf_counter() - t)
    finally:
        ctx.set_gather_bf16(0)
    e2e_T = sum(times[1:]) / (len(times) - 1) if len(times) > 1 else float("nan")
    a, b = img.double(), img_plain.double()
    return {"workload": f"fullbody packed int16/FP16 events, {'BF16' if bf16 else 'FP32'} gather",
            "value": n * args.iters * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "e2e": {"value": n * args.iters / e2e_T, "unit": UNIT, "h2d_bytes_per_step": int(rec.numel() * 2),
                    "d2h_bytes_per_step": int(img.numel() * 4 + cons.nbytes), "job_latency_s": e2e_T},
            "image_rel_l2_vs_plain_f32": float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)),
            "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]), "launch": list(ctx.get_launch()),
            "conservation_last": [float(x) for x in cons[-1]], "steps": args.steps}


def time_lut_leg(ctx, B, n, args, stream, img_exact):
    """The paper's own projector (Sec. 2.3): 32 equally spaced Gaussian samples
    per event, each deposited in its voxel, against the exact Siddon x Phi
    projector on the same resident events.  The tuned launch (threads per block,
    linear image or 2x2x2-brick copies) and, for comparison, both image layouts at
    the tuned thread count.  Accuracy: relative L2 distance of the sampled
    projector's image to the exact one after the same iterations from the same
    start, and of the two forward projections of that image."""
    import numpy as np
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx.set_projector(B.PROJ_SAMPLED, 32)
    cons = np.zeros((args.iters, 2))
    ctx.mlem(None, args.iters, None, None, cons)     # warm-up (+ autotune for this projector)
    st0 = ctx.get_stats()
    ms = _timed_steps(stream, args.steps, lambda: ctx.mlem(None, args.iters, None, None, cons))
    st1 = ctx.get_stats()
    tuned = ctx.get_launch()
    img_lut = torch.empty(ctx.n_vox, dtype=torch.float32).pin_memory()
    ctx.mlem(None, args.iters, None, img_lut, cons)
    layouts = {}
    try:
        for name, red in (("linear", 0), ("bricks", 1)):
            ctx.set_launch(tuned[0], 0, 0, 0, 0, red)
            ctx.mlem(None, args.iters, None, None, cons)     # warm-up
            ms_l = _timed_steps(stream, args.steps, lambda: ctx.mlem(None, args.iters, None, None, cons))
            img_l = torch.empty(ctx.n_vox, dtype=torch.float32).pin_memory()
            ctx.mlem(None, args.iters, None, img_l, cons)
            layouts[name] = {"value": n * args.iters * args.steps / (ms_l / 1e3), "unit": UNIT,
                             "ms_per_step": ms_l / args.steps,
                             "image_rel_l2_vs_tuned": float(torch.linalg.vector_norm(img_l.double() - img_lut.double())
                                                            / torch.linalg.vector_norm(img_lut.double()))}
    finally:
        ctx.set_launch(None)
    p_lut = torch.empty(n, dtype=torch.float32, device=dev)
    p_ex = torch.empty(n, dtype=torch.float32, device=dev)
    lam = img_exact.to(dev)
    ctx.forward(None, lam, p_lut)
    ctx.set_projector(B.PROJ_EXACT)
    ctx.forward(None, lam, p_ex)
    torch.cuda.synchronize(dev)
    a, b = img_lut.double(), img_exact.double()
    fwd_rel = float(torch.linalg.vector_norm(p_lut.double() - p_ex.double()) / torch.linalg.vector_norm(p_ex.double()))
    return {"workload": "fullbody, sampled TOF kernel, 32 samples (Sec. 2.3)", "value": n * args.iters * args.steps /
            (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "launch": {"threads": tuned[0], "layout": ["linear image", "2x2x2-brick copies"][tuned[5]]},
            "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
            "image_rel_l2_vs_exact": float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)),
            "forward_rel_l2_vs_exact": fwd_rel, "conservation_last": [float(x) for x in cons[-1]],
            "steps": args.steps, "layouts_at_tuned_threads": layouts}


def time_osem_leg(ctx, B, n, args, stream, subsets=5):
    """List-mode OSEM (NEXT-4): one iteration = `subsets` sub-iterations over
    consecutive blocks of the resident events (load order; subsets are defined on it)."""
    import numpy as np
    ctx.set_subsets(subsets)
    cons = np.zeros((args.iters * subsets, 2))
    ctx.mlem(None, args.iters, None, None, cons)                 # warm-up
    ms = _timed_steps(stream, args.steps, lambda: ctx.mlem(None, args.iters, None, None, cons))
    ctx.set_subsets(1)
    return {"workload": f"fullbody OSEM, {subsets} subsets, {args.iters} iterations per step",
            "value": n * args.iters * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "conservation_last": [float(x) for x in cons[-1]], "steps": args.steps}


def time_median_leg(ctx, B, n, args, stream):
    """The median-filter sieve (Sec. 2.4): one 3x3x3 filter of the full-body image
    (device in, device out) and a full MLEM step with the sieve after every iteration."""
    import numpy as np
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    img = torch.rand(ctx.n_vox, device=dev)
    out = torch.empty_like(img)
    ctx.median_filter(img, out)                                  # warm-up
    reps = 10
    ms_f = _timed_steps(stream, reps, lambda: ctx.median_filter(img, out)) / reps
    ctx.set_median_filter(1)
    cons = np.zeros((args.iters, 2))
    ctx.mlem(None, args.iters, None, None, cons)                 # warm-up (graph with the sieve)
    ms = _timed_steps(stream, args.steps, lambda: ctx.mlem(None, args.iters, None, None, cons))
    ctx.set_median_filter(0)
    return {"workload": "fullbody 150x150x600 median sieve, 3x3x3", "filter_ms": ms_f,
            "filter_gvox_per_s": ctx.n_vox / (ms_f / 1e3) / 1e9,
            "note": "filter_ms includes the host call's staging copies (device in/out) and its stream sync",
            "mlem_with_sieve": {"value": n * args.iters * args.steps / (ms / 1e3), "unit": UNIT,
                                "ms_per_step": ms / args.steps}}


def time_preprocess_leg(ctx, B, synth, n, stream):
    """Pre-processing on the resident events: attenuation weights exp(sum mu L)
    along each whole LOR and TOF scatter rejection at 95% confidence (Sec. 2.2,
    2.4) against the phantom's attenuation map; the events are left unchanged."""
    import torch
    mu = torch.from_numpy(synth.mu_image("fullbody")).to(torch.device("cuda", torch.cuda.current_device()))
    kept = ctx.preprocess(None, mu, 1.96, 0)                  # warm-up
    ms = _timed_steps(stream, 1, lambda: ctx.preprocess(None, mu, 1.96, 0))
    return {"workload": "fullbody attenuation weights + TOF scatter rejection (z = 1.96)", "ms": ms,
            "events_per_s": n / (ms / 1e3), "kept_fraction": kept / n}


def serve_leg(args, fb, fb_pinned, n_jobs, local):
    """Served reconstruction: a Poisson stream of n_jobs jobs mixing single-region
    slabs (150x150x80 voxels, events whose TOF point lies in the slab), full bodies
    (150x150x600) and small fields of view (128^3 voxels of 0.5 mm), 3 iterations
    each, 60/10/30%, at 0.8x the serial capacity measured on one job of each kind;
    then the same stream served one job at a time in arrival order (the plain form).
    fb: the full-body events (7, n) float32, fb_pinned: the same in pinned memory."""
    import numpy as np
    import torch
    from paper_1706_07075_b300 import synth
    from paper_1706_07075_b300.serve import Job, LibreconExecutor, Server, poisson_arrivals
    n_fb = fb.shape[1]
    p1, p2, d = fb[0:3], fb[3:6], fb[6]
    dz = p1[2] - p2[2]
    D = np.sqrt((p1[0] - p2[0]) ** 2 + (p1[1] - p2[1]) ** 2 + dz ** 2)
    z = 0.5 * (p1[2] + p2[2]) + d * dz / D
    del p1, p2, d, dz, D
    geo_fb = (400.0, 2400.0, 45.0)
    kinds = {"fullbody": (geo_fb, synth.grid_of("fullbody"), [fb_pinned])}
    slabs = []
    for z0 in np.arange(-1040.0, 900.0, 240.0):
        keep = (z >= z0) & (z < z0 + 320.0)
        if keep.sum() >= 1_000_000:
            slabs.append((z0, torch.from_numpy(np.ascontiguousarray(fb[:, keep])).pin_memory()))
    del z
    for z0, evs in slabs:
        kinds[f"region{int(z0)}"] = (geo_fb, (150, 150, 80, 4.0, 4.0, 4.0, -300.0, -300.0, float(z0)), [evs])
    kinds["smallfov"] = ((60.0, 100.0, 90.0), synth.grid_of("smallfov"),
                         [torch.from_numpy(synth.events("smallfov", 5_000_000, args.seed + k)).pin_memory()
                          for k in range(2)])
    budget = 200 << 30
    ex = LibreconExecutor(slots=3)
    lors_fb = synth.sensitivity_lors("fullbody", 20_000_000, args.seed)
    lors_sf = synth.sensitivity_lors("smallfov", 10_000_000, args.seed)
    for k, (geo, grid, _) in kinds.items():
        ex.register_sensitivity(k, geo, grid, lors_fb if geo == geo_fb else lors_sf)
    del lors_fb, lors_sf
    # serial service time of one job of each kind (warm)
    service = {}
    for k, (geo, grid, evs) in kinds.items():
        for rep in range(2):
            j = Job(0, 0.0, evs[0], geo, grid, args.iters, sens_key=k, kind=k)
            torch.cuda.synchronize()
            t = time.perf_counter()
            ex.run(j, 0)
            torch.cuda.synchronize()
            service[k] = time.perf_counter() - t
    region_kinds = [k for k in kinds if k.startswith("region")]
    mean_service = (0.6 * np.mean([service[k] for k in region_kinds]) + 0.1 * service["fullbody"] +
                    0.3 * service["smallfov"])
    rate = 0.8 / mean_service
    arrivals = poisson_arrivals(n_jobs, rate, args.seed)

    def make_jobs():
        # the same stream every call: arrival times, kinds and event sets from the seed
        rng = np.random.default_rng(args.seed)
        out = []
        for i, t in enumerate(arrivals):
            u = rng.uniform()
            kind = "region" if u < 0.6 else ("fullbody" if u < 0.7 else "smallfov")
            if kind == "region":
                kind = region_kinds[int(rng.integers(0, len(region_kinds)))]
            geo, grid, evs = kinds[kind]
            ev = evs[int(rng.integers(0, len(evs)))]
            out.append(Job(i, float(t), ev, geo, grid, args.iters, sens_key=kind, kind=kind))
        return out

    def by_kind(done):
        out = {}
        for j in done:
            out.setdefault("region" if j.kind.startswith("region") else j.kind, []).append(j.latency)
        return {k: {"p50_s": float(np.percentile(v, 50)), "p99_s": float(np.percentile(v, 99)), "jobs": len(v)}
                for k, v in out.items()}

    jobs = make_jobs()
    ex.keep_results = False
    ex.warm(jobs)
    srv = Server(ex, slots=3, hbm_budget_bytes=budget)
    sampler = ClockSampler(local)
    sampler.start()
    stats = srv.replay(jobs)
    clocks = sampler.stop()
    served_kind = by_kind(srv.done)
    # the same stream without stream priorities (every job at the default priority)
    ex.set_priorities(None)
    srv0 = Server(ex, slots=3, hbm_budget_bytes=budget)
    stats0 = srv0.replay(make_jobs())
    ex.set_priorities(4_000_000)
    srv1 = Server(ex, slots=1, hbm_budget_bytes=budget)
    stats1 = srv1.replay(make_jobs())
    ex.close()
    return {"workload": "served mix: region slabs 150x150x80 / full body 150x150x600 / small FOV 128^3 @ 0.5 mm, "
                        "60/10/30%, 3 iterations, Poisson arrivals at 0.8x the serial capacity",
            "jobs": stats["jobs"], "p50_s": stats["p50_s"], "p99_s": stats["p99_s"],
            "events_iters_per_s": stats["events_iters_per_s"], "max_concurrent": stats["max_concurrent"],
            "slots": 3, "hbm_budget_gb": budget >> 30, "arrival_rate_jobs_per_s": rate,
            "region_events": {k: int(kinds[k][2][0].shape[1]) for k in region_kinds},
            "fullbody_events": n_fb, "smallfov_events": 5_000_000, "serial_service_s": service,
            "latency_by_kind": served_kind,
            "priorities": "region slabs and small fields of view on high-priority streams, full bodies on "
                          "low-priority ones",
            "without_priorities": {"p50_s": stats0["p50_s"], "p99_s": stats0["p99_s"],
                                   "events_iters_per_s": stats0["events_iters_per_s"],
                                   "latency_by_kind": by_kind(srv0.done)},
            "one_job_at_a_time": {"p50_s": stats1["p50_s"], "p99_s": stats1["p99_s"],
                                  "events_iters_per_s": stats1["events_iters_per_s"],
                                  "latency_by_kind": by_kind(srv1.done)},
            "clocks": clocks}


def run_serve(args):
    """The served workload alone (--serve): one JSON line with p50/p99 latency."""
    import torch
    from paper_1706_07075_b300 import synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    fb = synth.events("fullbody", args.events, args.seed)
    leg = serve_leg(args, fb, torch.from_numpy(fb).pin_memory(), args.serve_jobs, local)
    line = {"metric": "served TOF-MLEM reconstruction: p50/p99 job latency and aggregate events x iterations / s",
            "value": leg["p50_s"], "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "dtype": "f32", "config": {"workload": leg["workload"]}}
    line.update({k: v for k, v in leg.items() if k != "workload"})
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

    # replicas: a job per rank; events: one job, each rank drawing its shard; regions:
    # one job, every rank holding all of its events
    n = args.events // world if args.shard == "events" else args.events
    t_gen = time.perf_counter()
    ev = synth.events("fullbody", n, args.seed + (0 if args.shard == "regions" else rank))
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
    if args.samples:
        ctx.set_projector(B.PROJ_SAMPLED, args.samples)
    if args.tiles:
        ctx.set_tiled_pass(max(1, args.tile_min), args.tile_lanes)
    az, pol = (int(x) for x in args.dir_bins.split(","))
    if args.cell_order or (az, pol) != (1, 1):
        ctx.set_event_order(args.cell_order or -1, az, pol)
    if args.shard in ("events", "regions"):
        if args.shard == "events":
            line = run_sharded(args, B, synth, rank, world, local, dev, stream, ctx, n * world)
        else:
            line = run_region_sharded(args, B, synth, rank, world, local, dev, stream, ctx, n)
        if rank == 0:
            print(json.dumps(line), flush=True)
        ctx.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    # warm-up (the first call also runs the launch autotuner)
    for _ in range(args.warmup):
        ctx.mlem(None, args.iters)
    cfg = ctx.get_launch()
    layout = ctx.get_layout()

    # timed region: events resident in HBM, each iteration a CUDA-graph replay (the
    # library's default path)
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
    ms = max_over_ranks(ms)
    value = aggregate_rate(n * args.iters * args.steps, world, ms)

    # the split of a step into event passes and updates: the same steps again with
    # per-kernel CUDA events on the context's stream (direct launches instead of
    # graph replay while timing is on)
    ctx.set_timing(1)
    ctx.reset_stats()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e2.record(stream)
    for _ in range(args.steps):
        ctx.mlem(None, args.iters, None, None, cons)
    e3.record(stream)
    torch.cuda.synchronize(dev)
    split_stats = ctx.get_stats()
    split_ms = e2.elapsed_time(e3)
    ctx.set_timing(0)

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
    tiles_info = {k: v for k, v in ctx.get_info().items() if k.startswith("tile")}

    legs = {}
    if not args.no_legs and not args.samples:
        legs["sampled_lut32"] = time_lut_leg(ctx, B, n, args, stream, img)
        legs["median_sieve"] = time_median_leg(ctx, B, n, args, stream)
        legs["osem5"] = time_osem_leg(ctx, B, n, args, stream)
        legs["preprocess"] = time_preprocess_leg(ctx, B, synth, n, stream)
        legs["regions"] = time_regions_leg(ctx, B, n, args, stream)
        legs["split_pass_update"] = time_split_leg(ctx, B, n, args, stream)
        # the packed legs load packed events into the context: they come last
        legs["packed_f32"] = time_packed_leg(ctx, B, synth, ev, n, args, stream, img, bf16=False)
        legs["packed_bf16"] = time_packed_leg(ctx, B, synth, ev, n, args, stream, img, bf16=True)
        legs["smallfov"] = time_smallfov_leg(B, synth, args, stream)
    if not args.no_legs and not args.samples and args.serve_leg_jobs > 0 and world == 1:
        ctx.close()                 # the served contexts hold their own copies of the events
        legs["serve"] = serve_leg(args, ev, pinned, args.serve_leg_jobs, local)

    # roofline of the dominant kernel (the fused event pass)
    passes = max(1, split_stats["pass_launches"])
    pass_ms = split_stats["pass_ms"] / passes
    upd_ms = split_stats["update_ms"] / passes
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": workload_config(args, n, world),
           "e2e": {"value": n * args.iters / e2e_T, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h), "job_latency_s": e2e_T},
           "gpu_launches": int(stats["kernel_launches"]),
           "clocks": clocks,
           "legs": legs,
           "extra": {"t_generate_s": t_gen, "t_sensitivity_s": t_sens, "t_load_s": t_load,
                     "launch": launch_record(ctx_cfg=cfg, layout=layout),
                     "tiles": tiles_info,
                     "pass_ms": pass_ms, "update_ms": upd_ms, "conservation_last": list(cons[-1]),
                     "pass_split_run": {"how": "the timed steps repeated with per-kernel CUDA events on the "
                                               "context's stream (direct launches, no graph replay)",
                                        "ms_per_step": split_ms / args.steps,
                                        "pass_launches": int(split_stats["pass_launches"])}}}
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
        lay = int(cfg[5]) if not layout[0] else 0
        traffic = NCU_PER_EVENT[lay]["dram_bytes"] * n if not args.samples and not layout[0] else None
        sm_mhz = (clocks.get("sm_mhz") or 2032.0) if isinstance(clocks, dict) else 2032.0
        out["roofline"] = roofline(n, visits, pass_ms, probes, peaks["hbm_gbs"], sm_mhz, traffic, lay)
        out["roofline"]["secondary"]["hbm_peak_source"] = src
        if args.samples:
            # the roofline above counts Siddon pieces: it describes the exact projector only
            out["roofline"] = {"bound": "l2_reductions", "achieved": None, "peak": probes.get("l2_red_gops"),
                               "unit": "Gred/s",
                               "frac": None, "traffic": None,
                               "note": "sampled projector timed: the Siddon-piece roofline does not apply"}
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
    if args.serve:
        return run_serve(args)
    if args.smallfov_only:
        import torch
        from paper_1706_07075_b300 import binding as B
        from paper_1706_07075_b300 import synth
        stream = torch.cuda.Stream()
        print(json.dumps({"smallfov": time_smallfov_leg(B, synth, args, stream)}), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
