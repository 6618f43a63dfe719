"""Served reconstruction on the GPU: jobs of three kinds (tiny scanner, small
field of view at 0.5 mm, a full-body region slab of 150 x 150 x 80 voxels)
arrive as a Poisson stream and share the GPU through the continuous-batching
server.  Each job's image must be the same when it runs alone and when it runs
in the mix (relative L2 <= 1e-5: only the order of the FP32 reductions
differs), and counts must be conserved."""
import numpy as np
import pytest

from gpu_common import rel_l2
from paper_1706_07075_b300 import synth
from paper_1706_07075_b300.serve import Job, LibreconExecutor, Server, poisson_arrivals

pytestmark = pytest.mark.gpu


def slab_pool(n_events, seed, z0_mm, slices=80):
    """Full-body events whose TOF point lies in an 80-slice slab, and the slab grid."""
    ev = synth.events("fullbody", n_events, seed)
    p1, p2, d = ev[0:3].astype(np.float64), ev[3:6].astype(np.float64), ev[6].astype(np.float64)
    u = (p1 - p2) / np.linalg.norm(p1 - p2, axis=0)
    z = 0.5 * (p1[2] + p2[2]) + d * u[2]
    keep = (z >= z0_mm) & (z < z0_mm + slices * 4.0)
    grid = (150, 150, slices, 4.0, 4.0, 4.0, -300.0, -300.0, z0_mm)
    return np.ascontiguousarray(ev[:, keep]), grid


@pytest.fixture(scope="module")
def pool():
    import torch
    tiny_g = synth.grid_of("tiny")
    fov_g = synth.grid_of("smallfov")
    slab_ev, slab_g = slab_pool(1_200_000, 61, -200.0)
    kinds = {
        "tiny": ((150.0, 200.0, 90.0), tiny_g, [synth.events("tiny", 100_000, 70 + k) for k in range(2)],
                 synth.sensitivity_lors("tiny", 200_000, 70)),
        "smallfov": ((60.0, 100.0, 90.0), fov_g, [synth.events("smallfov", 150_000, 80)],
                     synth.sensitivity_lors("smallfov", 200_000, 80)),
        "region": ((400.0, 2400.0, 45.0), slab_g, [slab_ev], synth.sensitivity_lors("fullbody", 300_000, 90)),
    }
    pinned = {k: [torch.from_numpy(e).pin_memory() for e in v[2]] for k, v in kinds.items()}
    return kinds, pinned


def make_jobs(kinds, pinned, n_jobs, seed):
    rng = np.random.default_rng(seed)
    arrivals = poisson_arrivals(n_jobs, 200.0, seed)
    names = ["region", "tiny", "smallfov"]
    jobs = []
    for i in range(n_jobs):
        kind = names[i % 3] if i < 3 else names[rng.integers(0, 3)]
        geo, grid, evs, _ = kinds[kind]
        which = int(rng.integers(0, len(evs)))
        jobs.append(Job(i, float(arrivals[i]), pinned[kind][which], geo, grid, 3, sens_key=kind,
                        kind=f"{kind}{which}"))
    return jobs


def run(kinds, jobs, slots):
    ex = LibreconExecutor(slots)
    for k, (geo, grid, _, lors) in kinds.items():
        ex.register_sensitivity(k, geo, grid, lors)
    srv = Server(ex, slots=slots, hbm_budget_bytes=64 << 30)
    try:
        stats = srv.replay(jobs)
    finally:
        ex.close()
    return stats


def test_each_result_is_the_same_alone_and_in_the_mix(pool):
    kinds, pinned = pool
    mixed = make_jobs(kinds, pinned, 12, 5)
    stats = run(kinds, mixed, slots=3)
    assert stats["jobs"] == 12 and stats["max_concurrent"] >= 2
    assert stats["p99_s"] >= stats["p50_s"] > 0
    alone = {}
    for j in mixed:
        if j.kind in alone:
            continue
        solo = Job(0, 0.0, j.events, j.geometry, j.grid, j.n_iter, sens_key=j.sens_key, kind=j.kind)
        run(kinds, [solo], slots=1)
        alone[j.kind] = solo.result
    for j in mixed:
        assert rel_l2(j.result, alone[j.kind]) <= 1e-5, j.kind
        n_eff, ssum = j.conservation[-1]
        assert ssum == pytest.approx(n_eff, rel=1e-5)


def test_a_binding_budget_bounds_the_device_memory(pool):
    # a budget well below what the cached contexts of three slots x three grids
    # would hold: the server charges the cached contexts (recon_info's
    # device_bytes), evicts idle ones, and the device memory in use, sampled with
    # cudaMemGetInfo during the stream, stays within the budget (plus a small
    # allowance for what the CUDA runtime keeps per context: streams, events,
    # graph executables)
    import threading
    import time
    import torch
    kinds, pinned = pool
    jobs = make_jobs(kinds, pinned, 15, 9)
    biggest = max(j.footprint() for j in jobs)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0, _ = torch.cuda.mem_get_info()
    ex = LibreconExecutor(3)
    for k, (geo, grid, _, lors) in kinds.items():
        ex.register_sensitivity(k, geo, grid, lors)
    sens = ex.resident_bytes()
    budget = sens + int(1.6 * biggest)
    peak = [0]
    stop = threading.Event()

    def sample():
        while not stop.is_set():
            free, _ = torch.cuda.mem_get_info()
            peak[0] = max(peak[0], free0 - free)
            time.sleep(0.002)

    th = threading.Thread(target=sample, daemon=True)
    th.start()
    srv = Server(ex, slots=3, hbm_budget_bytes=budget)
    try:
        stats = srv.replay(jobs)
    finally:
        stop.set()
        th.join()
        evicted = ex.evicted
        ex.close()
    allowance = 96 << 20
    print(f"\nbudget {budget / 2**20:.0f} MiB, peak charged {stats['peak_charged_bytes'] / 2**20:.0f} MiB, "
          f"peak in use {peak[0] / 2**20:.0f} MiB, contexts evicted {evicted}, max concurrent "
          f"{stats['max_concurrent']}")
    assert stats["jobs"] == 15
    assert stats["peak_charged_bytes"] <= budget
    assert evicted > 0
    assert peak[0] <= budget + allowance
    for j in jobs:
        n_eff, ssum = j.conservation[-1]
        assert ssum == pytest.approx(n_eff, rel=1e-5)
