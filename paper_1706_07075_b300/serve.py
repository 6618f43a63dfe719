"""Continuous-batching reconstruction server over the librecon C-ABI.

Jobs (list-mode events + scanner + grid + iteration count) arrive at any
time.  The scheduler admits queued jobs, oldest first, whenever a slot is
free and the job's device-memory footprint fits the remaining HBM budget; a
later, smaller job may pass an older one that does not fit yet (first fit in
arrival order).  With `max_overtakes` set, a job that later jobs have passed
that many times holds the line: no younger job starts until it does, so a
large job cannot starve behind a stream of small ones.  Each slot owns CUDA
streams and a reconstruction context per image grid, so the upload, the MLEM
iterations and the read-back of concurrent jobs overlap on the GPU; small grids
run on high-priority streams, so a small job's kernels do not wait for a
full-body pass to drain.  Sensitivity images are computed once
per (scanner, grid) and stay resident on the device; contexts are kept and
reused by later jobs on the same grid.

HBM budget: everything the executor keeps on the device counts against it.
An executor that caches state (contexts, sensitivity images) reports it through
`resident_bytes()`, the bytes already held for a job's grid on a slot through
`context_bytes(slot, job)`, and frees idle state through
`evict_idle(running, need)`.  A job is admitted on a slot when the resident
bytes, each running job at the larger of its footprint and what its context
already holds, and the new job's growth (its footprint less what the slot
already holds for its grid) fit the budget; if
they do not, idle cached contexts (least recently used first, never one a
running job uses) are closed first.  An executor without these methods caches
nothing, and a job then reserves its whole footprint while it runs.

Timing per job: queue wait, service time and latency (completion - arrival).
The scheduling logic is independent of the GPU: `Server` takes an executor
object, and `LibreconExecutor` is the one that runs jobs through librecon.
"""
import heapq
import threading
import time
from dataclasses import dataclass, field

import numpy as np

EVENT_BYTES = 72          # resident F32 event record (32 B), its cell-ordered copy (32 B), cell code and rank (4 B each)
IMAGE_BYTES_PER_VOXEL = 20  # lambda, C, s32 (4 B each) + s64 (8 B)
# host events go up in chunks of at most 2^23 events through two staging halves of
# 28 bytes per event each
STAGING_CHUNK_EVENTS = 1 << 23
STAGING_BYTES_PER_EVENT = 2 * 28
# the library's default event order bins events by cells of 4^3 voxels and 16 x 8
# direction bins; each bin key costs a count, a list entry (4 B each) and a 64-bit
# start
ORDER_CELL_VOXELS = 4
ORDER_DIRECTION_BINS = 16 * 8
ORDER_KEY_BYTES = 16


@dataclass
class Job:
    job_id: int
    arrival: float                # seconds on the server clock
    events: object                # (7, n) float32 array/tensor (pinned host memory for full overlap)
    geometry: tuple               # (radius, axial length, max axial angle)
    grid: tuple                   # (nx, ny, nz, vx, vy, vz, ox, oy, oz)
    n_iter: int
    sens_key: object = None       # key of the resident sensitivity image
    kind: str = ""
    result: object = None         # host float32 image after completion
    conservation: object = None
    admitted: float = None
    finished: float = None
    slot: int = None

    @property
    def n_events(self):
        return int(self.events.shape[1])

    def footprint(self):
        """Device bytes a context needs for this job: resident events with their
        binned copy, the images, the event-order bin table and the upload staging."""
        nx, ny, nz = self.grid[:3]
        c = ORDER_CELL_VOXELS
        keys = -(-nx // c) * -(-ny // c) * -(-nz // c) * ORDER_DIRECTION_BINS
        staging = min(self.n_events, STAGING_CHUNK_EVENTS) * STAGING_BYTES_PER_EVENT
        return (self.n_events * EVENT_BYTES + nx * ny * nz * IMAGE_BYTES_PER_VOXEL + keys * ORDER_KEY_BYTES +
                staging)

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


@dataclass(order=True)
class _Queued:
    arrival: float
    seq: int
    job: Job = field(compare=False)
    overtaken: int = field(default=0, compare=False)   # younger jobs admitted while this one waited


class Server:
    """Admission, slots and the HBM budget; `executor.run(job, slot)` does the work.

    max_overtakes: None (plain first fit) or the number of times younger jobs
    may be admitted past a waiting job before it blocks further admissions."""

    def __init__(self, executor, slots=3, hbm_budget_bytes=200 << 30, clock=time.perf_counter, max_overtakes=None):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        if max_overtakes is not None and max_overtakes < 0:
            raise ValueError("max_overtakes must be None or >= 0")
        self.max_overtakes = max_overtakes
        self.executor = executor
        self.slots = slots
        self.budget = int(hbm_budget_bytes)
        self.clock = clock
        self._queue = []
        self._seq = 0
        self._free_slots = list(range(slots))
        self._in_use = 0            # footprints of the running jobs (bytes)
        self._running_jobs = {}     # slot -> running job
        self.peak_charged = 0       # largest resident + reserved bytes seen at an admission
        self._lock = threading.Condition()
        self._threads = []
        self._errors = []
        self.done = []
        self.t0 = None
        self.max_concurrent = 0
        self._running = 0

    def now(self):
        return self.clock() - self.t0

    def start(self):
        self.t0 = self.clock()

    def submit(self, job):
        if job.footprint() > self.budget:
            raise ValueError(f"job {job.job_id} needs {job.footprint()} bytes, more than the whole budget")
        with self._lock:
            heapq.heappush(self._queue, _Queued(job.arrival, self._seq, job))
            self._seq += 1
            self._admit_locked()

    def _resident(self):
        f = getattr(self.executor, "resident_bytes", None)
        return int(f()) if f else 0

    def _held(self, slot, job):
        f = getattr(self.executor, "context_bytes", None)
        return int(f(slot, job)) if f else 0

    def _place(self, job):
        """(slot, growth) for a job: the free slot that already holds the most
        device memory for the job's grid, and the bytes the job may add to it."""
        slot = max(self._free_slots, key=lambda s: (self._held(s, job), -s))
        return slot, max(0, job.footprint() - self._held(slot, job))

    def _charged(self):
        """Device bytes charged now: the executor's resident state, each running job
        at the larger of its footprint and what its context already holds (that
        context counted once), plus anything else reserved in _in_use."""
        overlap = sum(min(j.footprint(), self._held(s, j)) for s, j in self._running_jobs.items())
        return self._resident() + self._in_use - overlap

    def _fits(self, growth):
        return self._charged() + growth <= self.budget

    def _admit_locked(self):
        """First fit in arrival order while slots and budget allow; a waiting job
        passed max_overtakes times stops younger jobs from being admitted."""
        kept = []
        while self._queue and self._free_slots:
            q = heapq.heappop(self._queue)
            slot, growth = self._place(q.job)
            if not self._fits(growth):
                evict = getattr(self.executor, "evict_idle", None)
                if evict is not None:
                    over = self._charged() + growth - self.budget
                    evict(dict(self._running_jobs), over)
                    slot, growth = self._place(q.job)
            if not self._fits(growth):
                if self._running == 0 and self._in_use == 0:
                    # nothing runs and nothing idle is left to free: it can never fit
                    q.job.finished = self.now()
                    self._errors.append((q.job.job_id, "does not fit the HBM budget beside the resident state"))
                    self.done.append(q.job)
                    continue
                kept.append(q)
                if self.max_overtakes is not None and q.overtaken >= self.max_overtakes:
                    break          # it holds the line until the budget frees up for it
                continue
            for older in kept:
                older.overtaken += 1
            self._free_slots.remove(slot)
            self._in_use += q.job.footprint()
            self._running_jobs[slot] = q.job
            self.peak_charged = max(self.peak_charged, self._charged())
            q.job.admitted = self.now()
            q.job.slot = slot
            self._running += 1
            self.max_concurrent = max(self.max_concurrent, self._running)
            t = threading.Thread(target=self._work, args=(q.job, slot, q.job.footprint()), daemon=True)
            self._threads.append(t)
            t.start()
        for q in kept:
            heapq.heappush(self._queue, q)

    def _work(self, job, slot, fp):
        try:
            self.executor.run(job, slot)
        except Exception as e:  # reported by drain(); the slot and memory are released
            self._errors.append((job.job_id, repr(e)))
        finally:
            with self._lock:
                job.finished = self.now()
                self.done.append(job)
                self._in_use -= fp
                self._running_jobs.pop(slot, None)
                self._free_slots.append(slot)
                self._free_slots.sort()
                self._running -= 1
                self._admit_locked()
                self._lock.notify_all()

    def drain(self, timeout=None):
        """Wait until every submitted job has finished."""
        deadline = None if timeout is None else time.monotonic() + timeout
        with self._lock:
            while self._queue or self._running:
                left = None if deadline is None else deadline - time.monotonic()
                if left is not None and left <= 0:
                    raise TimeoutError("jobs still running")
                self._lock.wait(left)
        for t in self._threads:
            t.join()
        if self._errors:
            raise RuntimeError(f"jobs failed: {self._errors}")

    def replay(self, jobs):
        """Submit jobs at their arrival times (seconds after start) and drain."""
        self.start()
        for job in sorted(jobs, key=lambda j: j.arrival):
            delay = job.arrival - self.now()
            if delay > 0:
                time.sleep(delay)
            self.submit(job)
        self.drain()
        return self.stats()

    def stats(self):
        lat = np.array([j.latency for j in self.done])
        ev_it = sum(j.n_events * j.n_iter for j in self.done)
        span = max(j.finished for j in self.done) - min(j.arrival for j in self.done) if self.done else 0.0
        return {"jobs": len(self.done), "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
                "events_iters_per_s": ev_it / span if span > 0 else None, "span_s": span,
                "max_concurrent": self.max_concurrent, "peak_charged_bytes": self.peak_charged}


class LibreconExecutor:
    """Runs jobs through librecon: CUDA streams per slot (a high-priority one for
    small grids, a low-priority one for large ones), contexts reused per grid,
    sensitivity images resident per key.  The device memory it holds is
    reported to the server: each cached context's buffers (recon_info's
    device_bytes, read after every job on the slot's own thread) and the
    sensitivity images."""

    def __init__(self, slots, device=0, sensitivities=None, keep_results=True, launch=(128, 0, 0, 0, 2),
                 low_priority_voxels=4_000_000):
        import torch
        from . import binding as B
        self.B = B
        self.torch = torch
        self.device = device
        torch.cuda.set_device(device)
        # two streams per slot: contexts on grids of more than low_priority_voxels voxels
        # (full bodies) run on the low-priority one, the rest (region slabs, small
        # fields of view) on the high-priority one, so that when a block slot frees up
        # the GPU takes a small job's blocks before the next blocks of a long pass
        # (None: every context on its slot's default-priority stream)
        self.low_priority_voxels = low_priority_voxels
        self.streams = [torch.cuda.Stream(device=device, priority=-1) for _ in range(slots)]
        self.low_streams = [torch.cuda.Stream(device=device, priority=0) for _ in range(slots)]
        self.contexts = [dict() for _ in range(slots)]   # per slot: grid -> Context
        self.loaded = [dict() for _ in range(slots)]     # per slot: grid -> sensitivity key resident in it
        self.ctx_bytes = {}                               # (slot, grid) -> device bytes the context holds
        self.last_used = {}                               # (slot, grid) -> use counter (LRU eviction)
        self._use = 0
        self.evicted = 0
        self.sens = dict(sensitivities or {})            # key -> device float64 tensor
        self.keep_results = keep_results
        self.launch = launch                              # fixed event-pass launch (None: autotune per job size)
        self._sens_lock = threading.Lock()
        self._lock = threading.Lock()                     # contexts, ctx_bytes, last_used

    @staticmethod
    def _key(job):
        return (tuple(job.grid), tuple(job.geometry))

    def _stream_for(self, slot, grid):
        """High-priority stream for grids up to low_priority_voxels voxels, low for
        larger ones; every grid on the default-priority stream when the rule is off."""
        if not self.low_priority_voxels:
            return self.low_streams[slot]
        nvox = grid[0] * grid[1] * grid[2]
        return (self.low_streams if nvox > self.low_priority_voxels else self.streams)[slot]

    def set_priorities(self, low_priority_voxels):
        """Change the priority rule (None: every context on its slot's default-priority
        stream) and move the cached contexts to the streams it gives.  Call between jobs."""
        self.low_priority_voxels = low_priority_voxels
        with self._lock:
            for slot, per_slot in enumerate(self.contexts):
                for (grid, _), ctx in per_slot.items():
                    ctx.set_stream(self._stream_for(slot, grid).cuda_stream)

    def register_sensitivity(self, key, geometry, grid, lors):
        """Compute a sensitivity image once and keep it on the device."""
        torch = self.torch
        with self._sens_lock:
            if key in self.sens:
                return self.sens[key]
            nvox = grid[0] * grid[1] * grid[2]
            s = torch.zeros(nvox, dtype=torch.float64, device=f"cuda:{self.device}")
            with self.B.Context(geometry, grid) as ctx:
                ctx.sensitivity(lors, s)
            torch.cuda.synchronize(self.device)
            self.sens[key] = s
            return s

    def resident_bytes(self):
        """Device bytes held between jobs: cached contexts and sensitivity images."""
        with self._lock:
            ctx = sum(self.ctx_bytes.values())
        return ctx + sum(int(t.numel()) * t.element_size() for t in self.sens.values())

    def context_bytes(self, slot, job):
        with self._lock:
            return self.ctx_bytes.get((slot, self._key(job)), 0)

    def evict_idle(self, running, need):
        """Close cached contexts no running job uses, least recently used first,
        until at least `need` bytes are freed; returns the bytes freed.
        running: slot -> job of the jobs on the GPU (and just admitted)."""
        busy = {(slot, self._key(job)) for slot, job in running.items()}
        freed = 0
        with self._lock:
            for sk in sorted(self.ctx_bytes, key=lambda k: self.last_used.get(k, 0)):
                if freed >= need:
                    break
                if sk in busy:
                    continue
                slot, key = sk
                ctx = self.contexts[slot].pop(key, None)
                if ctx is not None:
                    ctx.close()
                self.loaded[slot].pop(key, None)
                freed += self.ctx_bytes.pop(sk)
                self.last_used.pop(sk, None)
                self.evicted += 1
        return freed

    def _context(self, slot, job):
        key = self._key(job)
        with self._lock:
            ctx = self.contexts[slot].get(key)
            self._use += 1
            self.last_used[(slot, key)] = self._use
        if ctx is None:
            ctx = self.B.Context(job.geometry, job.grid)
            ctx.set_stream(self._stream_for(slot, job.grid).cuda_stream)
            if self.launch is not None:
                ctx.set_launch(*self.launch)
            with self._lock:
                self.contexts[slot][key] = ctx
                self.ctx_bytes[(slot, key)] = ctx.get_info()["device_bytes"]
        if self.loaded[slot].get(key) != job.sens_key:
            ctx.set_sensitivity(self.sens[job.sens_key])
            self.loaded[slot][key] = job.sens_key
        return ctx

    def warm(self, jobs):
        """Create every (slot, grid) context the jobs need and run one of each kind
        per slot, so that first-use costs stay out of the measured latencies."""
        seen = set()
        for job in jobs:
            for slot in range(len(self.streams)):
                key = (slot, tuple(job.grid), job.sens_key)
                if key in seen:
                    continue
                seen.add(key)
                keep = self.keep_results
                self.keep_results = False
                try:
                    self.run(job, slot)
                finally:
                    self.keep_results = keep

    def run(self, job, slot):
        torch = self.torch
        torch.cuda.set_device(self.device)
        ctx = self._context(slot, job)
        nvox = job.grid[0] * job.grid[1] * job.grid[2]
        img = torch.empty(nvox, dtype=torch.float32).pin_memory() if self.keep_results else None
        cons = np.zeros((job.n_iter, 2))
        try:
            ctx.mlem(self.B.make_events(job.events), job.n_iter, None, img, cons)
        finally:
            with self._lock:
                if self.contexts[slot].get(self._key(job)) is ctx:
                    self.ctx_bytes[(slot, self._key(job))] = ctx.get_info()["device_bytes"]
        job.result = img.numpy() if img is not None else None
        job.conservation = cons

    def close(self):
        with self._lock:
            for per_slot in self.contexts:
                for ctx in per_slot.values():
                    ctx.close()
                per_slot.clear()
            self.ctx_bytes.clear()
            self.last_used.clear()


def poisson_arrivals(n, rate_per_s, seed):
    """Arrival times of a Poisson stream (exponential gaps)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))
