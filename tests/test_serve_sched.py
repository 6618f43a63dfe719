"""Host-side logic of the continuous-batching server (no GPU): admission by
slots and HBM footprint, first fit in arrival order with an optional
overtake limit, release on completion and on failure, latency bookkeeping."""
import threading
import time

import numpy as np
import pytest

from paper_1706_07075_b300.serve import Job, Server, poisson_arrivals


class FakeExecutor:
    """Sleeps for a job-dependent time and records concurrency and memory use."""

    def __init__(self, server_ref, fail_ids=()):
        self.server_ref = server_ref
        self.fail_ids = set(fail_ids)
        self.lock = threading.Lock()
        self.running = 0
        self.peak_running = 0
        self.peak_bytes = 0
        self.order = []

    def run(self, job, slot):
        srv = self.server_ref[0]
        with self.lock:
            self.running += 1
            self.peak_running = max(self.peak_running, self.running)
            self.peak_bytes = max(self.peak_bytes, srv._in_use)
            self.order.append(job.job_id)
        time.sleep(0.002 * job.n_iter)
        with self.lock:
            self.running -= 1
        if job.job_id in self.fail_ids:
            raise RuntimeError("injected failure")
        job.result = job.job_id


def make_job(i, n_events, arrival=0.0, grid=(10, 10, 10, 1, 1, 1, 0, 0, 0), n_iter=3):
    return Job(i, arrival, np.zeros((7, n_events), np.float32), (100.0, 100.0, 90.0), grid, n_iter)


def test_slots_and_budget_are_never_exceeded():
    ref = [None]
    ex = FakeExecutor(ref)
    budget = 3 * make_job(0, 1_000_000).footprint()
    srv = Server(ex, slots=4, hbm_budget_bytes=budget)
    ref[0] = srv
    jobs = [make_job(i, 1_000_000 if i % 3 else 200_000, arrival=0.001 * i) for i in range(30)]
    stats = srv.replay(jobs)
    assert stats["jobs"] == 30 and all(j.result == j.job_id for j in jobs)
    assert ex.peak_running <= 4
    assert ex.peak_bytes <= budget
    assert stats["max_concurrent"] >= 2                      # work overlapped
    assert all(j.latency >= 0 and j.admitted >= j.arrival - 1e-9 for j in jobs)


def test_first_fit_lets_a_small_job_pass_a_large_one():
    ref = [None]
    ex = FakeExecutor(ref)
    small = make_job(0, 10).footprint()
    big = make_job(1, 10, grid=(1000, 1000, 100, 1, 1, 1, 0, 0, 0))     # 2 GB of images
    srv = Server(ex, slots=3, hbm_budget_bytes=big.footprint() + small)
    ref[0] = srv
    srv.start()
    with srv._lock:
        # occupy part of the budget so that the big job cannot start yet
        srv._in_use = 2 * small
    first = make_job(2, 10, arrival=0.0)
    srv.submit(big)                       # does not fit next to the reserved bytes
    srv.submit(first)                     # fits: admitted although it came later
    time.sleep(0.05)
    assert first.admitted is not None and big.admitted is None
    with srv._lock:
        srv._in_use -= 2 * small
        srv._admit_locked()
    srv.drain(timeout=5)
    assert big.result == 1


def test_overtake_limit_stops_a_large_job_from_starving():
    # with max_overtakes = 1 one later job may pass the waiting large job; the
    # next one waits behind it although it would fit, and both start once the
    # budget frees up for the large job
    ref = [None]
    ex = FakeExecutor(ref)
    small = make_job(0, 10).footprint()
    big = make_job(1, 10, grid=(1000, 1000, 100, 1, 1, 1, 0, 0, 0))
    srv = Server(ex, slots=3, hbm_budget_bytes=big.footprint() + small, max_overtakes=1)
    ref[0] = srv
    srv.start()
    with srv._lock:
        srv._in_use = 2 * small           # reserved: the big job cannot start yet
    s1, s2 = make_job(2, 10, arrival=0.0), make_job(3, 10, arrival=0.0)
    srv.submit(big)
    srv.submit(s1)                        # passes the big job (first overtake)
    srv.submit(s2)                        # would fit, but the big job holds the line
    time.sleep(0.05)
    assert s1.admitted is not None and s1.finished is not None
    assert big.admitted is None and s2.admitted is None
    with srv._lock:
        srv._in_use -= 2 * small
        srv._admit_locked()
    srv.drain(timeout=5)
    assert big.result == 1 and s2.result == 3
    assert big.admitted <= s2.admitted
    with pytest.raises(ValueError):
        Server(ex, max_overtakes=-1)


def test_failed_job_releases_its_slot_and_memory():
    ref = [None]
    ex = FakeExecutor(ref, fail_ids={3})
    srv = Server(ex, slots=2, hbm_budget_bytes=make_job(0, 1000).footprint() * 2)
    ref[0] = srv
    jobs = [make_job(i, 1000, arrival=0.0) for i in range(6)]
    srv.start()
    for j in jobs:
        srv.submit(j)
    with pytest.raises(RuntimeError, match="injected failure"):
        srv.drain(timeout=5)
    assert srv._in_use == 0 and sorted(srv._free_slots) == [0, 1]
    assert sum(1 for j in jobs if j.result is not None) == 5


def test_oversized_job_is_rejected_and_stats():
    ref = [None]
    srv = Server(FakeExecutor(ref), slots=1, hbm_budget_bytes=1000)
    ref[0] = srv
    with pytest.raises(ValueError):
        srv.submit(make_job(0, 10))
    t = poisson_arrivals(1000, 50.0, 3)
    assert np.all(np.diff(t) > 0) and abs(1000 / t[-1] - 50.0) < 10.0


class CachingExecutor:
    """Keeps one context per (slot, grid) that grows to the largest job it ran,
    like LibreconExecutor, and records the device bytes all contexts hold."""

    def __init__(self, resident_extra=0):
        self.lock = threading.Lock()
        self.ctx = {}                 # (slot, grid) -> bytes
        self.used = {}
        self.tick = 0
        self.extra = resident_extra   # e.g. sensitivity images
        self.peak_actual = 0
        self.evicted = 0

    def resident_bytes(self):
        with self.lock:
            return sum(self.ctx.values()) + self.extra

    def context_bytes(self, slot, job):
        with self.lock:
            return self.ctx.get((slot, job.grid), 0)

    def evict_idle(self, running, need):
        busy = {(s, j.grid) for s, j in running.items()}
        freed = 0
        with self.lock:
            for k in sorted(self.ctx, key=lambda k: self.used[k]):
                if freed >= need:
                    break
                if k not in busy:
                    freed += self.ctx.pop(k)
                    self.evicted += 1
        return freed

    def run(self, job, slot):
        with self.lock:
            k = (slot, job.grid)
            self.ctx[k] = max(self.ctx.get(k, 0), job.footprint())      # the context grows
            self.tick += 1
            self.used[k] = self.tick
            self.peak_actual = max(self.peak_actual, sum(self.ctx.values()) + self.extra)
        time.sleep(0.003)
        job.result = job.job_id


def test_cached_contexts_count_against_the_budget():
    # contexts stay allocated after their jobs; with a budget that binds, the
    # server charges them, evicts idle ones and never lets the device memory
    # the executor holds exceed the budget
    grids = [(10 * (k + 1), 10, 10, 1, 1, 1, 0, 0, 0) for k in range(4)]
    sizes = [make_job(0, 400_000, grid=g).footprint() for g in grids]
    ex = CachingExecutor(resident_extra=1000)
    budget = int(2.2 * max(sizes)) + 1000
    srv = Server(ex, slots=3, hbm_budget_bytes=budget)
    jobs = [make_job(i, 400_000, arrival=0.0005 * i, grid=grids[i % 4]) for i in range(40)]
    stats = srv.replay(jobs)
    assert stats["jobs"] == 40 and all(j.result == j.job_id for j in jobs)
    assert ex.peak_actual <= budget
    assert stats["peak_charged_bytes"] <= budget
    assert ex.evicted > 0                         # the budget did bind
    assert stats["max_concurrent"] >= 2


def test_a_job_that_cannot_fit_beside_resident_state_fails_instead_of_waiting():
    ex = CachingExecutor(resident_extra=900)
    job = make_job(0, 10)
    srv = Server(ex, slots=1, hbm_budget_bytes=job.footprint() + 100)
    srv.start()
    srv.submit(job)
    with pytest.raises(RuntimeError, match="does not fit"):
        srv.drain(timeout=5)
