"""The event-sharded MLEM driver (paper_1706_07075_b300.shard) on CPU: two gloo
ranks, each with half of the events of a small dense system, must give the
image of textbook MLEM over all events (Sec. 2.4).  The ranks' contexts are
stand-ins that do the event pass and the update in numpy on a dense matrix, so
the test checks the driver's exchange (what is summed, when, and from which
start image) without a GPU."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_ITER = 6


def system(seed=3):
    rng = np.random.default_rng(seed)
    n_ev, n_vox = 400, 64
    A = rng.uniform(0.0, 1.0, (n_ev, n_vox)) * (rng.uniform(size=(n_ev, n_vox)) < 0.2)
    s = A.sum(axis=0) + rng.uniform(0.0, 0.5, n_vox)
    s[:3] = 0.0                                   # voxels outside the mask
    w = np.ones(n_ev)
    return A, s, w


class DenseCtx:
    """Event pass and update of one rank's rows of A, like recon_event_pass and
    recon_update."""

    def __init__(self, A, s, w):
        self.A, self.s, self.w = A, s, w
        self.lam = np.zeros(A.shape[1])

    def event_pass(self, events, image, from_start, c_buf):
        if from_start:
            self.lam = np.where(self.s > 0, 1.0, 0.0)
        p = self.A @ self.lam
        r = np.where(p > 0, self.w / np.where(p > 0, p, 1.0), 0.0)
        c_buf[:] = __import__("torch").from_numpy(self.A.T @ r)
        return float(self.w[p > 0].sum())

    def update(self, c_buf, image_out=None):
        C = c_buf.numpy()
        m = self.s > 0
        new = np.zeros_like(self.lam)
        new[m] = self.lam[m] * C[m] / self.s[m]
        self.lam = new
        if image_out is not None:
            image_out[:] = new
        return float((self.s * new).sum())


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_1706_07075_b300.shard import sharded_mlem, torch_allreduce_sum
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    A, s, w = system()
    rows = np.arange(A.shape[0]) % world == rank            # interleaved shards of unequal content
    ctx = DenseCtx(A[rows], s, w[rows])
    c_buf = torch.zeros(A.shape[1], dtype=torch.float64)
    img = np.zeros(A.shape[1])
    hist = sharded_mlem(ctx, N_ITER, c_buf, torch_allreduce_sum(), img)
    q.put((rank, img, hist))
    dist.destroy_process_group()


def textbook_mlem(A, s, w, n_iter):
    m = s > 0
    lam = np.where(m, w.sum() / s[m].sum(), 0.0)
    for _ in range(n_iter):
        p = A @ lam
        r = np.where(p > 0, w / np.where(p > 0, p, 1.0), 0.0)
        new = np.zeros_like(lam)
        new[m] = lam[m] * (A.T @ r)[m] / s[m]
        lam = new
    return lam


def test_two_gloo_ranks_give_mlem_over_all_events():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    A, s, w = system()
    ref = textbook_mlem(A, s, w, N_ITER)
    for rank, img, hist in res:
        np.testing.assert_allclose(img, ref, rtol=1e-12, atol=1e-15)
        assert len(hist) == N_ITER
        for n_eff, ssum in hist:
            assert n_eff == pytest.approx(w.sum())
            assert ssum == pytest.approx(n_eff, rel=1e-12)        # count conservation over all events
    np.testing.assert_array_equal(res[0][1], res[1][1])            # the ranks hold the same image



def test_region_blocks_cover_every_region_once():
    sys.path.insert(0, ROOT)
    from paper_1706_07075_b300.shard import region_block
    for n in (1, 2, 9, 10):
        for world in (1, 2, 3, 4, 8, 16):
            blocks = [region_block(n, r, world) for r in range(world)]
            covered = [k for lo, hi in blocks for k in range(lo, hi)]
            assert covered == list(range(n))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1
