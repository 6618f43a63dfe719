"""Event-sharded MLEM through the C-ABI (recon_event_pass, recon_update): two
ranks as two processes on the one GPU, each holding half of the tiny workload's
events in its own context, sum their C images over gloo through host memory
once per iteration.  Their image must equal one context's recon_mlem over all
events (relative L2 <= 1e-5: the FP32 sums run in another order) and the FP64
oracle's MLEM at the plain gates (Sec. 2.4).  The ranks' kernels never wait on
each other: the only exchange is the host-side all-reduce between passes."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from gpu_common import SIGMA, geometry, grid_tuple, max_rel_above, rel_l2, workload_grid
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_ITER = 4
N_EVENTS = 120_000
SEED = 77


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        import torch
        import torch.distributed as dist
        from paper_1706_07075_b300 import binding as Bb
        from paper_1706_07075_b300 import synth as S
        from paper_1706_07075_b300.shard import sharded_mlem, torch_allreduce_sum
        from gpu_common import geometry as geo, grid_tuple as gt, workload_grid as wg
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
        ev = S.events("tiny", N_EVENTS, SEED, workers=1)
        lors = S.sensitivity_lors("tiny", 400_000, SEED, workers=1)
        shard = np.ascontiguousarray(ev[:, rank::world])
        g = wg("tiny")
        with Bb.Context(geo("tiny"), gt(g), 300.0) as ctx:
            ctx.sensitivity(lors)
            ctx.load_events(Bb.make_events(shard))
            c_buf = torch.zeros(g.n_vox, dtype=torch.float32)
            img = np.zeros(g.n_vox, np.float32)
            hist = sharded_mlem(ctx, N_ITER, c_buf, torch_allreduce_sum(), img)
        q.put((rank, img, hist, None))
        dist.destroy_process_group()
    except Exception as e:  # reported by the parent
        q.put((rank, None, None, repr(e)))


def test_two_ranks_on_one_gpu_equal_one_context_and_the_oracle():
    world = 2
    mpc = mp.get_context("spawn")
    q = mpc.Queue()
    port = _free_port()
    procs = [mpc.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
    for rank, img, hist, err in res:
        assert err is None, (rank, err)
    for p in procs:
        assert p.exitcode == 0
    ev = synth.events("tiny", N_EVENTS, SEED, workers=1)
    lors = synth.sensitivity_lors("tiny", 400_000, SEED, workers=1)
    g = workload_grid("tiny")
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.sensitivity(lors)
        one = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((N_ITER, 2))
        ctx.mlem(B.make_events(ev), N_ITER, None, one, cons)
    lam_ref, hist_ref = oracle.mlem(g, ev.astype(np.float64), oracle.sensitivity(g, lors), N_ITER, SIGMA)
    for rank, img, hist, _ in res:
        assert rel_l2(img, one) <= 1e-5
        assert rel_l2(img, lam_ref) <= 1e-4
        assert max_rel_above(img, lam_ref, 0.01) <= 1e-3
        for k in range(N_ITER):
            assert hist[k][0] == pytest.approx(cons[k, 0], abs=0.5)       # N_eff over both shards
            assert hist[k][1] == pytest.approx(hist[k][0], rel=1e-5)      # sum s lambda = N_eff
    np.testing.assert_array_equal(res[0][1], res[1][1])                  # same image on both ranks


def test_event_pass_and_update_equal_one_mlem_iteration():
    # one context: recon_event_pass + recon_update from the start image reproduce
    # recon_mlem's iterations (same kernels; the uniform start's scale cancels)
    ev = synth.events("tiny", 50_000, 12, workers=1)
    lors = synth.sensitivity_lors("tiny", 200_000, 12, workers=1)
    g = workload_grid("tiny")
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.sensitivity(lors)
        ctx.load_events(B.make_events(ev))
        ref = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((3, 2))
        ctx.mlem(None, 3, None, ref, cons)
        C = np.zeros(g.n_vox, np.float32)
        img = np.zeros(g.n_vox, np.float32)
        for k in range(3):
            n_eff = ctx.event_pass(None, None, 1 if k == 0 else 0, C)
            assert n_eff == pytest.approx(cons[k, 0], abs=0.5)
            ssum = ctx.update(C, img)
            assert ssum == pytest.approx(cons[k, 1], rel=1e-5)
        with pytest.raises(B.ReconError):
            ctx.event_pass(None, None, 0, None)
        with pytest.raises(B.ReconError):
            ctx.update(None)
    assert rel_l2(img, ref) <= 1e-5


def _region_rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        import torch
        import torch.distributed as dist
        from paper_1706_07075_b300 import binding as Bb
        from paper_1706_07075_b300 import synth as S
        from paper_1706_07075_b300.shard import regions_mlem_sharded
        from gpu_common import geometry as geo, grid_tuple as gt, workload_grid as wg
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
        ev = S.events("tiny", N_EVENTS, SEED, workers=1)
        lors = S.sensitivity_lors("tiny", 400_000, SEED, workers=1)
        g = wg("tiny")
        with Bb.Context(geo("tiny"), gt(g), 300.0) as ctx:
            ctx.sensitivity(lors)
            ctx.load_events(Bb.make_events(ev))
            img = torch.zeros(g.n_vox, dtype=torch.float32)
            block = regions_mlem_sharded(ctx, REGIONS, MARGIN, 6.0, N_ITER, img, rank, world,
                                         lambda t: dist.all_reduce(t))
        q.put((rank, img.numpy().copy(), block, None))
        dist.destroy_process_group()
    except Exception as e:  # reported by the parent
        q.put((rank, None, None, repr(e)))


REGIONS = [(0, 16), (16, 32), (32, 48)]
MARGIN = 3.0 * 19.0965 + 6.0


def test_region_sharded_ranks_equal_one_context():
    # regions split over two ranks (one and two regions), the stitched images summed
    # once at the end over gloo: equal to one context that reconstructs all three
    world = 2
    mpc = mp.get_context("spawn")
    q = mpc.Queue()
    port = _free_port()
    procs = [mpc.Process(target=_region_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
    for rank, img, block, err in res:
        assert err is None, (rank, err)
    assert [r[2] for r in res] == [(0, 1), (1, 3)]
    ev = synth.events("tiny", N_EVENTS, SEED, workers=1)
    lors = synth.sensitivity_lors("tiny", 400_000, SEED, workers=1)
    g = workload_grid("tiny")
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.sensitivity(lors)
        one = np.zeros(g.n_vox, np.float32)
        ctx.mlem_regions(B.make_events(ev), REGIONS, MARGIN, 6.0, N_ITER, one)
    for rank, img, _, _ in res:
        assert rel_l2(img, one) <= 1e-5
    np.testing.assert_array_equal(res[0][1], res[1][1])
