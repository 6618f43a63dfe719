"""recon_split_regions_noalloc: the region split for callers that cannot
allocate device memory (a CUDA graph being recorded that must not gain
allocation nodes, or a process whose GPU memory belongs to another
allocator).  It must give exactly what the allocating entry point
recon_split_regions gives — region codes, offsets and index lists are integer
results, compared bit for bit — on two calls in a row with different inputs,
since the two calls share the library's static scratch array.

This file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

from gpu_common import geometry, grid_tuple, workload_grid
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

pytestmark = pytest.mark.gpu

REGIONS = [(0, 67), (67, 134), (134, 200), (200, 267), (267, 334), (334, 400), (400, 467), (467, 534), (534, 600)]


def split_with_context(ev, regions, shell):
    g = workload_grid("fullbody")
    n = ev.shape[1]
    with B.Context(geometry("fullbody"), grid_tuple(g), 300.0) as ctx:
        codes = np.zeros(n, np.uint8)
        offs = np.zeros(len(regions) + 1, np.int64)
        ctx.split_regions(B.make_events(ev), regions, 0.0, shell, codes, offs, None)
        idx = np.zeros(max(1, int(offs[-1])), np.int32)
        ctx.split_regions(None, regions, 0.0, shell, None, None, idx)
    return codes, offs, idx[: int(offs[-1])]


def split_without_allocation(ev, regions, shell):
    n = ev.shape[1]
    g = B.recon_grid(*grid_tuple(workload_grid("fullbody")))
    dev = torch.from_numpy(ev).cuda()
    codes = torch.full((max(n, 1),), 7, dtype=torch.uint8, device="cuda")       # stale contents on purpose
    cap = 2 * n + 1
    idx = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    offs = np.zeros(len(regions) + 1, np.int64)
    B.recon_split_regions_noalloc(g, B.make_events(dev), regions, shell, codes, offs, idx, cap)
    torch.cuda.synchronize()
    return codes.cpu().numpy()[:n], offs, idx.cpu().numpy()[: int(offs[-1])]


def test_noalloc_split_matches_allocating_split_twice():
    cases = [(synth.events("fullbody", 2_000_003, 51), REGIONS, 6.0),
             (synth.events("fullbody", 777_777, 52), [(0, 150), (150, 300), (300, 450), (450, 600)], 10.0)]
    for ev, regions, shell in cases:
        ref = split_with_context(ev, regions, shell)
        got = split_without_allocation(ev, regions, shell)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        assert got[1][-1] > 0.9 * ev.shape[1]


def test_noalloc_split_rejects_sizes_beyond_its_scratch():
    g = B.recon_grid(*grid_tuple(workload_grid("fullbody")))
    dev = torch.zeros((7, 64), dtype=torch.float32, device="cuda")
    ev = B.make_events(dev)
    ev.n = 400_000_000                     # beyond the 64-region limit; rejected before any device access
    regions = [(k, k + 1) for k in range(64)]
    offs = np.zeros(65, np.int64)
    with pytest.raises(B.ReconError) as e:
        B.recon_split_regions_noalloc(g, ev, regions, 0.0, dev, offs, dev, 0)
    assert e.value.status == B.RECON_EINVAL
    assert "scratch limit" in B.recon_last_error(None)
    host = B.make_events(np.zeros((7, 4), np.float32))
    with pytest.raises(B.ReconError):
        B.recon_split_regions_noalloc(g, host, REGIONS, 6.0, dev, offs, dev, 0)   # events must be on the device
