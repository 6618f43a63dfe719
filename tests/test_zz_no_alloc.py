"""recon_split_regions_noalloc: the region split for callers that cannot
allocate device memory — a process whose GPU memory belongs to another
allocator (a framework's caching pool, an acquisition service that reserves
the whole GPU at start-up), or a real-time path that cannot wait for cudaFree
or risk an allocation failing half-way through a scan.

It must give exactly what the allocating entry point recon_split_regions gives
(region codes, offsets and index lists are integer results, compared bit for
bit) on two calls in a row with different inputs, since the two calls share
the library's static scratch array.  Once a first call has loaded the library's
kernels and its static array, further calls leave the device's free memory
unchanged.  Host memory passed as a device buffer is rejected before any kernel
runs.

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


def device_buffers(ev):
    """Device events, codes with stale contents on purpose, and an index list of
    twice the events (every event can feed two regions)."""
    n = ev.shape[1]
    dev = torch.from_numpy(ev).cuda()
    codes = torch.full((max(n, 1),), 7, dtype=torch.uint8, device="cuda")
    cap = 2 * n + 1
    idx = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    return dev, codes, idx, cap


def split_without_allocation(bufs, regions, shell, stream=None):
    dev, codes, idx, cap = bufs
    g = B.recon_grid(*grid_tuple(workload_grid("fullbody")))
    offs = np.zeros(len(regions) + 1, np.int64)
    handle = stream.cuda_stream if stream is not None else None
    B.recon_split_regions_noalloc(g, B.make_events(dev), regions, shell, codes, offs, idx, cap, handle)
    torch.cuda.synchronize()
    n = dev.shape[1]
    return codes.cpu().numpy()[:n], offs, idx.cpu().numpy()[: int(offs[-1])]


def test_noalloc_split_matches_allocating_split_twice():
    cases = [(synth.events("fullbody", 2_000_003, 51), REGIONS, 6.0),
             (synth.events("fullbody", 777_777, 52), [(0, 150), (150, 300), (300, 450), (450, 600)], 10.0)]
    for ev, regions, shell in cases:
        ref = split_with_context(ev, regions, shell)
        got = split_without_allocation(device_buffers(ev), regions, shell)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        assert got[1][-1] > 0.9 * ev.shape[1]


def test_noalloc_split_allocates_nothing_on_a_side_stream():
    # a first call loads the library's kernels and its static array; after it the
    # device's free memory stays the same over further calls, which here run on a
    # non-default torch stream and must still match the allocating split
    ev = synth.events("fullbody", 1_234_567, 53)
    ref = split_with_context(ev, REGIONS, 6.0)
    bufs = device_buffers(ev)
    side = torch.cuda.Stream()
    split_without_allocation(bufs, REGIONS, 6.0, side)               # warm call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        got = split_without_allocation(bufs, REGIONS, 6.0, side)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_split_rejects_host_buffers_before_any_kernel():
    ev = synth.events("fullbody", 4096, 54)
    dev, codes, idx, cap = device_buffers(ev)
    g = B.recon_grid(*grid_tuple(workload_grid("fullbody")))
    offs = np.zeros(len(REGIONS) + 1, np.int64)
    host_codes = np.zeros(ev.shape[1], np.uint8)
    with pytest.raises(B.ReconError) as e:
        B.recon_split_regions_noalloc(g, B.make_events(dev), REGIONS, 6.0, host_codes, offs, idx, cap)
    assert e.value.status == B.RECON_EINVAL
    assert "code_out" in B.recon_last_error(None)
    pinned_idx = torch.zeros(cap, dtype=torch.int32).pin_memory()
    with pytest.raises(B.ReconError) as e:
        B.recon_split_regions_noalloc(g, B.make_events(dev), REGIONS, 6.0, codes, offs, pinned_idx, cap)
    assert e.value.status == B.RECON_EINVAL
    assert "idx_out" in B.recon_last_error(None)
    # events that claim to be on the device but are host memory
    host_ev = B.make_events(ev)
    host_ev.on_device = 1
    with pytest.raises(B.ReconError) as e:
        B.recon_split_regions_noalloc(g, host_ev, REGIONS, 6.0, codes, offs, idx, cap)
    assert e.value.status == B.RECON_EINVAL
    assert "event plane" in B.recon_last_error(None)
    # the library still works after the rejections
    got = split_without_allocation((dev, codes, idx, cap), REGIONS, 6.0)
    ref = split_with_context(ev, REGIONS, 6.0)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


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
