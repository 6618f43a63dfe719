"""GPU median-filter sieve (Sec. 2.4) vs the oracle.

The filter is pure selection (min/max), so on the same FP32 image the GPU
result equals the oracle's bit for bit.  Inside MLEM the sieve runs after
each update; the median is 1-Lipschitz in the max norm, so the FP32-vs-FP64
difference of the iterates passes through it without growth and the MLEM
tolerances of the plain parity tests apply unchanged.
"""
import numpy as np
import pytest

import oracle
from gpu_common import SIGMA, geometry, grid_tuple, max_rel_above, rel_l2, tiny_inputs, workload_grid
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

pytestmark = pytest.mark.gpu


def random_image(n, seed, zero_frac=0.2):
    rng = np.random.default_rng(seed)
    img = rng.uniform(0.0, 4.0, n).astype(np.float32)
    img[rng.uniform(size=n) < zero_frac] = 0.0
    img[rng.uniform(size=n) < 0.1] = 1.0                   # ties
    return img


@pytest.mark.parametrize("grid", [(32, 32, 48, 4.0), (37, 19, 23, 2.0), (1, 1, 1, 4.0), (33, 9, 17, 3.0),
                                  (150, 7, 40, 4.0)])
def test_median_filter_bitexact(grid):
    nx, ny, nz, v = grid
    g = (nx, ny, nz, v, v, v, -nx * v / 2, -ny * v / 2, -nz * v / 2)
    n = nx * ny * nz
    img = random_image(n, n)
    out = np.zeros(n, np.float32)
    with B.Context(geometry("tiny"), g, 300.0) as ctx:
        ctx.median_filter(img, out)
    ref = oracle.median3(img.astype(np.float64), (nz, ny, nx))
    assert np.array_equal(out, ref.astype(np.float32))


def test_median_filter_fullbody_grid_sampled():
    g = workload_grid("fullbody")
    img = random_image(g.n_vox, 77)
    out = np.zeros(g.n_vox, np.float32)
    with B.Context(geometry("fullbody"), grid_tuple(g), 300.0) as ctx:
        ctx.median_filter(img, out)
        again = img.copy()                  # in place: input and output may alias
        ctx.median_filter(again, again)
    assert np.array_equal(again, out)
    rng = np.random.default_rng(78)
    vox = np.concatenate([rng.choice(g.n_vox, 200_000, replace=False),
                          np.arange(0, 2 * g.nx * g.ny), np.arange(g.n_vox - 2 * g.nx * g.ny, g.n_vox)])
    ref = oracle.median3_at(img.astype(np.float64), g.shape_zyx, vox)
    assert np.array_equal(out[vox], ref.astype(np.float32))


@pytest.mark.parametrize("graphs", [1, 0])
def test_mlem_with_sieve_matches_oracle(graphs):
    ev, lors = tiny_inputs()
    g = workload_grid("tiny")
    s_ref = oracle.sensitivity(g, lors)
    lam_ref, hist = oracle.mlem(g, ev.astype(np.float64), s_ref, 5, SIGMA, median=True)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        ctx.set_median_filter(1)
        ctx.set_graphs(graphs)
        lam = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((5, 2))
        ctx.mlem(B.make_events(ev), 5, None, lam, cons)
    assert rel_l2(lam, lam_ref) <= 1e-4
    assert max_rel_above(lam, lam_ref, 0.01) <= 1e-3
    assert np.all(lam[s_ref <= 0] == 0)
    for k in range(5):
        assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)
        assert cons[k, 1] == pytest.approx(hist[k][1], rel=1e-5)      # sum s lambda of the update


def test_region_mlem_with_sieve_matches_oracle():
    ev = synth.events("tiny", 120_000, 29)
    lors = synth.sensitivity_lors("tiny", 500_000, 29)
    g = workload_grid("tiny")
    regions = [(0, 16), (16, 32), (32, 48)]
    margin = 3.0 * SIGMA + 6.0
    s_ref = oracle.sensitivity(g, lors)
    img_ref, imgs_ref, hists, codes, offs, idx = oracle.mlem_regions(g, ev.astype(np.float64), s_ref, regions, 6.0,
                                                                     margin, 3, SIGMA, median=True)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        ctx.set_median_filter(1)
        nslab = ctx.region_slab_voxels(regions, margin)
        img = np.zeros(g.n_vox, np.float32)
        slabs = np.zeros(nslab, np.float32)
        cons = np.zeros((3, 3, 2))
        ctx.mlem_regions(B.make_events(ev), regions, margin, 6.0, 3, img, slabs, cons)
    assert rel_l2(slabs, np.concatenate(imgs_ref)) <= 1e-4
    assert rel_l2(img, img_ref) <= 1e-4
    assert max_rel_above(img, img_ref, 0.01) <= 1e-3
    for r in range(3):
        for k in range(3):
            assert cons[k, r, 0] == pytest.approx(hists[r][k][0], abs=0.5)


def test_median_filter_argument_checks():
    g = workload_grid("tiny")
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        with pytest.raises(B.ReconError):
            ctx.median_filter(None, np.zeros(g.n_vox, np.float32))
