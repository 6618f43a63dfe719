"""Pins of the oracle's median-filter sieve (Sec. 2.4): against scipy's
median filter (an independent library routine), closed forms on constant
images at faces, edges and corners (zero padding outside the grid), impulse
removal, ramps, and the mask rule."""
import numpy as np
import pytest
from scipy import ndimage

import oracle


@pytest.mark.parametrize("shape", [(5, 4, 6), (7, 9, 3), (1, 1, 1), (2, 3, 1)])
def test_median3_matches_scipy(shape):
    rng = np.random.default_rng(sum(shape))
    img = rng.uniform(0, 1, shape)
    img[rng.uniform(size=shape) < 0.3] = 0.0          # ties at zero
    ref = ndimage.median_filter(img, size=3, mode="constant", cval=0.0)
    out = oracle.median3(img.ravel(), shape).reshape(shape)
    assert np.array_equal(out, ref)


def test_median3_constant_image_faces_edges_corners():
    c = 2.5
    shape = (6, 7, 8)
    out = oracle.median3(np.full(int(np.prod(shape)), c), shape).reshape(shape)
    # inside: 27 of 27 neighbours are c; face: 18 of 27; edge: 12; corner: 8.
    # The 14th smallest of 27 is c when at most 13 zeros are present.
    assert out[2, 3, 4] == c
    assert out[0, 3, 4] == c and out[2, 0, 4] == c and out[2, 3, 7] == c      # faces: 9 zeros
    assert out[0, 0, 4] == 0.0 and out[5, 3, 0] == 0.0                         # edges: 15 zeros
    assert out[0, 0, 0] == 0.0 and out[5, 6, 7] == 0.0                         # corners: 19 zeros


def test_median3_removes_impulse_and_keeps_ramp():
    shape = (5, 5, 5)
    img = np.ones(shape)
    img[2, 2, 2] = 1000.0
    out = oracle.median3(img.ravel(), shape).reshape(shape)
    assert out[2, 2, 2] == 1.0
    ramp = np.broadcast_to(np.arange(9.0)[None, None, :], (7, 7, 9)).copy()
    outr = oracle.median3(ramp.ravel(), ramp.shape).reshape(ramp.shape)
    # interior of a linear ramp: the neighbourhood holds x-1, x, x+1 nine times each
    np.testing.assert_array_equal(outr[1:-1, 1:-1, 1:-1], ramp[1:-1, 1:-1, 1:-1])


def test_sieve_keeps_mask_zero():
    shape = (4, 5, 6)
    rng = np.random.default_rng(3)
    lam = rng.uniform(1, 2, shape).ravel()
    s = np.ones_like(lam)
    s[:10] = 0.0
    lam[:10] = 0.0
    out = oracle.sieve(lam, s, shape)
    assert np.all(out[:10] == 0.0)
    assert np.all(out[10:][s[10:] > 0] >= 0.0)


def test_mlem_with_sieve_runs_filter_after_each_update():
    # one iteration with the sieve equals one plain iteration followed by the sieve
    from paper_1706_07075_b300 import synth
    g = oracle.Grid(*synth.grid_of("tiny"))
    ev = synth.events("tiny", 3000, 9).astype(np.float64)
    lors = synth.sensitivity_lors("tiny", 20000, 9)
    s = oracle.sensitivity(g, lors)
    sigma = oracle.tof_sigma_mm(300.0)
    lam1, h1 = oracle.mlem(g, ev, s, 1, sigma)
    lam2, h2 = oracle.mlem(g, ev, s, 1, sigma, median=True)
    assert np.array_equal(lam2, oracle.sieve(lam1, s, g.shape_zyx))
    assert h1 == h2


def test_median3_at_equals_median3():
    shape = (6, 5, 7)
    rng = np.random.default_rng(12)
    img = rng.uniform(0, 1, shape).ravel()
    full = oracle.median3(img, shape)
    vox = rng.choice(img.size, 60, replace=False)
    assert np.array_equal(oracle.median3_at(img, shape, vox), full[vox])
