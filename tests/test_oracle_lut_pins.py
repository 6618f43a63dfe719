"""Pins of the oracle's sampled TOF kernel (Sec. 2.3): N equally spaced samples
of the Gaussian, weights in proportion to the Gaussian and summing to one,
each deposited in the voxel that contains it.

Reading of Sec. 2.3 used here: the samples are the midpoints of N equal
intervals of the window [-K sigma, K sigma] (K = 3, the window of the exact
projector), centred on the TOF point M + d u.

Each test checks the oracle against a closed form, a brute-force construction
written in this file, an invariant, or the exact Siddon x Phi projector (pinned
on its own in test_oracle_pins.py) in the limit of many samples.
"""
import math

import numpy as np
import pytest
from scipy.special import ndtr

import oracle
from oracle import Grid

SIGMA = oracle.tof_sigma_mm(300.0)
K = 3.0


def events_from(p1, p2, d):
    p1 = np.atleast_2d(np.asarray(p1, float))
    p2 = np.atleast_2d(np.asarray(p2, float))
    return [p1[:, 0], p1[:, 1], p1[:, 2], p2[:, 0], p2[:, 1], p2[:, 2], np.atleast_1d(np.asarray(d, float))]


@pytest.mark.parametrize("n", [1, 2, 15, 32, 64])
def test_samples_unit_sum_symmetric_equal_spacing(n):
    t, w = oracle.lut_samples(n, SIGMA, K)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.all(w > 0)
    np.testing.assert_allclose(t, -t[::-1], atol=1e-12)
    np.testing.assert_allclose(w, w[::-1], rtol=1e-14)
    if n > 1:
        np.testing.assert_allclose(np.diff(t), 2 * K * SIGMA / n, rtol=1e-12)
    # first and last sample half a spacing inside the window
    assert t[0] == pytest.approx(-K * SIGMA + K * SIGMA / n, rel=1e-14)
    # weights fall off as the Gaussian: w_k / w_0 = exp(-(t_k^2 - t_0^2) / (2 sigma^2))
    ratio = np.exp(-(t ** 2 - t[0] ** 2) / (2 * SIGMA ** 2))
    np.testing.assert_allclose(w / w[0], ratio, rtol=1e-12)


def test_samples_second_moment_converges_to_truncated_normal_variance():
    # Var of N(0,1) truncated to [-K, K] = 1 - 2 K phi(K) / (2 Phi(K) - 1)
    phi = math.exp(-0.5 * K * K) / math.sqrt(2 * math.pi)
    var = SIGMA ** 2 * (1 - 2 * K * phi / (2 * ndtr(K) - 1))
    errs = []
    for n in (32, 256, 2048):
        t, w = oracle.lut_samples(n, SIGMA, K)
        errs.append(abs(np.sum(w * t * t) - var) / var)
    assert errs[-1] < 1e-5
    assert errs[0] > errs[1] > errs[2]          # midpoint rule: error falls as 1/N^2
    assert errs[1] / errs[2] == pytest.approx(64.0, rel=0.05)


def test_axis_line_samples_land_in_bruteforce_voxels():
    # line along +x through voxel centres in y and z: sample k sits at x = d + t_k
    g = Grid(200, 3, 3, 2.0, 2.0, 2.0, -200.0, -3.0, -3.0)
    lam = np.arange(g.n_vox, dtype=float) + 1.0
    for n in (15, 32):
        t, w = oracle.lut_samples(n, SIGMA, K)
        for d in (0.0, 7.3, -41.9, 120.7):
            ev = events_from([500.0, 0.0, 0.0], [-500.0, 0.0, 0.0], d)
            p = oracle.forward_lut(g, ev, lam, n, SIGMA, K)[0]
            ref = 0.0
            for tk, wk in zip(t, w):
                x = d + tk
                ix = math.floor((x - g.ox) / g.vx)
                if 0 <= ix < g.nx:
                    ref += wk * lam[ix + g.nx * (1 + g.ny * 1)]
            assert p == pytest.approx(ref, rel=1e-14)
    # reversed endpoints flip u: the samples of d then sit at x = -(d + t_k)
    t, w = oracle.lut_samples(32, SIGMA, K)
    ev = events_from([-500.0, 0.0, 0.0], [500.0, 0.0, 0.0], 30.0)
    p = oracle.forward_lut(g, ev, lam, 32, SIGMA, K)[0]
    ref = sum(wk * lam[math.floor((-(30.0 + tk) - g.ox) / g.vx) + g.nx * 4] for tk, wk in zip(t, w))
    assert p == pytest.approx(ref, rel=1e-14)


def test_unit_mass_inside_grid_and_clipped_mass_outside():
    g = Grid.centred(64, 64, 64, 4.0)
    rng = np.random.default_rng(11)
    n_ev = 200
    u = rng.normal(size=(n_ev, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    c = rng.uniform(-30, 30, (n_ev, 3))
    d = rng.uniform(-10, 10, n_ev)
    ev = events_from(c + 400 * u, c - 400 * u, d)
    p = oracle.forward_lut(g, ev, np.ones(g.n_vox), 32, SIGMA, K)
    np.testing.assert_allclose(p, 1.0, atol=1e-14)
    # TOF point far outside the grid: no sample lands inside
    far = events_from([0.0, 0.0, 900.0], [0.0, 0.0, -900.0], 600.0)
    assert oracle.forward_lut(g, far, np.ones(g.n_vox), 32, SIGMA, K)[0] == 0.0


def test_lut_adjoint_and_thread_invariance():
    g = Grid(20, 18, 16, 3.0, 3.5, 4.0, -31.0, -30.0, -33.0)
    rng = np.random.default_rng(5)
    n_ev = 3000
    p1 = rng.uniform(-80, 80, (n_ev, 3))
    p2 = rng.uniform(-80, 80, (n_ev, 3))
    ev = events_from(p1, p2, rng.uniform(-40, 40, n_ev))
    lam = rng.uniform(0.5, 2.0, g.n_vox)
    r = rng.uniform(0.0, 1.0, n_ev)
    fp = oracle.forward_lut(g, ev, lam, 32, SIGMA, K)
    bp = oracle.backproject_lut(g, ev, r, 32, SIGMA, K)
    assert np.dot(fp, r) == pytest.approx(np.dot(lam, bp), rel=1e-12)
    bp1 = oracle.backproject_lut(g, ev, r, 32, SIGMA, K, threads=1)
    np.testing.assert_allclose(bp1, bp, rtol=1e-12, atol=1e-15)


def test_many_samples_converge_to_exact_projector():
    # The sampled kernel is a midpoint rule for the integral of the truncated
    # Gaussian along the line; as N grows each voxel's sampled mass tends to
    # its exact TOF mass [Phi(b) - Phi(a)] / (2 Phi(K) - 1).
    g = Grid(24, 24, 24, 4.0, 4.0, 4.0, -48.0, -48.0, -48.0)
    rng = np.random.default_rng(8)
    n_ev = 400
    c = rng.uniform(-10, 10, (n_ev, 3))
    u = rng.normal(size=(n_ev, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    ev = events_from(c + 300 * u, c - 300 * u, rng.uniform(-20, 20, n_ev))
    lam = rng.uniform(0.0, 1.0, g.n_vox)
    exact = oracle.forward(g, ev, lam, SIGMA, K)
    errs = [np.max(np.abs(oracle.forward_lut(g, ev, lam, n, SIGMA, K) - exact) / exact) for n in (32, 512, 8192)]
    assert errs[2] < 2e-3
    assert errs[0] > errs[1] > errs[2]


def test_ambiguous_samples_are_those_near_a_voxel_plane():
    # line along +x through voxel centres in y and z (half a voxel from every y, z
    # plane): sample k sits at x = d + t_k, so its distance to the nearest x plane
    # in voxels is known by hand.  Samples within eps voxels of a plane (the grid's
    # faces included) count; samples more than a voxel outside the grid do not.
    g = Grid(200, 3, 3, 2.0, 2.0, 2.0, -200.0, -3.0, -3.0)
    n = 32
    t, _ = oracle.lut_samples(n, SIGMA, K)
    eps = oracle.LUT_EPS_VOXELS
    on_plane = 10.0 - t[5]                       # sample 5 exactly at x = 10 mm, a plane
    cases = {0.0: None, 7.3: None, on_plane: 1, on_plane + 0.5 * eps * g.vx: 1, on_plane + 4 * eps * g.vx: 0,
             -200.0 - t[0]: 1, 300.0: 0}
    for d, expect_k5 in cases.items():
        ev = events_from([500.0, 0.0, 0.0], [-500.0, 0.0, 0.0], d)
        got = int(oracle.lut_ambiguous(g, ev, n, SIGMA, K)[0])
        q = (d + t - g.ox) / g.vx
        near = np.abs(q - np.round(q)) < eps
        reach = (q >= -1.0) & (q <= g.nx + 1.0)
        assert got == int(np.sum(near & reach)), d
        if expect_k5 is not None and d != -200.0 - t[0]:
            assert bool(near[5] & reach[5]) == bool(expect_k5)
    # the first sample exactly on the grid's low face: inside versus outside is ambiguous
    ev = events_from([500.0, 0.0, 0.0], [-500.0, 0.0, 0.0], -200.0 - t[0])
    assert oracle.lut_ambiguous(g, ev, n, SIGMA, K)[0] >= 1
    # a TOF point far from the grid: nothing to decide
    far = events_from([0.0, 0.0, 900.0], [0.0, 0.0, -900.0], 600.0)
    assert oracle.lut_ambiguous(g, far, n, SIGMA, K)[0] == 0
    # isotropic lines: the share of ambiguous samples is 2 eps per axis crossing
    # the grid, ~6 eps in all
    rng = np.random.default_rng(12)
    gg = Grid.centred(64, 64, 64, 4.0)
    m = 20_000
    u = rng.normal(size=(m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    c = rng.uniform(-40, 40, (m, 3))
    ev = events_from(c + 400 * u, c - 400 * u, rng.uniform(-10, 10, m))
    share = oracle.lut_ambiguous(gg, ev, n, SIGMA, K).sum() / (m * n)
    assert share == pytest.approx(6 * eps, rel=0.15)
