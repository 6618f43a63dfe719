"""Pins of the oracle's pre-processing: attenuation weights exp(integral of mu
along the LOR) (Sec. 2.4) and TOF scatter rejection at 95% confidence
(Sec. 2.2): closed-form chords through a box-shaped body, and hand-built
events inside, outside and on both sides of the +-1.96 sigma edge."""
import numpy as np
import pytest

import oracle
from oracle import Grid

SIGMA = oracle.tof_sigma_mm(300.0)
Z95 = 1.96


def events_from(p1, p2, d):
    p1 = np.atleast_2d(np.asarray(p1, float))
    p2 = np.atleast_2d(np.asarray(p2, float))
    return [p1[:, 0], p1[:, 1], p1[:, 2], p2[:, 0], p2[:, 1], p2[:, 2], np.atleast_1d(np.asarray(d, float))]


def box_body(grid, lo_idx, hi_idx, mu):
    """mu inside the voxel box [lo_idx, hi_idx) (x, y, z index ranges), 0 elsewhere."""
    m = np.zeros(grid.shape_zyx)
    m[lo_idx[2]:hi_idx[2], lo_idx[1]:hi_idx[1], lo_idx[0]:hi_idx[0]] = mu
    lo = np.array([grid.ox + lo_idx[0] * grid.vx, grid.oy + lo_idx[1] * grid.vy, grid.oz + lo_idx[2] * grid.vz])
    hi = np.array([grid.ox + hi_idx[0] * grid.vx, grid.oy + hi_idx[1] * grid.vy, grid.oz + hi_idx[2] * grid.vz])
    return m.ravel(), lo, hi


def slab_chord(lo, hi, p1, p2):
    """Length of the line through p1, p2 inside the box [lo, hi] (slab method)."""
    M = 0.5 * (p1 + p2)
    u = (p1 - p2) / np.linalg.norm(p1 - p2)
    a, b = -np.inf, np.inf
    for k in range(3):
        if u[k] == 0:
            if not (lo[k] <= M[k] < hi[k]):
                return 0.0
            continue
        t0, t1 = (lo[k] - M[k]) / u[k], (hi[k] - M[k]) / u[k]
        a, b = max(a, min(t0, t1)), min(b, max(t0, t1))
    return max(0.0, b - a)


def test_attenuation_weight_is_exp_of_mu_times_body_chord():
    g = Grid(24, 20, 16, 4.0, 5.0, 6.0, -48.0, -50.0, -48.0)
    mu0 = 0.0096                                  # water, 1/mm
    mu, lo, hi = box_body(g, (4, 3, 2), (19, 16, 13), mu0)
    rng = np.random.default_rng(1)
    n = 300
    p1 = rng.uniform(-300, 300, (n, 3))
    p2 = -p1 + rng.uniform(-40, 40, (n, 3))
    ev = events_from(p1, p2, np.zeros(n))
    w, keep, kept = oracle.preprocess(g, ev, mu, SIGMA, z=0.0)
    assert kept == n and np.all(keep == 1)
    ref = np.exp(mu0 * np.array([slab_chord(lo, hi, p1[i], p2[i]) for i in range(n)]))
    np.testing.assert_allclose(w, ref, rtol=1e-12)


def test_zero_mu_gives_unit_weight_and_rejects_everything():
    g = Grid.centred(10, 10, 10, 4.0)
    ev = events_from([[-100.0, 1.0, 2.0]] * 3, [[100.0, 1.0, 2.0]] * 3, [0.0, 5.0, -7.0])
    w, keep, kept = oracle.preprocess(g, ev, np.zeros(g.n_vox), SIGMA, z=0.0)
    np.testing.assert_array_equal(w, 1.0)
    w, keep, kept = oracle.preprocess(g, ev, np.zeros(g.n_vox), SIGMA, z=Z95)
    assert kept == 0 and np.all(w == 0) and np.all(keep == 0)


def test_rejection_at_the_95_percent_edge():
    # body: x in [-40, 40) (voxels 10..29 of 4 mm), all y, z; line along +x through y = z = 2
    g = Grid(40, 10, 10, 4.0, 4.0, 4.0, -80.0, -20.0, -20.0)
    mu, lo, hi = box_body(g, (10, 0, 0), (30, 10, 10), 0.01)
    half = Z95 * SIGMA                             # 37.43 mm
    # the TOF point sits at x = d (u = +x, M = origin); the window is [d - half, d + half]
    cases = {
        0.0: 1,                                    # inside the body
        39.9: 1,                                   # inside, near the edge
        40.0 + half - 0.01: 1,                     # window still reaches x < 40 by 0.01 mm
        40.0 + half + 0.01: 0,                     # window ends 0.01 mm past the body
        -40.0 - half + 0.01: 1,
        -40.0 - half - 0.01: 0,
        75.0: 1,                                   # TOF point outside the body but inside +-1.96 sigma of it
        120.0: 0,
    }
    d = np.array(list(cases))
    n = d.size
    ev = events_from(np.tile([300.0, 2.0, 2.0], (n, 1)), np.tile([-300.0, 2.0, 2.0], (n, 1)), d)
    w, keep, kept = oracle.preprocess(g, ev, mu, SIGMA, z=Z95)
    np.testing.assert_array_equal(keep, np.array(list(cases.values()), np.uint8))
    assert kept == sum(cases.values())
    np.testing.assert_allclose(w[keep == 1], np.exp(0.01 * 80.0), rtol=1e-13)
    assert np.all(w[keep == 0] == 0)
    # reversed endpoints flip u: the same events with P1 and P2 swapped and d negated
    ev2 = events_from(np.tile([-300.0, 2.0, 2.0], (n, 1)), np.tile([300.0, 2.0, 2.0], (n, 1)), -d)
    w2, keep2, _ = oracle.preprocess(g, ev2, mu, SIGMA, z=Z95)
    np.testing.assert_array_equal(keep2, keep)
    np.testing.assert_allclose(w2, w, rtol=1e-13)


def test_lines_missing_the_grid():
    g = Grid.centred(8, 8, 8, 4.0)
    ev = events_from([[100.0, 100.0, 0.0]], [[100.0, -100.0, 0.0]], [0.0])
    w, keep, kept = oracle.preprocess(g, ev, np.ones(g.n_vox), SIGMA, z=Z95)
    assert kept == 0 and w[0] == 0.0
    w, keep, kept = oracle.preprocess(g, ev, np.ones(g.n_vox), SIGMA, z=0.0)
    assert kept == 1 and w[0] == 1.0
