"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
value printed in the paper (tests/golden), a closed form, an independent
brute-force construction written in this file, a library routine (scipy), or
an invariant of the method.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import ndtr

import oracle
from oracle import Grid
from paper_1706_07075_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ------------------------------------------------------------ brute force

def brute_segments(grid, p1, p2, t_lo=-np.inf, t_hi=np.inf):
    """Per-voxel intersection of the line with every half-open voxel box.

    The line is M + t u with M = (P1 + P2)/2 and u = (P1 - P2)/|P1 - P2|.
    Returns {linear voxel index: (t_a, t_b)} for positive-length pieces.
    """
    p1 = np.asarray(p1, float)
    p2 = np.asarray(p2, float)
    M = 0.5 * (p1 + p2)
    u = (p1 - p2) / np.linalg.norm(p1 - p2)
    iz, iy, ix = np.meshgrid(np.arange(grid.nz), np.arange(grid.ny), np.arange(grid.nx), indexing="ij")
    idx = [ix.ravel(), iy.ravel(), iz.ravel()]
    org = [grid.ox, grid.oy, grid.oz]
    vox = [grid.vx, grid.vy, grid.vz]
    a = np.full(idx[0].size, -np.inf)
    b = np.full(idx[0].size, np.inf)
    inside = np.ones(idx[0].size, bool)
    for k in range(3):
        lo = org[k] + idx[k] * vox[k]
        hi = org[k] + (idx[k] + 1) * vox[k]
        if u[k] == 0.0:
            inside &= (M[k] >= lo) & (M[k] < hi)
            continue
        t0 = (lo - M[k]) / u[k]
        t1 = (hi - M[k]) / u[k]
        a = np.maximum(a, np.minimum(t0, t1))
        b = np.minimum(b, np.maximum(t0, t1))
    a = np.maximum(a, t_lo)
    b = np.minimum(b, t_hi)
    keep = inside & (b > a)
    lin = idx[0] + grid.nx * (idx[1] + grid.ny * idx[2])
    return {int(j): (float(x), float(y)) for j, x, y in zip(lin[keep], a[keep], b[keep])}


def box_chord(grid, p1, p2):
    """Length of the line inside the whole grid box (slab method)."""
    p1 = np.asarray(p1, float)
    p2 = np.asarray(p2, float)
    M = 0.5 * (p1 + p2)
    u = (p1 - p2) / np.linalg.norm(p1 - p2)
    lo = np.array([grid.ox, grid.oy, grid.oz])
    hi = lo + np.array([grid.nx * grid.vx, grid.ny * grid.vy, grid.nz * grid.vz])
    a, b = -np.inf, np.inf
    for k in range(3):
        if u[k] == 0.0:
            if not (lo[k] <= M[k] < hi[k]):
                return 0.0, None, None
            continue
        t0, t1 = sorted(((lo[k] - M[k]) / u[k], (hi[k] - M[k]) / u[k]))
        a, b = max(a, t0), min(b, t1)
    return max(0.0, b - a), a, b


def trunc_gauss_mass(a, b, K):
    """Mass on [a, b] (sigma units) of the standard normal truncated to +-K."""
    return (ndtr(b) - ndtr(a)) / (ndtr(K) - ndtr(-K))


def random_lines(rng, n, half):
    p1 = rng.uniform(-half, half, (n, 3))
    p2 = rng.uniform(-half, half, (n, 3))
    return p1, p2


ODD_GRID = Grid(5, 4, 6, 3.0, 2.5, 4.0, -7.0, -4.5, -11.0)   # anisotropic, off-centre


def events_from(p1, p2, d):
    p1 = np.atleast_2d(p1)
    p2 = np.atleast_2d(p2)
    return [p1[:, 0], p1[:, 1], p1[:, 2], p2[:, 0], p2[:, 1], p2[:, 2], np.atleast_1d(np.asarray(d, float))]


# ------------------------------------------------------------ constants

def test_sigma_matches_paper_value():
    g = golden("paper_constants.json")
    s = oracle.tof_sigma_mm(g["tof_fwhm_ps"]["value"])
    assert abs(s / g["sigma_mm_for_300ps"]["value"] - 1.0) < g["sigma_mm_for_300ps"]["rel_tol"]


def test_sigma_closed_form_scaling():
    # FWHM of a Gaussian is 2 sqrt(2 ln 2) sigma, and d = c dt / 2 halves it.
    s1, s2 = oracle.tof_sigma_mm(100.0), oracle.tof_sigma_mm(600.0)
    assert s2 == pytest.approx(6.0 * s1, rel=1e-14)
    assert s1 == pytest.approx(0.5 * 29.9792458 / 2.3548200450309493, rel=1e-12)


def test_tof_weight_is_truncated_normal_mass():
    rng = np.random.default_rng(1)
    sigma, K = 19.0965, 3.0
    for _ in range(200):
        d = rng.uniform(-50, 50)
        ta, tb = np.sort(rng.uniform(d - K * sigma, d + K * sigma, 2))
        ref = trunc_gauss_mass((ta - d) / sigma, (tb - d) / sigma, K)
        assert oracle.tof_weight(ta, tb, d, sigma, K) == pytest.approx(ref, rel=1e-12, abs=1e-16)
    # the whole window has unit mass; an asymmetric piece pins the sign of d
    assert oracle.tof_weight(-K * sigma + 3.0, K * sigma + 3.0, 3.0, sigma, K) == pytest.approx(1.0, abs=1e-15)
    w = oracle.tof_weight(0.0, 10.0, 5.0, sigma, K)
    assert w == pytest.approx(trunc_gauss_mass(-5 / sigma, 5 / sigma, K), rel=1e-12)
    w_off = oracle.tof_weight(0.0, 10.0, 30.0, sigma, K)
    assert w_off == pytest.approx(trunc_gauss_mass(-30 / sigma, -20 / sigma, K), rel=1e-12)


# ------------------------------------------------------------ ray tracing

@pytest.mark.parametrize("seed", range(4))
def test_trace_matches_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    g = ODD_GRID
    p1, p2 = random_lines(rng, 60, 25.0)
    for a, b in zip(p1, p2):
        t_lo, t_hi = (-np.inf, np.inf) if rng.uniform() < 0.5 else np.sort(rng.uniform(-20, 20, 2))
        vox, ta, tb = oracle.trace(g, a, b, t_lo, t_hi)
        ref = brute_segments(g, a, b, t_lo, t_hi)
        got = {int(j): (x, y) for j, x, y in zip(vox, ta, tb) if y - x > 1e-12}
        ref = {j: v for j, v in ref.items() if v[1] - v[0] > 1e-12}
        assert set(got) == set(ref)
        for j in ref:
            assert got[j][0] == pytest.approx(ref[j][0], abs=1e-11)
            assert got[j][1] == pytest.approx(ref[j][1], abs=1e-11)
        assert np.all(np.diff(ta) >= 0) and np.all(tb >= ta)


def test_count_visits_matches_bruteforce_pieces():
    # the work unit of the measurement: the number of positive-length voxel pieces
    # inside the TOF windows, counted by brute force over every voxel box
    rng = np.random.default_rng(77)
    g = ODD_GRID
    sigma, K = 3.0, 3.0
    p1, p2 = random_lines(rng, 120, 12.0)
    d = rng.uniform(-6.0, 6.0, 120)
    brute = 0
    for a, b, di in zip(p1, p2, d):
        brute += len(brute_segments(g, a, b, di - K * sigma, di + K * sigma))
    assert brute > 200
    assert oracle.count_visits(g, events_from(p1, p2, d), sigma, K) == brute
    # axis-parallel closed form: a line along x through voxel centres, window inside
    # the grid from x = -5.5 to x = 5.5 (planes at -4, -1, 2, 5): 5 pieces
    y, z = -4.5 + 1.25, -11.0 + 2.0
    ev = events_from([100.0, y, z], [-100.0, y, z], [0.0])
    assert oracle.count_visits(g, ev, 5.5 / K, K) == 5


def test_trace_axis_parallel_index_convention():
    g = ODD_GRID
    # along z through voxel column (ix, iy) = (3, 1)
    x, y = -7.0 + 3.5 * 3.0, -4.5 + 1.5 * 2.5
    vox, ta, tb = oracle.trace(g, [x, y, 100.0], [x, y, -100.0])
    assert list(vox) == [3 + 5 * (1 + 4 * k) for k in range(6)]
    assert np.allclose(tb - ta, 4.0, atol=1e-12)
    # P1 at +z, so u = +z and t increases with z: the first segment is the lowest slice
    assert ta[0] == pytest.approx(-11.0, abs=1e-12)
    # along x through (iy, iz) = (2, 4)
    y, z = -4.5 + 2.5 * 2.5, -11.0 + 4.5 * 4.0
    vox, ta, tb = oracle.trace(g, [-100.0, y, z], [100.0, y, z])
    assert sorted(vox) == [ix + 5 * (2 + 4 * 4) for ix in range(5)]
    assert np.allclose(tb - ta, 3.0, atol=1e-12)


def test_trace_in_plane_rays_take_higher_index():
    g = ODD_GRID
    # a ray lying exactly in the plane x = ox + 2 vx belongs to column ix = 2
    xp = -7.0 + 2 * 3.0
    vox, ta, tb = oracle.trace(g, [xp, -30.0, -3.0], [xp, 30.0, 5.0])
    assert len(vox) > 0 and all(j % 5 == 2 for j in vox)
    ref = brute_segments(g, [xp, -30.0, -3.0], [xp, 30.0, 5.0])
    assert set(int(j) for j in vox) == set(ref)
    # on an edge (x and y planes): column (2, 3)
    yp = -4.5 + 3 * 2.5
    vox, ta, tb = oracle.trace(g, [xp, yp, -50.0], [xp, yp, 50.0])
    assert list(sorted(vox)) == [2 + 5 * (3 + 4 * k) for k in range(6)]
    # on the upper face of the grid (x = ox + nx vx): outside the half-open box
    vox, _, _ = oracle.trace(g, [-7.0 + 15.0, -30.0, 0.0], [-7.0 + 15.0, 30.0, 1.0])
    assert len(vox) == 0
    # on the lower face: inside, column 0
    vox, _, _ = oracle.trace(g, [-7.0, -30.0, 0.0], [-7.0, 30.0, 1.0])
    assert len(vox) > 0 and all(j % 5 == 0 for j in vox)


def test_chord_sums_equal_box_chord():
    rng = np.random.default_rng(7)
    g = Grid.centred(32, 32, 48, 4.0)
    p1, p2 = random_lines(rng, 300, 150.0)
    hits = 0
    for a, b in zip(p1, p2):
        vox, ta, tb = oracle.trace(g, a, b)
        L, _, _ = box_chord(g, a, b)
        assert np.sum(tb - ta) == pytest.approx(L, abs=1e-10)
        hits += L > 0
    assert hits > 100
    # space diagonal of a cube of side 12: 12 sqrt(3)
    cube = Grid.centred(3, 3, 3, 4.0)
    vox, ta, tb = oracle.trace(cube, [20.0, 20.0, 20.0], [-20.0, -20.0, -20.0])
    assert np.sum(tb - ta) == pytest.approx(12.0 * math.sqrt(3.0), abs=1e-12)
    assert sorted(vox) == [0, 13, 26]


def test_degenerate_lines():
    g = ODD_GRID
    assert len(oracle.trace(g, [1.0, 1.0, 1.0], [1.0, 1.0, 1.0])[0]) == 0     # P1 == P2
    assert len(oracle.trace(g, [100.0, 100.0, 0.0], [100.0, -100.0, 0.0])[0]) == 0  # misses
    assert len(oracle.trace(g, [0.0, 0.0, -100.0], [0.0, 0.0, 100.0], 5.0, 5.0)[0]) == 0  # empty window


# ------------------------------------------------------------ TOF rows

def test_row_has_unit_mass_inside_grid():
    sigma, K = oracle.tof_sigma_mm(300.0), 3.0
    g = Grid.centred(64, 64, 64, 4.0)  # 256 mm cube, window 115 mm
    rng = np.random.default_rng(3)
    for _ in range(50):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        c = rng.uniform(-30, 30, 3)
        d = rng.uniform(-10, 10)
        p1, p2 = c + 400 * u, c - 400 * u         # M = c, TOF point c + d u
        vox, a = oracle.system_row(g, events_from(p1, p2, d), 0, sigma, K)
        assert a.sum() == pytest.approx(1.0, abs=1e-13)
        assert np.all(a >= 0)


def test_row_mass_of_clipped_window_is_closed_form():
    sigma, K = oracle.tof_sigma_mm(300.0), 3.0
    g = ODD_GRID
    rng = np.random.default_rng(4)
    for _ in range(100):
        p1, p2 = random_lines(rng, 1, 40.0)
        d = rng.uniform(-60, 60)
        L, a, b = box_chord(g, p1[0], p2[0])
        vox, w = oracle.system_row(g, events_from(p1, p2, d), 0, sigma, K)
        if L == 0:
            assert len(w) == 0
            continue
        lo, hi = max(a, d - K * sigma), min(b, d + K * sigma)
        ref = trunc_gauss_mass((lo - d) / sigma, (hi - d) / sigma, K) if hi > lo else 0.0
        assert w.sum() == pytest.approx(ref, rel=1e-12, abs=1e-15)


def dense_system(grid, ev, sigma, K):
    """Brute-force A (events x voxels): exact TOF mass of every voxel piece."""
    n = ev[0].shape[0]
    A = np.zeros((n, grid.n_vox))
    for i in range(n):
        p1 = [ev[0][i], ev[1][i], ev[2][i]]
        p2 = [ev[3][i], ev[4][i], ev[5][i]]
        d = ev[6][i]
        segs = brute_segments(grid, p1, p2, d - K * sigma, d + K * sigma)
        for j, (ta, tb) in segs.items():
            A[i, j] = trunc_gauss_mass((ta - d) / sigma, (tb - d) / sigma, K)
    return A


def dense_chords(grid, lors):
    s = np.zeros(grid.n_vox)
    for l in range(lors.shape[1]):
        for j, (ta, tb) in brute_segments(grid, lors[0:3, l], lors[3:6, l]).items():
            s[j] += tb - ta
    return s


def small_problem(seed, n_ev=400, n_lor=600):
    rng = np.random.default_rng(seed)
    g = Grid.centred(8, 8, 8, 4.0)
    sigma = 8.0                       # a kernel narrower than the grid, so TOF matters
    c = rng.normal(0, 5, (n_ev, 3)) + np.array([3.0, -2.0, 1.0])
    u = rng.normal(size=(n_ev, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    l1, l2 = rng.uniform(40, 80, n_ev), rng.uniform(40, 80, n_ev)
    p1 = c + u * l1[:, None]
    p2 = c - u * l2[:, None]
    d = 0.5 * (l2 - l1) + rng.normal(0, sigma, n_ev)
    ev = events_from(p1, p2, d)
    lu = rng.normal(size=(n_lor, 3))
    lu /= np.linalg.norm(lu, axis=1, keepdims=True)
    lc = rng.uniform(-16, 16, (n_lor, 3))
    lors = np.concatenate([(lc + 60 * lu).T, (lc - 60 * lu).T])
    return g, sigma, ev, lors


def test_projectors_match_dense_bruteforce_matrix():
    g, sigma, ev, lors = small_problem(11, n_ev=150)
    A = dense_system(g, ev, sigma, 3.0)
    rng = np.random.default_rng(12)
    lam = rng.uniform(0.1, 2.0, g.n_vox)
    r = rng.uniform(0.0, 3.0, ev[0].size)
    assert np.allclose(oracle.forward(g, ev, lam, sigma, 3.0), A @ lam, rtol=1e-12, atol=1e-15)
    assert np.allclose(oracle.backproject(g, ev, r, sigma, 3.0), A.T @ r, rtol=1e-12, atol=1e-14)
    s = oracle.sensitivity(g, lors)
    assert np.allclose(s, dense_chords(g, lors), rtol=1e-12, atol=1e-11)


def test_forward_backward_adjoint_and_thread_invariance():
    ev = synth.events("tiny", 3000, 5).astype(np.float64)
    g = Grid.centred(32, 32, 48, 4.0)
    sigma = oracle.tof_sigma_mm(300.0)
    rng = np.random.default_rng(5)
    lam = rng.uniform(0, 1, g.n_vox)
    r = rng.uniform(0, 1, ev.shape[1])
    p = oracle.forward(g, ev, lam, sigma)
    C = oracle.backproject(g, ev, r, sigma)
    assert np.dot(p, r) == pytest.approx(np.dot(C, lam), rel=1e-12)
    C1 = oracle.backproject(g, ev, r, sigma, threads=1)
    assert np.allclose(C, C1, rtol=1e-13, atol=1e-16)


# ------------------------------------------------------------ MLEM

def textbook_mlem(A, s, n_iter, w=None):
    """Dense MLEM: lambda <- lambda / s * A^T (w / A lambda) on {s > 0}."""
    n, J = A.shape
    w = np.ones(n) if w is None else w
    mask = s > 0
    lam = np.where(mask, w.sum() / s[mask].sum(), 0.0)
    for _ in range(n_iter):
        p = A @ lam
        ratio = np.where(p > 0, w / np.where(p > 0, p, 1.0), 0.0)
        lam = np.where(mask, lam * (A.T @ ratio) / np.where(mask, s, 1.0), 0.0)
    return lam


def test_mlem_matches_dense_textbook_mlem_8cubed():
    g, sigma, ev, lors = small_problem(21, n_ev=2000, n_lor=1500)
    A = dense_system(g, ev, sigma, 3.0)
    s = dense_chords(g, lors)
    lam_ref = textbook_mlem(A, s, 6)
    lam, hist = oracle.mlem(g, ev, oracle.sensitivity(g, lors), 6, sigma, 3.0)
    assert np.max(np.abs(lam - lam_ref)) <= 1e-12 * np.max(np.abs(lam_ref))
    # weighted events (the region division's w = 1/2) follow the same algebra
    w = np.where(np.arange(ev[0].size) % 3 == 0, 0.5, 1.0)
    lam_w, _ = oracle.mlem(g, ev, oracle.sensitivity(g, lors), 3, sigma, 3.0, weights=w)
    assert np.allclose(lam_w, textbook_mlem(A, s, 3, w), rtol=1e-11, atol=1e-14 * lam_ref.max())


def test_one_voxel_closed_form():
    # a single voxel: p_i = a_i lambda, C = sum_i a_i / (a_i lambda), so lambda1 = N / s
    g = Grid(1, 1, 1, 10.0, 10.0, 10.0, -5.0, -5.0, -5.0)
    rng = np.random.default_rng(8)
    n = 37
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    ev = events_from(50 * u, -50 * u, rng.uniform(-3, 3, n))
    s = np.array([12.5])
    lam, hist = oracle.mlem(g, ev, s, 1, 4.0, 3.0)
    assert lam[0] == pytest.approx(n / 12.5, rel=1e-14)
    assert hist[0][0] == n


def test_mlem_invariants_on_tiny_subset():
    ev = synth.events("tiny", 6000, 1706).astype(np.float64)
    lors = synth.sensitivity_lors("tiny", 20000, 1706)
    g = Grid.centred(32, 32, 48, 4.0)
    sigma = oracle.tof_sigma_mm(300.0)
    s = oracle.sensitivity(g, lors)
    lam, hist = oracle.mlem(g, ev, s, 5, sigma)
    assert np.all(lam >= 0)
    for n_eff, ssum, _ in hist:
        assert ssum == pytest.approx(n_eff, rel=1e-12)          # count conservation
    ll = [h[2] for h in hist]
    assert all(b >= a - 1e-9 * abs(a) for a, b in zip(ll, ll[1:]))   # monotone likelihood
    assert np.all(lam[s == 0] == 0)


def test_mlem_resumes_from_a_saved_image():
    # checkpoint / resume: an MLEM iteration depends only on the image it starts
    # from (Sec. 2.4), so n iterations equal k iterations, saved, then n - k more
    # started from the saved image; the oracle reproduces them bit for bit
    ev = synth.events("tiny", 4000, 1707).astype(np.float64)
    lors = synth.sensitivity_lors("tiny", 20000, 1707)
    g = Grid.centred(32, 32, 48, 4.0)
    sigma = oracle.tof_sigma_mm(300.0)
    s = oracle.sensitivity(g, lors)
    lam3, hist3 = oracle.mlem(g, ev, s, 3, sigma)
    lam1, hist1 = oracle.mlem(g, ev, s, 1, sigma)
    lam_r, hist_r = oracle.mlem(g, ev, s, 2, sigma, init=lam1)
    assert np.array_equal(lam_r, lam3)
    assert hist1 + hist_r == hist3
    assert not np.array_equal(lam1, lam3)


# ------------------------------------------------------------ region division

def test_region_codes_golden_boundaries():
    gd = golden("region_boundary_events.json")
    evs = gd["events"]
    ev = [np.array([e["p1"][k] for e in evs], float) for k in range(3)] + \
         [np.array([e["p2"][k] for e in evs], float) for k in range(3)] + [np.array([e["d"] for e in evs], float)]
    codes, z = oracle.region_codes(ev, gd["z_bounds"], gd["shell_mm"], return_z=True)
    assert list(z) == [e["z_tof"] for e in evs]
    assert list(codes) == [e["code"] for e in evs]


FULLBODY_REGIONS = synth.FULLBODY_REGIONS   # nine body regions; some events fall outside them


def test_region_codes_one_or_two_consecutive_regions():
    ev = synth.events("fullbody", 20000, 3).astype(np.float64)
    g = Grid.centred(150, 150, 600, 4.0)
    zb = oracle.region_bounds(g, FULLBODY_REGIONS)
    codes, z = oracle.region_codes(ev, zb, 6.0, return_z=True)
    offs, idx = oracle.region_members(codes, 9)
    # every event inside the widened range feeds one or two consecutive regions
    inside = (z >= zb[0] - 6.0) & (z < zb[-1] + 6.0)
    assert np.array_equal(codes != 0xFF, inside)
    counts = np.zeros(ev.shape[1], int)
    for r in range(9):
        members = idx[offs[r]:offs[r + 1]]
        assert np.all(np.diff(members) > 0)            # stable, ascending
        mem = np.zeros(ev.shape[1], bool)
        mem[members] = True
        ref = (z >= zb[r] - 6.0) & (z < zb[r + 1] + 6.0)
        assert np.array_equal(mem, ref)
        counts += mem
    assert counts.max() <= 2 and np.all(counts[inside] >= 1)
    assert 0 < np.count_nonzero(~inside) < 0.01 * ev.shape[1]   # below the feet or above the head
    # duplicates only within a shell of a core boundary
    dup = (codes != 0xFF) & ((codes & 0x80) != 0)   # 0xFF (no region) also has the top bit
    near = np.min(np.abs(z[:, None] - zb[None, 1:-1]), axis=1) <= 6.0
    assert np.all(near[dup])


def test_region_slabs_reproduce_paper_extended_sizes():
    gc = golden("paper_constants.json")
    gd = gc["regions"]
    g = Grid.centred(350, 350, 1000, 2.0)
    k = np.cumsum([0] + gd["core_slices"])
    assert k[-1] == gc["image_matrix"]["value"][2]
    regions = [(int(k[i]), int(k[i + 1])) for i in range(9)]
    slabs = oracle.region_slabs(g, regions, gd["margin_mm"])
    sizes = [hi - lo for lo, hi in slabs]
    assert sizes[1:8] == [gd["middle_extended_slices"]] * 7


def test_region_stitch_counts_each_event_once():
    ev = synth.events("tiny", 4000, 9).astype(np.float64)
    lors = synth.sensitivity_lors("tiny", 20000, 9)
    g = Grid.centred(32, 32, 48, 4.0)
    sigma = oracle.tof_sigma_mm(300.0)
    s = oracle.sensitivity(g, lors)
    regions = [(0, 16), (16, 32), (32, 48)]
    img, imgs, hists, codes, offs, idx = oracle.mlem_regions(g, ev, s, regions, 6.0, 3 * sigma + 6.0, 2, sigma)
    n_in = np.sum(codes != 0xFF)
    total = sum(h[-1][1] for h in hists)
    n_eff = sum(h[-1][0] for h in hists)
    assert total == pytest.approx(n_eff, rel=1e-12)
    assert n_eff <= n_in + 1e-9
    assert n_eff >= 0.99 * n_in
    # the stitched image holds the same total as the slabs
    s3 = s.reshape(g.shape_zyx)
    assert float(np.sum(s3.reshape(-1) * img)) == pytest.approx(total, rel=1e-12)
