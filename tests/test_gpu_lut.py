"""GPU sampled TOF kernel (Sec. 2.3, the paper's own projector) vs the oracle.

The oracle decides each sample's voxel in FP64 from the exact sample position
c + t_k u; the kernel decides it in FP32.  The two can differ only for a sample
within the kernel's FP32 error of a voxel plane (at most ~2e-4 voxel on these
grids), so every test runs both sides on the events none of whose samples lies
within oracle.LUT_EPS_VOXELS = 1e-3 voxel of a plane (oracle.lut_ambiguous;
about 15% of the events have such a sample at 32 samples per event).  On those
events the set of voxels an event touches is the same on both sides, which the
tests check through the p_i = 0 pattern and through per-event tolerances far
below the change one moved sample causes (the smallest weight of 32 samples is
~1e-3, times a random image contrast of ~0.3).  The remaining difference is FP32
accumulation: p_i sums at most 64 products (relative ~64 ulp worst case, held to
2e-5), C_j sums FP32 reductions (held to 1e-5 relative L2).
"""
import numpy as np
import pytest

import oracle
from gpu_common import (SIGMA, geometry, grid_tuple, lut_unambiguous, max_rel_above, rel_l2, tiny_inputs,
                        workload_grid)
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    ev, lors = tiny_inputs()
    g = workload_grid("tiny")
    ctx = B.Context(geometry("tiny"), grid_tuple(g), 300.0)
    yield g, ev, lors, ctx
    ctx.close()


@pytest.mark.parametrize("n", [1, 15, 32, 64])
def test_sample_table_matches_oracle(tiny, n):
    g, ev, lors, ctx = tiny
    ctx.set_projector(B.PROJ_SAMPLED, n)
    t, w = ctx.get_tof_samples()
    t_ref, w_ref = oracle.lut_samples(n, SIGMA)
    assert np.array_equal(t, t_ref.astype(np.float32))
    np.testing.assert_allclose(w, w_ref, rtol=1e-7)
    ctx.set_projector(B.PROJ_EXACT)
    assert ctx.get_tof_samples()[0].size == 0


def test_projector_argument_checks(tiny):
    g, ev, lors, ctx = tiny
    for bad in [(B.PROJ_SAMPLED, 0), (B.PROJ_SAMPLED, 65), (7, 32)]:
        with pytest.raises(B.ReconError):
            ctx.set_projector(*bad)
    ctx.set_projector(B.PROJ_EXACT)


@pytest.mark.parametrize("n", [15, 32])
def test_forward_lut_matches_oracle(tiny, n):
    g, ev, lors, ctx = tiny
    ev = lut_unambiguous(g, ev, n)
    ctx.set_projector(B.PROJ_SAMPLED, n)
    rng = np.random.default_rng(20 + n)
    lam = rng.uniform(0.5, 1.5, g.n_vox).astype(np.float32)
    p = np.zeros(ev.shape[1], np.float32)
    ctx.forward(B.make_events(ev), lam, p)
    ctx.set_projector(B.PROJ_EXACT)
    p_ref = oracle.forward_lut(g, ev.astype(np.float64), lam.astype(np.float64), n, SIGMA)
    assert np.array_equal(p > 0, p_ref > 0)
    sel = p_ref > 0
    assert np.max(np.abs(p[sel] - p_ref[sel]) / p_ref[sel]) < 2e-5
    assert rel_l2(p, p_ref) < 2e-6


def test_backproject_lut_matches_oracle(tiny):
    g, ev, lors, ctx = tiny
    ev = lut_unambiguous(g, ev, 32)
    ctx.set_projector(B.PROJ_SAMPLED, 32)
    rng = np.random.default_rng(4)
    r = rng.uniform(0.0, 2.0, ev.shape[1]).astype(np.float32)
    C = np.zeros(g.n_vox, np.float32)
    ctx.backproject(B.make_events(ev), r, C)
    ctx.set_projector(B.PROJ_EXACT)
    C_ref = oracle.backproject_lut(g, ev.astype(np.float64), r.astype(np.float64), 32, SIGMA)
    assert np.array_equal(C > 0, C_ref > 0)
    assert rel_l2(C, C_ref) < 1e-5
    assert max_rel_above(C, C_ref, 0.01) < 1e-4


def test_single_sample_lands_on_tof_point(tiny):
    # n = 1: the whole event goes to the voxel of c = M + d u
    g, ev, lors, ctx = tiny
    ctx.set_projector(B.PROJ_SAMPLED, 1)
    sub = lut_unambiguous(g, ev[:, :5000], 1)
    n_ev = sub.shape[1]
    lam = np.arange(1, g.n_vox + 1, dtype=np.float32)   # exact integers: p names the voxel
    p = np.zeros(n_ev, np.float32)
    ctx.forward(B.make_events(sub), lam, p)
    ctx.set_projector(B.PROJ_EXACT)
    p_ref = oracle.forward_lut(g, sub.astype(np.float64), lam.astype(np.float64), 1, SIGMA)
    assert np.array_equal(p, p_ref.astype(np.float32))


@pytest.mark.parametrize("graphs", [1, 0])
def test_mlem_lut_matches_oracle_5_iterations(tiny, graphs):
    g, ev, lors, ctx = tiny
    ev = lut_unambiguous(g, ev, 32)
    s_ref = oracle.sensitivity(g, lors)
    ctx.set_sensitivity(s_ref)
    ctx.set_projector(B.PROJ_SAMPLED, 32)
    ctx.set_graphs(graphs)
    lam = np.zeros(g.n_vox, np.float32)
    cons = np.zeros((5, 2))
    ctx.mlem(B.make_events(ev), 5, None, lam, cons)
    ctx.set_projector(B.PROJ_EXACT)
    ctx.set_graphs(1)
    lam_ref, hist = _oracle_lut_mlem_tiny(g, ev, s_ref)
    assert rel_l2(lam, lam_ref) <= 1e-4
    assert max_rel_above(lam, lam_ref, 0.01) <= 1e-3
    for k in range(5):
        assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)
        assert cons[k, 1] == pytest.approx(cons[k, 0], rel=1e-5)     # sum s lambda = N_eff


_ref_cache = {}


def _oracle_lut_mlem_tiny(g, ev, s_ref):
    if "mlem5" not in _ref_cache:
        _ref_cache["mlem5"] = oracle.mlem(g, ev.astype(np.float64), s_ref, 5, SIGMA, lut_samples=32)
    return _ref_cache["mlem5"]


@pytest.mark.parametrize("graphs", [1, 0])
def test_mlem_lut_brick_layout_matches_oracle(tiny, graphs):
    # the sampled pass over 2x2x2-brick copies of lambda and C: the same visits and
    # weights at brick-layout indices.  Resident events (every pass in
    # bricks) and host events (the streamed first pass linear, the rest in bricks).
    g, ev, lors, ctx = tiny
    ev = lut_unambiguous(g, ev, 32)
    s_ref = oracle.sensitivity(g, lors)
    ctx.set_sensitivity(s_ref)
    ctx.set_projector(B.PROJ_SAMPLED, 32)
    ctx.set_graphs(graphs)
    ctx.load_events(B.make_events(ev))
    lin = np.zeros(g.n_vox, np.float32)
    ctx.mlem(None, 5, None, lin, np.zeros((5, 2)))
    ctx.set_brick_layout(1)
    try:
        out = []
        for events in (None, B.make_events(ev)):
            img = np.zeros(g.n_vox, np.float32)
            cons = np.zeros((5, 2))
            ctx.mlem(events, 5, None, img, cons)
            out.append((img, cons))
    finally:
        ctx.set_brick_layout(0)
        ctx.set_projector(B.PROJ_EXACT)
        ctx.set_graphs(1)
    lam_ref, hist = _oracle_lut_mlem_tiny(g, ev, s_ref)
    for img, cons in out:
        assert rel_l2(img, lam_ref) <= 1e-4
        assert max_rel_above(img, lam_ref, 0.01) <= 1e-3
        for k in range(5):
            assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)
            assert cons[k, 1] == pytest.approx(cons[k, 0], rel=1e-5)
        assert rel_l2(img, lin) <= 1e-5
        assert max_rel_above(img, lin, 0.01) <= 1e-4


def test_mlem_lut_brick_layout_odd_grid():
    # odd extents on every axis: the bricks pad each axis by one voxel
    lors = synth.sensitivity_lors("tiny", 300_000, 31)
    g = oracle.Grid.centred(33, 31, 47, 4.0)
    ev = lut_unambiguous(g, synth.events("tiny", 50_000, 31), 32)
    s_ref = oracle.sensitivity(g, lors)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        with pytest.raises(B.ReconError):
            ctx.set_brick_layout(2)
        ctx.set_sensitivity(s_ref)
        ctx.set_projector(B.PROJ_SAMPLED, 32)
        ctx.set_brick_layout(1)
        ctx.load_events(B.make_events(ev))
        img = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((3, 2))
        ctx.mlem(None, 3, None, img, cons)
    lam_ref, hist = oracle.mlem(g, ev.astype(np.float64), s_ref, 3, SIGMA, lut_samples=32)
    assert rel_l2(img, lam_ref) <= 1e-4
    assert max_rel_above(img, lam_ref, 0.01) <= 1e-3
    for k in range(3):
        assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)
        assert cons[k, 1] == pytest.approx(cons[k, 0], rel=1e-5)


def test_region_mlem_lut_matches_oracle():
    lors = synth.sensitivity_lors("tiny", 500_000, 23)
    g = workload_grid("tiny")
    ev = lut_unambiguous(g, synth.events("tiny", 120_000, 23), 32)
    regions = [(0, 16), (16, 32), (32, 48)]
    margin = 3.0 * SIGMA + 6.0
    s_ref = oracle.sensitivity(g, lors)
    img_ref, imgs_ref, hists, codes, offs, idx = oracle.mlem_regions(g, ev.astype(np.float64), s_ref, regions, 6.0,
                                                                     margin, 3, SIGMA, lut_samples=32)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        ctx.set_projector(B.PROJ_SAMPLED, 32)
        img = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((3, 3, 2))
        ctx.mlem_regions(B.make_events(ev), regions, margin, 6.0, 3, img, None, cons)
    assert rel_l2(img, img_ref) <= 1e-4
    assert max_rel_above(img, img_ref, 0.01) <= 1e-3
    for r in range(3):
        for k in range(3):
            assert cons[k, r, 0] == pytest.approx(hists[r][k][0], abs=0.5)


def test_forward_lut_fullbody_sampled_events():
    # full-body grid and event distribution, flat launch as the bench times it;
    # the oracle recomputes a strided sample of the events
    g = workload_grid("fullbody")
    ev = lut_unambiguous(g, synth.events("fullbody", 2_000_000, 5), 32)
    rng = np.random.default_rng(6)
    lam = rng.uniform(0.5, 1.5, g.n_vox).astype(np.float32)
    with B.Context(geometry("fullbody"), grid_tuple(g), 300.0) as ctx:
        ctx.set_projector(B.PROJ_SAMPLED, 32)
        p = np.zeros(ev.shape[1], np.float32)
        ctx.forward(B.make_events(ev), lam, p)
    pick = np.arange(0, ev.shape[1], 97)
    sub = ev[:, pick].astype(np.float64)
    p_ref = oracle.forward_lut(g, sub, lam.astype(np.float64), 32, SIGMA)
    assert np.array_equal(p[pick] > 0, p_ref > 0)
    sel = p_ref > 0
    assert np.max(np.abs(p[pick][sel] - p_ref[sel]) / p_ref[sel]) < 2e-5


def test_lut_packed_events_match_dequantized_oracle():
    ev = synth.events("tiny", 100_000, 41)
    rec = synth.pack_events(ev)
    q = rec[:, :6].astype(np.float64).T * synth.LATTICE_MM
    d = rec[:, 6].view(np.float16).astype(np.float64)
    evq = np.concatenate([q, d[None, :]])
    g = workload_grid("tiny")
    keep = oracle.lut_ambiguous(g, evq, 32, SIGMA) == 0            # decided on the dequantized events
    rec, evq, ev = np.ascontiguousarray(rec[keep]), np.ascontiguousarray(evq[:, keep]), ev[:, keep]
    rng = np.random.default_rng(42)
    lam = rng.uniform(0.5, 1.5, g.n_vox).astype(np.float32)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_projector(B.PROJ_SAMPLED, 32)
        p = np.zeros(ev.shape[1], np.float32)
        ctx.forward(B.make_events(rec, packed=True, lattice_mm=synth.LATTICE_MM), lam, p)
    p_ref = oracle.forward_lut(g, evq, lam.astype(np.float64), 32, SIGMA)
    assert np.array_equal(p > 0, p_ref > 0)
    sel = p_ref > 0
    assert np.max(np.abs(p[sel] - p_ref[sel]) / p_ref[sel]) < 2e-5


def test_lut_empty_event_list(tiny):
    g, ev, lors, ctx = tiny
    ctx.set_projector(B.PROJ_SAMPLED, 32)
    p = np.zeros(0, np.float32)
    ctx.forward(B.make_events(np.zeros((7, 0), np.float32)), np.ones(g.n_vox, np.float32), p)
    ctx.set_projector(B.PROJ_EXACT)


def test_region_mlem_lut_with_sieve_matches_oracle():
    # the paper's configuration: sampled kernel, nine-region style division (three
    # regions here), median sieve between iterations
    lors = synth.sensitivity_lors("tiny", 400_000, 24)
    g = workload_grid("tiny")
    ev = lut_unambiguous(g, synth.events("tiny", 100_000, 24), 32)
    regions = [(0, 16), (16, 32), (32, 48)]
    margin = 3.0 * SIGMA + 6.0
    s_ref = oracle.sensitivity(g, lors)
    img_ref, imgs_ref, hists, codes, offs, idx = oracle.mlem_regions(g, ev.astype(np.float64), s_ref, regions, 6.0,
                                                                     margin, 3, SIGMA, lut_samples=32, median=True)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        ctx.set_projector(B.PROJ_SAMPLED, 32)
        ctx.set_median_filter(1)
        img = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((3, 3, 2))
        ctx.mlem_regions(B.make_events(ev), regions, margin, 6.0, 3, img, None, cons)
    assert rel_l2(img, img_ref) <= 1e-4
    assert max_rel_above(img, img_ref, 0.01) <= 1e-3
    for r in range(3):
        for k in range(3):
            assert cons[k, r, 0] == pytest.approx(hists[r][k][0], abs=0.5)


def test_mlem_lut_autotuned_matches_oracle():
    # enough events for the autotuner (at least 2^20): it picks threads per block and
    # the image layout (linear, or 2x2x2-brick copies of lambda and C)
    # for the sampled projector; whatever it picks, the image holds the plain gates
    g = workload_grid("tiny")
    ev = lut_unambiguous(g, synth.events("tiny", 1_400_000, 29), 32)
    assert ev.shape[1] >= 1 << 20
    lors = synth.sensitivity_lors("tiny", 1_000_000, 29)
    s_ref = oracle.sensitivity(g, lors)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        ctx.set_projector(B.PROJ_SAMPLED, 32)
        ctx.load_events(B.make_events(ev))
        img = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((3, 2))
        ctx.mlem(None, 3, None, img, cons)
        launch = ctx.get_launch()
        assert ctx.get_stats()["autotune_runs"] >= 1
    assert launch[0] in (128, 192, 256) and launch[5] in (0, 1)
    lam_ref, hist = oracle.mlem(g, ev.astype(np.float64), s_ref, 3, SIGMA, lut_samples=32)
    print(f"\nsampled projector, tuned launch {launch}: rel L2 {rel_l2(img, lam_ref):.2e}")
    assert rel_l2(img, lam_ref) <= 1e-4
    assert max_rel_above(img, lam_ref, 0.01) <= 1e-3
    for k in range(3):
        assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)
        assert cons[k, 1] == pytest.approx(cons[k, 0], rel=1e-5)
