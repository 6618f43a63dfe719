"""GPU path vs the FP64 oracle on the tiny workload (32x32x48 voxels of 4 mm,
200k events, 2M sensitivity LORs, 5 iterations), element by element.

Tolerances: relative L2 <= 1e-4 and per-voxel relative error <= 1e-3 on
voxels above 1% of the maximum for images after the MLEM iterations.  The
single passes are held tighter.  The floor of the FP32 event pass is its walk:
a plane crossing tau = (X - c) / u carries about ulp(|X - c|) / |u| of
rounding, so a line nearly parallel to a voxel plane moves up to ~1e-2 mm of
chord between two voxels, which stays below 1e-4 of p_i (per event) while the
relative L2 over all events stays near 1e-6.  The sensitivity walk runs in
FP64: the same crossing error is ulp_64(|X - c|) / |u_k|, ~1e-5 mm only for a
line with |u_k| ~ 1e-8, so s is held to 1e-9 relative L2 and 1e-6 per voxel.
"""
import numpy as np
import pytest

import oracle
from gpu_common import (SIGMA, max_rel_above, new_context, oracle_sensitivity, rel_l2, tiny_inputs,
                        workload_grid)
from paper_1706_07075_b300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    ev, lors = tiny_inputs()
    g = workload_grid("tiny")
    s_ref = oracle_sensitivity("tiny", lors.shape[1], 1706)
    ctx = new_context("tiny")
    yield g, ev, lors, s_ref, ctx
    ctx.close()


def test_sensitivity_matches_oracle(tiny):
    g, ev, lors, s_ref, ctx = tiny
    s = np.zeros(g.n_vox)
    ctx.sensitivity(lors, s)
    assert np.array_equal(s > 0, s_ref > 0) or np.sum((s > 0) != (s_ref > 0)) <= 2
    assert rel_l2(s, s_ref) < 1e-9
    assert max_rel_above(s, s_ref, 0.01) < 1e-6


def test_forward_matches_oracle(tiny):
    g, ev, lors, s_ref, ctx = tiny
    rng = np.random.default_rng(2)
    lam = rng.uniform(0.5, 1.5, g.n_vox).astype(np.float32)
    p = np.zeros(ev.shape[1], np.float32)
    ctx.forward(B.make_events(ev), lam, p)
    p_ref = oracle.forward(g, ev.astype(np.float64), lam.astype(np.float64), SIGMA)
    sel = p_ref > 1e-3 * p_ref.max()
    assert np.all((p > 0) == (p_ref > 0)) or np.sum((p > 0) != (p_ref > 0)) < 1e-5 * p.size
    assert np.max(np.abs(p[sel] - p_ref[sel]) / p_ref[sel]) < 1e-4
    assert rel_l2(p, p_ref) < 2e-6


def test_backproject_matches_oracle(tiny):
    g, ev, lors, s_ref, ctx = tiny
    rng = np.random.default_rng(3)
    r = rng.uniform(0.0, 2.0, ev.shape[1]).astype(np.float32)
    C = np.zeros(g.n_vox, np.float32)
    ctx.backproject(B.make_events(ev), r, C)
    C_ref = oracle.backproject(g, ev.astype(np.float64), r.astype(np.float64), SIGMA)
    assert rel_l2(C, C_ref) < 1e-5
    assert max_rel_above(C, C_ref, 0.01) < 1e-4


@pytest.mark.parametrize("graphs", [1, 0])
def test_mlem_matches_oracle_5_iterations(tiny, graphs):
    g, ev, lors, s_ref, ctx = tiny
    ctx.sensitivity(lors)
    ctx.set_graphs(graphs)
    lam = np.zeros(g.n_vox, np.float32)
    cons = np.zeros((5, 2))
    ctx.mlem(B.make_events(ev), 5, None, lam, cons)
    lam_ref, hist = _oracle_mlem_tiny()
    assert rel_l2(lam, lam_ref) <= 1e-4
    assert max_rel_above(lam, lam_ref, 0.01) <= 1e-3
    for k in range(5):
        n_eff, ssum = cons[k]
        assert n_eff == pytest.approx(hist[k][0], abs=0.5)          # same events with p > 0
        assert ssum == pytest.approx(n_eff, rel=1e-5)               # count conservation (FP32 image)
    assert np.all(lam >= 0)


def test_mlem_resumes_from_a_saved_image(tiny):
    # checkpoint / resume through the C-ABI: 3 iterations equal 1 iteration, the
    # image read back, then 2 iterations started from it (recon_mlem's init).  The
    # image stays FP32 between iterations on both routes, so only the order of the
    # FP32 reductions differs.
    g, ev, lors, s_ref, ctx = tiny
    ctx.sensitivity(lors)
    lam3 = np.zeros(g.n_vox, np.float32)
    cons3 = np.zeros((3, 2))
    ctx.mlem(B.make_events(ev), 3, None, lam3, cons3)
    lam1 = np.zeros(g.n_vox, np.float32)
    cons1 = np.zeros((1, 2))
    ctx.mlem(B.make_events(ev), 1, None, lam1, cons1)
    lam_r = np.zeros(g.n_vox, np.float32)
    cons_r = np.zeros((2, 2))
    ctx.mlem(B.make_events(ev), 2, lam1, lam_r, cons_r)
    assert rel_l2(lam_r, lam3) <= 1e-5
    assert max_rel_above(lam_r, lam3, 0.01) <= 1e-4
    assert cons1[0, 0] == cons3[0, 0]
    assert np.all(np.abs(cons_r[:, 0] - cons3[1:, 0]) <= 0.5)      # same events with p > 0
    np.testing.assert_allclose(cons_r[:, 1], cons3[1:, 1], rtol=1e-6)
    assert rel_l2(lam1, lam3) > 1e-3                                 # the check is not vacuous


_cache = {}


def _oracle_mlem_tiny():
    if "mlem" not in _cache:
        ev, lors = tiny_inputs()
        g = workload_grid("tiny")
        s_ref = oracle_sensitivity("tiny", lors.shape[1], 1706)
        _cache["mlem"] = oracle.mlem(g, ev.astype(np.float64), s_ref, 5, SIGMA)
    return _cache["mlem"]


def test_streamed_upload_matches_resident_events():
    # host events: the upload is streamed in 8 M-event chunks through two staging
    # halves and the first pass runs per chunk; three chunks exercise the reuse of
    # a half.  The resident path (events loaded first, then events = NULL) must
    # give the same iterations up to FP32 reduction order: a voxel here sums
    # ~12 k reductions per iteration in an order that changes from run to run
    # (~1e-5 relative after three iterations), the plain MLEM tolerance holds.
    from gpu_common import geometry, grid_tuple
    from paper_1706_07075_b300 import synth
    g = workload_grid("tiny")
    ev = synth.events("tiny", 17_000_000, 77)
    lors = synth.sensitivity_lors("tiny", 400_000, 77)
    out = []
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.sensitivity(lors)
        for streamed in (True, False):
            lam = np.zeros(g.n_vox, np.float32)
            cons = np.zeros((3, 2))
            if streamed:
                ctx.mlem(B.make_events(ev), 3, None, lam, cons)
            else:
                ctx.load_events(B.make_events(ev))
                ctx.mlem(None, 3, None, lam, cons)
            out.append((lam, cons))
    (a, ca), (b, cb) = out
    assert rel_l2(a, b) < 1e-4
    assert max_rel_above(a, b, 0.01) < 1e-3
    np.testing.assert_allclose(ca[:, 0], cb[:, 0], atol=2.0)              # same events with p > 0
    np.testing.assert_allclose(ca[:, 1], ca[:, 0], rtol=1e-5)


@pytest.mark.parametrize("tail_eval", [0, 1, 2, 3])
def test_piece_mass_forms_match_oracle(tiny, tail_eval):
    # the four evaluations of a piece's Gaussian mass (fitted tails, erfcf tails,
    # midpoint Taylor series through h^6 and through h^4) against the oracle's libm
    # erfc, forward and 3 iterations
    g, ev, lors, s_ref, ctx = tiny
    ctx.set_launch(128, 0, 0, 0, tail_eval)
    rng = np.random.default_rng(30 + tail_eval)
    lam = rng.uniform(0.5, 1.5, g.n_vox).astype(np.float32)
    p = np.zeros(ev.shape[1], np.float32)
    ctx.forward(B.make_events(ev), lam, p)
    p_ref = oracle.forward(g, ev.astype(np.float64), lam.astype(np.float64), SIGMA)
    sel = p_ref > 1e-3 * p_ref.max()
    assert np.max(np.abs(p[sel] - p_ref[sel]) / p_ref[sel]) < 1e-4
    assert rel_l2(p, p_ref) < 2e-6
    ctx.set_sensitivity(s_ref)
    img = np.zeros(g.n_vox, np.float32)
    ctx.mlem(None, 3, None, img)
    ctx.set_launch(None)
    lam_ref, _ = oracle.mlem(g, ev.astype(np.float64), s_ref, 3, SIGMA)
    assert rel_l2(img, lam_ref) <= 1e-4
    assert max_rel_above(img, lam_ref, 0.01) <= 1e-3


def test_starting_backprojection_matches_oracle(tiny):
    g, ev, lors, s_ref, ctx = tiny
    ctx.set_sensitivity(s_ref)
    ctx.set_start_image(1)
    lam0 = np.zeros(g.n_vox, np.float32)
    ctx.mlem(B.make_events(ev), 0, None, lam0)                 # no iteration: the start image itself
    lam3 = np.zeros(g.n_vox, np.float32)
    ctx.mlem(None, 3, None, lam3)
    ctx.set_start_image(0)
    ref0 = oracle.start_backprojection(g, ev.astype(np.float64), s_ref, SIGMA)
    assert rel_l2(lam0, ref0) < 1e-5
    assert max_rel_above(lam0, ref0, 0.01) < 1e-4
    ref3, _ = oracle.mlem(g, ev.astype(np.float64), s_ref, 3, SIGMA, init=ref0)
    assert rel_l2(lam3, ref3) <= 1e-4
    assert max_rel_above(lam3, ref3, 0.01) <= 1e-3
    with pytest.raises(B.ReconError):
        ctx.set_start_image(2)
