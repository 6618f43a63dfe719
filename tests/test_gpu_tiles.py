"""Shared-memory tiled event pass vs the oracle and vs the global-memory pass.

The tiled pass computes the same pieces and masses (each event's window split
among eight lanes: a voxel cut by a lane boundary gets two partial masses
whose sum is its mass), so the plain MLEM tolerances apply: relative L2 1e-4,
per voxel 1e-3 above 1% of max (percentile gate for the sparse full-body
case, as in the region tests).
"""
import numpy as np
import pytest

import oracle
from gpu_common import SIGMA, grid_tuple, max_rel_above, rel_l2, tiny_inputs, workload_grid
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth
from test_gpu_regions import SPARSE_MAX, SPARSE_P999, per_voxel_gate, smooth_sensitivity

pytestmark = pytest.mark.gpu


def run_mlem(geom, g, ev, sens, n_iter, tiled, graphs=1, lanes=1):
    with B.Context(geom, grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(sens)
        if tiled:
            ctx.set_tiled_pass(tiled, lanes)
        else:
            ctx.set_event_order(0)                  # global-memory pass in load order
        ctx.set_graphs(graphs)
        lam = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((n_iter, 2))
        ctx.mlem(B.make_events(ev), n_iter, None, lam, cons)
        info = ctx.get_info()
    return lam, cons, info


@pytest.mark.parametrize("graphs,lanes", [(1, 1), (0, 1), (1, 8)])
def test_tiled_mlem_tiny_matches_oracle(graphs, lanes):
    # a 45 degree axial acceptance makes the tiles fit (the tiny scanner's LORs are
    # all flatter than that; the fallback path has its own test below)
    ev, lors = tiny_inputs()
    g = workload_grid("tiny")
    s_ref = oracle.sensitivity(g, lors)
    lam_ref, hist = oracle.mlem(g, ev.astype(np.float64), s_ref, 5, SIGMA)
    lam, cons, info = run_mlem((150.0, 200.0, 45.0), g, ev, s_ref, 5, True, graphs, lanes)
    assert info["tile_cells"] > 0 and info["tile_events"] + info["tile_fallback_events"] == ev.shape[1]
    assert rel_l2(lam, lam_ref) <= 1e-4
    assert max_rel_above(lam, lam_ref, 0.01) <= 1e-3
    for k in range(5):
        assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)
        assert cons[k, 1] == pytest.approx(cons[k, 0], rel=1e-5)


def test_tiled_mlem_fullbody_matches_oracle():
    g = workload_grid("fullbody")
    ev = synth.events("fullbody", 300_000, 91)
    s = smooth_sensitivity(g)
    lam_ref, hist = oracle.mlem(g, ev.astype(np.float64), s, 2, SIGMA)
    lam, cons, info = run_mlem((400.0, 2400.0, 45.0), g, ev, s, 2, 2)       # tile cells of >= 2 events
    assert info["tile_cells"] > 1000
    assert info["tile_fallback_events"] < 0.5 * ev.shape[1]
    assert rel_l2(lam, lam_ref) <= 1e-4
    p999, pmax = per_voxel_gate(lam, lam_ref)
    assert p999 <= SPARSE_P999 and pmax <= SPARSE_MAX
    for k in range(2):
        assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)


def test_tiled_and_global_passes_agree_fullbody():
    g = workload_grid("fullbody")
    ev = synth.events("fullbody", 4_000_000, 92)
    s = smooth_sensitivity(g)
    a, ca, ia = run_mlem((400.0, 2400.0, 45.0), g, ev, s, 3, 16)
    b, cb, ib = run_mlem((400.0, 2400.0, 45.0), g, ev, s, 3, False)
    assert ia["tile_cells"] > 0 and ib["tile_cells"] == 0
    assert rel_l2(a, b) < 1e-4
    np.testing.assert_allclose(ca[:, 0], cb[:, 0], atol=2.0)


def test_narrow_acceptance_sends_events_to_fallback():
    # a 10 degree acceptance gives a thin tile: the steeper tiny events leave it and take
    # the global-memory pass; the result is unchanged
    ev, lors = tiny_inputs()
    ev = np.ascontiguousarray(ev[:, :50_000])
    g = workload_grid("tiny")
    s_ref = oracle.sensitivity(g, lors)
    lam_ref, hist = oracle.mlem(g, ev.astype(np.float64), s_ref, 3, SIGMA)
    lam, cons, info = run_mlem((150.0, 200.0, 10.0), g, ev, s_ref, 3, 2)
    assert info["tile_fallback_events"] > 0.1 * ev.shape[1]
    assert rel_l2(lam, lam_ref) <= 1e-4
    assert max_rel_above(lam, lam_ref, 0.01) <= 1e-3


def test_cell_ordered_pass_matches_oracle():
    ev, lors = tiny_inputs()
    g = workload_grid("tiny")
    s_ref = oracle.sensitivity(g, lors)
    lam_ref, hist = oracle.mlem(g, ev.astype(np.float64), s_ref, 5, SIGMA)
    with B.Context((150.0, 200.0, 90.0), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        ctx.set_event_order(3)
        lam = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((5, 2))
        ctx.mlem(B.make_events(ev), 5, None, lam, cons)
        info = ctx.get_info()
    assert info["tile_events"] == ev.shape[1] and info["tile_fallback_events"] == 0
    assert rel_l2(lam, lam_ref) <= 1e-4
    assert max_rel_above(lam, lam_ref, 0.01) <= 1e-3
    for k in range(5):
        assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)


def test_order_and_tile_argument_checks():
    g = workload_grid("tiny")
    with B.Context((150.0, 200.0, 45.0), grid_tuple(g), 300.0) as ctx:
        for bad in (-2, 65):
            with pytest.raises(B.ReconError):
                ctx.set_event_order(bad)
        with pytest.raises(B.ReconError):
            ctx.set_tiled_pass(-1)
        with pytest.raises(B.ReconError):
            ctx.set_tiled_pass(1, 4)
        ctx.set_event_order(-1)
        ctx.set_event_order(0)


def test_direction_binned_order_matches_oracle():
    ev, lors = tiny_inputs()
    g = workload_grid("tiny")
    s_ref = oracle.sensitivity(g, lors)
    lam_ref, hist = oracle.mlem(g, ev.astype(np.float64), s_ref, 3, SIGMA)
    with B.Context((150.0, 200.0, 90.0), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        ctx.set_event_order(2, 8, 4)
        lam = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((3, 2))
        ctx.mlem(B.make_events(ev), 3, None, lam, cons)
        with pytest.raises(B.ReconError):
            ctx.set_event_order(2, 0, 4)
    assert rel_l2(lam, lam_ref) <= 1e-4
    assert max_rel_above(lam, lam_ref, 0.01) <= 1e-3
    for k in range(3):
        assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)
