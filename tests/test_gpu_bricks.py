"""The exact projector's pass over 2x2x2-voxel brick copies of lambda and C
(recon_launch.reduction = 1): the same Siddon pieces and TOF masses as the linear
pass, gathered and reduced at brick-layout indices, so the FP32 sums run in another
order.  Held to the plain gates against the FP64 oracle (Sec. 2.4 MLEM) and to
1e-5 relative L2 against the linear pass (FP32 summation order only)."""
import numpy as np
import pytest

import oracle
from gpu_common import (SIGMA, geometry, grid_tuple, max_rel_above, oracle_sensitivity, rel_l2, tiny_inputs,
                        workload_grid)
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

pytestmark = pytest.mark.gpu

_cache = {}


def oracle_tiny_mlem():
    if "mlem" not in _cache:
        ev, lors = tiny_inputs()
        g = workload_grid("tiny")
        s_ref = oracle_sensitivity("tiny", lors.shape[1], 1706)
        _cache["mlem"] = (s_ref,) + oracle.mlem(g, ev.astype(np.float64), s_ref, 5, SIGMA)
    return _cache["mlem"]


@pytest.mark.parametrize("graphs,resident", [(1, True), (0, True), (1, False)])
def test_brick_reductions_match_oracle(graphs, resident):
    ev, _ = tiny_inputs()
    g = workload_grid("tiny")
    s_ref, lam_ref, hist = oracle_tiny_mlem()
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        ctx.set_graphs(graphs)
        ctx.set_launch(128, 0, 0, 0, 2, 0)
        lin = np.zeros(g.n_vox, np.float32)
        ctx.mlem(B.make_events(ev), 5, None, lin, None)
        ctx.set_launch(128, 0, 0, 0, 2, 1)
        if resident:
            ctx.load_events(B.make_events(ev))
        img = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((5, 2))
        ctx.mlem(None if resident else B.make_events(ev), 5, None, img, cons)
        assert ctx.get_launch()[5] == 1
    assert rel_l2(img, lam_ref) <= 1e-4
    assert max_rel_above(img, lam_ref, 0.01) <= 1e-3
    assert rel_l2(img, lin) <= 1e-5
    for k in range(5):
        assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)
        assert cons[k, 1] == pytest.approx(cons[k, 0], rel=1e-5)
    assert np.all(img >= 0)


def test_brick_reductions_odd_grid_and_osem():
    # odd extents on every axis (the bricks pad each axis) and OSEM subsets (the
    # brick copies are refreshed before every sub-iteration's pass)
    ev = synth.events("tiny", 60_000, 33)
    lors = synth.sensitivity_lors("tiny", 300_000, 33)
    g = oracle.Grid.centred(33, 31, 47, 4.0)
    s_ref = oracle.sensitivity(g, lors)
    lam_ref, hist = oracle.mlem(g, ev.astype(np.float64), s_ref, 3, SIGMA)
    osem_ref, osem_hist = oracle.osem(g, ev.astype(np.float64), s_ref, 2, 3, SIGMA)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        ctx.set_launch(192, 0, 0, 0, 0, 1)
        ctx.load_events(B.make_events(ev))
        img = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((3, 2))
        ctx.mlem(None, 3, None, img, cons)
        ctx.set_subsets(3)
        osem = np.zeros(g.n_vox, np.float32)
        ocons = np.zeros((6, 2))
        ctx.mlem(None, 2, None, osem, ocons)
    assert rel_l2(img, lam_ref) <= 1e-4
    assert max_rel_above(img, lam_ref, 0.01) <= 1e-3
    for k in range(3):
        assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)
    assert rel_l2(osem, osem_ref) <= 1e-4
    assert max_rel_above(osem, osem_ref, 0.01) <= 1e-3
    for k in range(6):
        assert ocons[k, 1] == pytest.approx(3 * ocons[k, 0], rel=1e-5)


def test_brick_reduction_launch_checks():
    g = workload_grid("tiny")
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        for bad in [(128, 4, 64, 0, 2, 1), (128, 0, 0, 32, 2, 1), (128, 0, 0, 0, 2, 2)]:
            with pytest.raises(B.ReconError):
                ctx.set_launch(*bad)
