"""The small field of view of the served mix against the FP64 oracle: a 60 mm
radius scanner, 128^3 voxels of 0.5 mm (a 64 mm cube), 1 M events of the
small phantom (about 200 Siddon pieces each inside the +-3 sigma window, so
~100 pieces per voxel), sensitivity from 2 M LORs, 3 MLEM iterations (Sec. 2.4)
in the autotuned default launch and event order.  Plain gates: relative L2
<= 1e-4, per-voxel relative error <= 1e-3 on voxels above 1% of the maximum."""
import numpy as np
import pytest

import oracle
from gpu_common import SIGMA, geometry, max_rel_above, rel_l2, workload_grid
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

pytestmark = pytest.mark.gpu

N_EVENTS = 1_000_000
N_LORS = 2_000_000
N_ITER = 3


def test_smallfov_mlem_matches_oracle():
    g = workload_grid("smallfov")
    ev = synth.events("smallfov", N_EVENTS, 1710)
    lors = synth.sensitivity_lors("smallfov", N_LORS, 1710)
    with B.Context(geometry("smallfov"), synth.grid_of("smallfov"), 300.0) as ctx:
        s = np.zeros(g.n_vox)
        ctx.sensitivity(lors, s)
        ctx.load_events(B.make_events(ev))
        img = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((N_ITER, 2))
        ctx.mlem(None, N_ITER, None, img, cons)
        launch = ctx.get_launch()
    s_ref = oracle.sensitivity(g, lors)
    lam_ref, hist = oracle.mlem(g, ev.astype(np.float64), s_ref, N_ITER, SIGMA)
    l2, mx = rel_l2(img, lam_ref), max_rel_above(img, lam_ref, 0.01)
    print(f"\nsmall FOV, {N_EVENTS} events, {N_ITER} iterations, launch {launch}: rel L2 {l2:.2e}, "
          f"max rel above 1% {mx:.2e}; sensitivity rel L2 {rel_l2(s, s_ref):.2e}")
    assert rel_l2(s, s_ref) < 1e-9
    assert l2 <= 1e-4
    assert mx <= 1e-3
    for k in range(N_ITER):
        assert cons[k, 0] == pytest.approx(hist[k][0], abs=0.5)
        assert cons[k, 1] == pytest.approx(cons[k, 0], rel=1e-5)
    assert np.all(img >= 0)
