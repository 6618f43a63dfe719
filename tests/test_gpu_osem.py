"""GPU list-mode OSEM (named in Sec. 2.4's title) vs the oracle: B consecutive
event blocks, sub-iteration update lambda C^b / (s / B).  Same tolerances as
the MLEM parity tests; conservation per sub-iteration: sum s lambda = B N_eff."""
import numpy as np
import pytest

import oracle
from gpu_common import SIGMA, geometry, grid_tuple, max_rel_above, rel_l2, tiny_inputs, workload_grid
from paper_1706_07075_b300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_osem():
    ev, lors = tiny_inputs()
    g = workload_grid("tiny")
    s_ref = oracle.sensitivity(g, lors)
    return g, ev, s_ref


@pytest.mark.parametrize("subsets,graphs", [(4, 1), (4, 0), (7, 1)])
def test_osem_matches_oracle(tiny_osem, subsets, graphs):
    g, ev, s_ref = tiny_osem
    n_iter = 2
    lam_ref, hist = oracle.osem(g, ev.astype(np.float64), s_ref, n_iter, subsets, SIGMA)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        ctx.set_subsets(subsets)
        ctx.set_graphs(graphs)
        lam = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((n_iter * subsets, 2))
        ctx.mlem(B.make_events(ev), n_iter, None, lam, cons)
    assert rel_l2(lam, lam_ref) <= 1e-4
    assert max_rel_above(lam, lam_ref, 0.01) <= 1e-3
    for k, (n_eff, ssum) in enumerate(hist):
        assert cons[k, 0] == pytest.approx(n_eff, abs=0.5)
        assert cons[k, 1] == pytest.approx(subsets * cons[k, 0], rel=1e-5)


def test_one_subset_is_mlem(tiny_osem):
    g, ev, s_ref = tiny_osem
    out = []
    for subsets in (None, 1):
        with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
            ctx.set_sensitivity(s_ref)
            if subsets:
                ctx.set_subsets(subsets)
            lam = np.zeros(g.n_vox, np.float32)
            ctx.mlem(B.make_events(ev), 2, None, lam)
            out.append(lam)
    # FP32 reductions land in a different order on every run, so two runs agree
    # to rounding, not bit for bit
    assert rel_l2(out[1], out[0]) < 1e-6


def test_more_subsets_than_events(tiny_osem):
    g, ev, s_ref = tiny_osem
    sub = np.ascontiguousarray(ev[:, :10])
    lam_ref, hist = oracle.osem(g, sub.astype(np.float64), s_ref, 1, 16, SIGMA)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        ctx.set_subsets(16)
        lam = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((16, 2))
        ctx.mlem(B.make_events(sub), 1, None, lam, cons)
        with pytest.raises(B.ReconError):
            ctx.set_subsets(0)
    np.testing.assert_allclose(lam, lam_ref, rtol=1e-4, atol=1e-6 * max(lam_ref.max(), 1e-30))
    np.testing.assert_allclose(cons[:, 0], [h[0] for h in hist], atol=0.5)
