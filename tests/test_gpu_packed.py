"""Precision-packed events (int16 endpoints on a 0.05 mm lattice + FP16 TOF
offset, 16 bytes per event) and the BF16 forward gather, vs the FP64 oracle
run on the dequantized events.

FP32 gather: the image tolerances (relative L2 <= 1e-4, per-voxel <= 1e-3).
BF16 gather: BF16 keeps 8 significant bits, so each gathered lambda_j carries
up to 2^-9 relative rounding; p_i averages ~40 of them, and MLEM feeds the
error back each iteration.  The gate is relative L2 <= 5e-3 after 5
iterations; the measured error is printed for the record.
"""
import numpy as np
import pytest

import oracle
from gpu_common import SIGMA, geometry, grid_tuple, max_rel_above, rel_l2, workload_grid
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

pytestmark = pytest.mark.gpu


def dequantized(rec):
    q = rec[:, :6].astype(np.float64).T * synth.LATTICE_MM
    d = rec[:, 6].view(np.float16).astype(np.float64)
    return np.concatenate([q, d[None, :]])


@pytest.fixture(scope="module")
def packed_case():
    ev = synth.events("tiny", 150_000, 31)
    lors = synth.sensitivity_lors("tiny", 800_000, 31)
    rec = synth.pack_events(ev)
    g = workload_grid("tiny")
    s = oracle.sensitivity(g, lors)
    evq = dequantized(rec)
    lam_q, hist_q = oracle.mlem(g, evq, s, 5, SIGMA)
    lam_f, _ = oracle.mlem(g, ev.astype(np.float64), s, 5, SIGMA)
    return g, ev, lors, rec, lam_q, hist_q, lam_f


def run(g, lors, events, bf16, launch=None):
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.sensitivity(lors)
        ctx.set_gather_bf16(bf16)
        if launch:
            ctx.set_launch(*launch)
        img = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((5, 2))
        ctx.mlem(events, 5, None, img, cons)
    return img, cons


def test_packed_events_fp32_gather_match_dequantized_oracle(packed_case):
    g, ev, lors, rec, lam_q, hist_q, lam_f = packed_case
    img, cons = run(g, lors, B.make_events(rec, packed=True, lattice_mm=synth.LATTICE_MM), False)
    assert rel_l2(img, lam_q) <= 1e-4
    assert max_rel_above(img, lam_q, 0.01) <= 1e-3
    assert cons[-1, 1] == pytest.approx(cons[-1, 0], rel=1e-5)
    print(f"\npacked FP32-gather: rel L2 vs dequantized oracle {rel_l2(img, lam_q):.2e}, "
          f"vs unquantized FP64 oracle {rel_l2(img, lam_f):.2e}")


def test_packed_events_brick_layout_match_dequantized_oracle(packed_case):
    # packed events over the 2x2x2-brick copies (the layout the autotuner picks for
    # packed events with FP32 gathers on the full body): the first pass streams the
    # host events in the linear layout, the later passes run over the bricks
    g, ev, lors, rec, lam_q, hist_q, lam_f = packed_case
    img, cons = run(g, lors, B.make_events(rec, packed=True, lattice_mm=synth.LATTICE_MM), False,
                    launch=(128, 0, 0, 0, 3, 1))
    assert rel_l2(img, lam_q) <= 1e-4
    assert max_rel_above(img, lam_q, 0.01) <= 1e-3
    for k in range(5):
        assert cons[k, 0] == pytest.approx(hist_q[k][0], abs=0.5)
        assert cons[k, 1] == pytest.approx(cons[k, 0], rel=1e-5)


def test_packed_events_bf16_gather_error_is_bounded(packed_case):
    g, ev, lors, rec, lam_q, hist_q, lam_f = packed_case
    img, cons = run(g, lors, B.make_events(rec, packed=True, lattice_mm=synth.LATTICE_MM), True)
    err = rel_l2(img, lam_q)
    print(f"\npacked BF16-gather: rel L2 vs dequantized oracle {err:.2e}, vs unquantized {rel_l2(img, lam_f):.2e}")
    assert err <= 5e-3
    # p_i comes from the BF16 copy while the update multiplies the FP32 image, so
    # sum_j s_j lambda_j = sum_i w_i p_i(FP32) / p_i(BF16) matches N_eff only to
    # the BF16 rounding of p_i, averaged over the events
    assert cons[-1, 1] == pytest.approx(cons[-1, 0], rel=1e-3)


def test_fp32_events_bf16_gather(packed_case):
    g, ev, lors, rec, lam_q, hist_q, lam_f = packed_case
    img, cons = run(g, lors, B.make_events(ev), True)
    assert rel_l2(img, lam_f) <= 5e-3
