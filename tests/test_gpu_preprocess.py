"""GPU event pre-processing (attenuation weights, Sec. 2.4; TOF scatter
rejection at 95% confidence, Sec. 2.2) vs the oracle.

The keep/reject decision is an integer decided by floating point: the GPU
clips the window and walks the line in FP32, the oracle in FP64.  An event
may therefore differ only where the decision is not unique at FP32
resolution: the oracle's decision flips when z moves by +-5e-5 (1e-3 mm of
window), which the tests check for every mismatch.

Weights: w = exp(integral), so the relative error of w is the absolute error
of the FP32 line integral.  Its floor is geometric, as for the sensitivity
image: the FP32 line direction carries ~6e-8 relative rounding, which moves a
1 m long LOR sideways by ~1e-4 mm, and a line nearly parallel to a voxel plane
turns that into up to millimetres of chord moved between voxels of different
mu.  Typical events agree to ~1e-6 (99.9th percentile held to 1e-5); the
worst event of a full-body sample is held to 2e-4.
"""
import numpy as np
import pytest

import oracle
from gpu_common import SIGMA, geometry, grid_tuple, max_rel_above, rel_l2, tiny_inputs, workload_grid
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

pytestmark = pytest.mark.gpu
Z95 = 1.96
DZ = 5e-5


def ambiguous(g, ev64, mu, idx):
    """Events among idx whose oracle decision flips within z = 1.96 +- DZ."""
    sub = [e[idx] for e in ev64]
    _, k_lo, _ = oracle.preprocess(g, sub, mu, SIGMA, z=Z95 - DZ)
    _, k_hi, _ = oracle.preprocess(g, sub, mu, SIGMA, z=Z95 + DZ)
    return k_lo != k_hi


def check_against_oracle(g, ev, mu, w, keep, kept):
    ev64 = ev.astype(np.float64)
    w_ref, keep_ref, kept_ref = oracle.preprocess(g, ev64, mu.astype(np.float64), SIGMA, z=Z95)
    assert kept == int(keep.sum())
    diff = np.nonzero(keep != keep_ref)[0]
    if diff.size:
        assert np.all(ambiguous(g, ev64, mu.astype(np.float64), diff)), diff[:10]
    both = (keep == 1) & (keep_ref == 1)
    rel = np.abs(w[both] - w_ref[both]) / w_ref[both]
    assert np.percentile(rel, 99.9) < 1e-5
    assert rel.max() < 2e-4
    assert np.all(w[keep == 0] == 0)
    assert 0.1 < kept_ref / ev.shape[1] < 1.0          # the phantom rejects some, keeps most
    return w_ref, keep_ref, diff


def test_preprocess_tiny_matches_oracle():
    ev, _ = tiny_inputs()
    g = workload_grid("tiny")
    mu = synth.mu_image("tiny")
    n = ev.shape[1]
    w = np.zeros(n, np.float32)
    keep = np.zeros(n, np.uint8)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        kept = ctx.preprocess(B.make_events(ev), mu, Z95, 0, w, keep)
    check_against_oracle(g, ev, mu, w, keep, kept)


def test_preprocess_without_rejection_keeps_all():
    ev, _ = tiny_inputs()
    g = workload_grid("tiny")
    mu = synth.mu_image("tiny")
    sub = np.ascontiguousarray(ev[:, :20000])
    w = np.zeros(sub.shape[1], np.float32)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        kept = ctx.preprocess(B.make_events(sub), mu, 0.0, 0, w, None)
    w_ref, keep_ref, kept_ref = oracle.preprocess(g, sub.astype(np.float64), mu.astype(np.float64), SIGMA, z=0.0)
    assert kept == kept_ref == sub.shape[1]
    rel = np.abs(w - w_ref) / w_ref
    assert np.percentile(rel, 99.9) < 1e-5 and rel.max() < 2e-4


def test_preprocess_fullbody_sampled():
    g = workload_grid("fullbody")
    ev = synth.events("fullbody", 2_000_000, 12)
    mu = synth.mu_image("fullbody")
    n = ev.shape[1]
    w = np.zeros(n, np.float32)
    keep = np.zeros(n, np.uint8)
    with B.Context(geometry("fullbody"), grid_tuple(g), 300.0) as ctx:
        kept = ctx.preprocess(B.make_events(ev), mu, Z95, 0, w, keep)
    assert kept == int(keep.sum())
    pick = np.arange(0, n, 101)
    check_against_oracle(g, np.ascontiguousarray(ev[:, pick]), mu, w[pick], keep[pick], int(keep[pick].sum()))


def test_preprocess_apply_then_mlem_matches_weighted_oracle():
    ev, lors = tiny_inputs()
    g = workload_grid("tiny")
    mu = synth.mu_image("tiny").astype(np.float64)
    ev64 = ev.astype(np.float64)
    w_ref, keep_ref, _ = oracle.preprocess(g, ev64, mu, SIGMA, z=Z95)
    # inputs: drop the events whose decision is not unique at FP32 resolution
    amb = ambiguous(g, ev64, mu, np.arange(ev.shape[1]))
    ev = np.ascontiguousarray(ev[:, ~amb])
    w_ref, keep_ref = w_ref[~amb], keep_ref[~amb]
    s_ref = oracle.sensitivity(g, lors)
    lam_ref, hist = oracle.mlem(g, ev.astype(np.float64), s_ref, 3, SIGMA, weights=w_ref)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        kept = ctx.preprocess(B.make_events(ev), mu.astype(np.float32), Z95, 1)
        assert kept == int(keep_ref.sum())
        lam = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((3, 2))
        ctx.mlem(None, 3, None, lam, cons)
    assert rel_l2(lam, lam_ref) <= 1e-4
    assert max_rel_above(lam, lam_ref, 0.01) <= 1e-3
    for k in range(3):
        assert cons[k, 0] == pytest.approx(hist[k][0], rel=1e-5)


def test_preprocess_packed_events():
    ev = synth.events("tiny", 60_000, 43)
    rec = synth.pack_events(ev)
    q = rec[:, :6].astype(np.float64).T * synth.LATTICE_MM
    d = rec[:, 6].view(np.float16).astype(np.float64)
    evq = np.concatenate([q, d[None, :]])
    g = workload_grid("tiny")
    mu = synth.mu_image("tiny")
    n = ev.shape[1]
    w = np.zeros(n, np.float32)
    keep = np.zeros(n, np.uint8)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        kept = ctx.preprocess(B.make_events(rec, packed=True, lattice_mm=synth.LATTICE_MM), mu, Z95, 0, w, keep)
    check_against_oracle(g, evq.astype(np.float32), mu, w, keep, kept)


def test_preprocess_argument_checks():
    g = workload_grid("tiny")
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        with pytest.raises(B.ReconError):
            ctx.preprocess(None, np.zeros(g.n_vox, np.float32))          # no events yet
        ev = synth.events("tiny", 100, 1)
        with pytest.raises(B.ReconError):
            ctx.preprocess(B.make_events(ev), None)
        with pytest.raises(B.ReconError):
            ctx.preprocess(B.make_events(ev), np.zeros(g.n_vox, np.float32), -1.0)


def test_preprocess_apply_packed_then_mlem():
    # packed events keep their weight in FP16: the weighted MLEM then matches the oracle
    # (same FP16-rounded weights on both sides) to the plain tolerances
    ev = synth.events("tiny", 120_000, 47)
    rec = synth.pack_events(ev)
    q = rec[:, :6].astype(np.float64).T * synth.LATTICE_MM
    d = rec[:, 6].view(np.float16).astype(np.float64)
    evq = np.concatenate([q, d[None, :]])
    g = workload_grid("tiny")
    mu = synth.mu_image("tiny").astype(np.float64)
    lors = synth.sensitivity_lors("tiny", 500_000, 47)
    s_ref = oracle.sensitivity(g, lors)
    amb = ambiguous(g, evq, mu, np.arange(evq.shape[1]))
    rec = np.ascontiguousarray(rec[~amb])
    evq = evq[:, ~amb]
    w_ref, keep_ref, _ = oracle.preprocess(g, evq, mu, SIGMA, z=Z95)
    w16 = w_ref.astype(np.float16).astype(np.float64)            # the packed record's FP16 weight
    lam_ref, hist = oracle.mlem(g, evq, s_ref, 3, SIGMA, weights=w16)
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        kept = ctx.preprocess(B.make_events(rec, packed=True, lattice_mm=synth.LATTICE_MM), mu.astype(np.float32),
                              Z95, 1)
        assert kept == int(keep_ref.sum())
        lam = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((3, 2))
        ctx.mlem(None, 3, None, lam, cons)
    assert rel_l2(lam, lam_ref) <= 1e-3
    assert max_rel_above(lam, lam_ref, 0.01) <= 1e-2
    for k in range(3):
        assert cons[k, 0] == pytest.approx(hist[k][0], rel=1e-3)
