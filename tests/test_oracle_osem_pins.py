"""Pins of the oracle's list-mode OSEM (named in Sec. 2.4's title): against a
dense textbook OSEM on the brute-force system matrix, the per-sub-iteration
conservation sum_j s_j lambda_j = B N_eff, and B = 1 reducing to MLEM."""
import numpy as np
import pytest

import oracle
from test_oracle_pins import dense_chords, dense_system, small_problem


def textbook_osem(A, s, n_iter, B):
    n, J = A.shape
    mask = s > 0
    lam = np.where(mask, n / s[mask].sum(), 0.0)
    blocks = [(b * n // B, (b + 1) * n // B) for b in range(B)]
    for _ in range(n_iter):
        for lo, hi in blocks:
            Ab = A[lo:hi]
            p = Ab @ lam
            ratio = np.where(p > 0, 1.0 / np.where(p > 0, p, 1.0), 0.0)
            lam = np.where(mask, lam * (Ab.T @ ratio) * B / np.where(mask, s, 1.0), 0.0)
    return lam


def test_osem_matches_dense_textbook_osem_8cubed():
    g, sigma, ev, lors = small_problem(31, n_ev=1800, n_lor=1500)
    A = dense_system(g, ev, sigma, 3.0)
    s_dense = dense_chords(g, lors)
    s = oracle.sensitivity(g, lors)
    for B in (2, 3, 5):
        lam, hist = oracle.osem(g, ev, s, 2, B, sigma, 3.0)
        ref = textbook_osem(A, s_dense, 2, B)
        assert np.max(np.abs(lam - ref)) <= 1e-11 * np.max(ref)
        assert len(hist) == 2 * B
        for n_eff, ssum in hist:
            assert ssum == pytest.approx(B * n_eff, rel=1e-12)


def test_osem_one_subset_is_mlem():
    g, sigma, ev, lors = small_problem(32, n_ev=600, n_lor=800)
    s = oracle.sensitivity(g, lors)
    lam1, h1 = oracle.osem(g, ev, s, 3, 1, sigma, 3.0)
    lam2, h2 = oracle.mlem(g, ev, s, 3, sigma, 3.0)
    assert np.array_equal(lam1, lam2)
    assert [h[:2] for h in h2] == h1


def test_subset_ranges_partition_the_list():
    for n, B in [(10, 3), (7, 7), (100, 1), (5, 8)]:
        r = oracle.subset_ranges(n, B)
        assert r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r[:-1], r[1:]))


def test_start_backprojection_dense_and_first_iteration():
    g, sigma, ev, lors = small_problem(33, n_ev=500, n_lor=1500)
    A = dense_system(g, ev, sigma, 3.0)
    s_dense = dense_chords(g, lors)
    s = oracle.sensitivity(g, lors)
    lam0 = oracle.start_backprojection(g, ev, s, sigma, 3.0)
    mask = s_dense > 0
    ref = np.where(mask, (A.T @ np.ones(A.shape[0])) / np.where(mask, s_dense, 1.0), 0.0)
    assert np.max(np.abs(lam0 - ref)) <= 1e-11 * np.max(ref)
    # with a positive sensitivity everywhere, one MLEM iteration from a constant image
    # of events whose windows lie inside the grid is the starting backprojection
    s_pos = np.full(g.n_vox, 7.0)
    inside = np.isclose(A.sum(axis=1), 1.0, rtol=1e-12)
    ev_in = [e[inside] for e in ev]
    lam1, _ = oracle.mlem(g, ev_in, s_pos, 1, sigma, 3.0)
    np.testing.assert_allclose(lam1, oracle.start_backprojection(g, ev_in, s_pos, sigma, 3.0), rtol=1e-11,
                               atol=1e-15)
