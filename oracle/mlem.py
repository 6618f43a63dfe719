"""List-mode TOF-MLEM and the nine-region division, FP64, in plain numpy.

TEST INFRASTRUCTURE (see oracle/__init__.py).

MLEM (Sec. 2.4; Shepp & Vardi 1982 written for list-mode events):
    p_i      = sum_j a_ij lambda_j                      forward projection
    C_j      = sum_{i: p_i > 0} a_ij w_i / p_i          backprojection of w/p
    lambda_j <- lambda_j C_j / s_j   where s_j > 0, else 0
with w_i = 1 except in the region division.  Readings taken where the paper
is silent: events with p_i = 0 are skipped; the start image is uniform on the
mask {s_j > 0} with sum_j s_j lambda_j = sum_i w_i.

Region division (Sec. 2.5): regions are consecutive core slice ranges
[lo_r, hi_r); core boundaries z_b[r] = oz + lo_r vz.  Each event goes to the
regions whose core, widened by the 6 mm shell on both sides, contains its
TOF-estimated z; an event fed to two regions carries w_i = 1/2 in each, so the
summed image counts every event once.  Region r is reconstructed on the slab
of slices [lo_r - m, hi_r + m) (clipped to the grid), m = ceil(margin / vz),
with the global sensitivity restricted to the slab; the nine images are then
summed into the whole-body volume (Sec. 2.5, last paragraph).
"""
import math

import numpy as np

from .core import Grid, backproject, backproject_lut, forward, forward_lut, region_codes, region_members
from .filters import sieve


def uniform_start(sens, weights_total):
    s = np.asarray(sens, np.float64).reshape(-1)
    mask = s > 0
    lam = np.zeros_like(s)
    if mask.any():
        lam[mask] = weights_total / s[mask].sum()
    return lam


def start_backprojection(grid, events, sens, sigma, K=3.0, weights=None, threads=None):
    """Starting image from a backprojection of the events (Sec. 3.5.4 and Table 2
    seed MLEM with a "starting backprojection"; its normalisation is not given).
    Reading: lambda0_j = sum_i a_ij w_i / s_j on {s_j > 0}, 0 elsewhere, i.e. the
    events' TOF-weighted backprojection divided by the sensitivity, so that
    sum_j s_j lambda0_j = sum_i w_i (mass of event i's window inside the mask)."""
    s = np.asarray(sens, np.float64).reshape(-1)
    n = np.asarray(events[0]).shape[0]
    w = np.ones(n) if weights is None else np.asarray(weights, np.float64)
    bp = backproject(grid, events, w, sigma, K, threads)
    lam = np.zeros_like(s)
    mask = s > 0
    lam[mask] = bp[mask] / s[mask]
    return lam


def mlem(grid, events, sens, n_iter, sigma, K=3.0, weights=None, init=None, threads=None, return_p=False,
         lut_samples=None, median=False):
    """Run n_iter MLEM iterations.

    Returns (lambda, history) where history[k] = (N_eff, sum_j s_j lambda_j,
    log-likelihood at the image the iteration started from).  N_eff is the
    weight of the events with p_i > 0 in iteration k.  lut_samples=N swaps the
    exact projector for the sampled TOF kernel of Sec. 2.3 (N samples).
    median=True applies the median-filter sieve of Sec. 2.4 (oracle.filters)
    after each update; the history then holds sum_j s_j lambda_j of the
    update, before the filter.
    """
    s = np.asarray(sens, np.float64).reshape(-1)
    assert s.size == grid.n_vox
    n = np.asarray(events[0]).shape[0]
    w = np.ones(n) if weights is None else np.asarray(weights, np.float64)
    mask = s > 0
    lam = uniform_start(s, w.sum()) if init is None else np.asarray(init, np.float64).reshape(-1).copy()
    history = []
    p = None
    for _ in range(n_iter):
        if lut_samples:
            p = forward_lut(grid, events, lam, lut_samples, sigma, K, threads)
        else:
            p = forward(grid, events, lam, sigma, K, threads)
        valid = p > 0
        r = np.zeros(n)
        r[valid] = w[valid] / p[valid]
        loglik = float(np.sum(w[valid] * np.log(p[valid])) - np.sum(s * lam))
        if lut_samples:
            Cimg = backproject_lut(grid, events, r, lut_samples, sigma, K, threads)
        else:
            Cimg = backproject(grid, events, r, sigma, K, threads)
        new = np.zeros_like(lam)
        new[mask] = lam[mask] * Cimg[mask] / s[mask]
        lam = new
        history.append((float(w[valid].sum()), float(np.sum(s * lam)), loglik))
        if median:
            lam = sieve(lam, s, grid.shape_zyx)
    if return_p:
        return lam, history, p
    return lam, history


def region_bounds(grid, regions):
    """Core z boundaries z_b[0..R] of consecutive slice ranges [lo, hi)."""
    for a, b in zip(regions[:-1], regions[1:]):
        if a[1] != b[0]:
            raise ValueError("regions must be consecutive slice ranges")
    ks = [regions[0][0]] + [hi for (_, hi) in regions]
    return np.array([grid.oz + k * grid.vz for k in ks], np.float64)


def region_slabs(grid, regions, margin_mm):
    """Slice range [lo, hi) reconstructed for each region."""
    m = int(math.ceil(margin_mm / grid.vz - 1e-12))
    return [(max(0, lo - m), min(grid.nz, hi + m)) for (lo, hi) in regions]


def slab_grid(grid, lo, hi):
    return Grid(grid.nx, grid.ny, hi - lo, grid.vx, grid.vy, grid.vz, grid.ox, grid.oy, grid.oz + lo * grid.vz)


def stitch(grid, slabs, images):
    """Whole-body image = sum over regions of each slab image at its place."""
    out = np.zeros(grid.shape_zyx)
    for (lo, hi), img in zip(slabs, images):
        out[lo:hi] += np.asarray(img).reshape(hi - lo, grid.ny, grid.nx)
    return out.reshape(-1)


def mlem_regions(grid, events, sens, regions, shell_mm, margin_mm, n_iter, sigma, K=3.0, threads=None,
                 lut_samples=None, median=False):
    """Divide events by TOF-estimated z, reconstruct each slab, sum the slabs.

    Returns (image, per-region images, per-region histories, codes, offsets, idx).
    """
    events = [np.asarray(e, np.float64) for e in events]
    zb = region_bounds(grid, regions)
    codes = region_codes(events, zb, shell_mm)
    offsets, idx = region_members(codes, len(regions))
    w_all = np.where((codes & 0x80) != 0, 0.5, 1.0)
    slabs = region_slabs(grid, regions, margin_mm)
    s3 = np.asarray(sens, np.float64).reshape(grid.shape_zyx)
    images, hists = [], []
    for r, (lo, hi) in enumerate(slabs):
        members = idx[offsets[r]:offsets[r + 1]]
        ev_r = [e[members] for e in events]
        g_r = slab_grid(grid, lo, hi)
        lam_r, h_r = mlem(g_r, ev_r, s3[lo:hi].reshape(-1), n_iter, sigma, K, weights=w_all[members],
                          threads=threads, lut_samples=lut_samples, median=median)
        images.append(lam_r)
        hists.append(h_r)
    return stitch(grid, slabs, images), images, hists, codes, offsets, idx


def subset_ranges(n, n_subsets):
    """Event ranges of the OSEM subsets: B consecutive blocks of the list."""
    return [(b * n // n_subsets, (b + 1) * n // n_subsets) for b in range(n_subsets)]


def osem(grid, events, sens, n_iter, n_subsets, sigma, K=3.0, weights=None, init=None, threads=None):
    """List-mode OSEM (named in the title of Sec. 2.4; the paper reconstructs
    with MLEM).  Reading: subset b holds the events of block b of the list
    (subset_ranges; list-mode data arrive in random order, so blocks are random
    partitions), and a sub-iteration is one MLEM update with that subset's
    backprojection against the sensitivity scaled by 1/B:
        lambda_j <- lambda_j C_j^b / (s_j / B)   where s_j > 0, else 0.
    Returns (lambda, history) with one (N_eff of the subset, sum_j s_j lambda_j)
    entry per sub-iteration; sum_j s_j lambda_j = B N_eff after each one.
    """
    s = np.asarray(sens, np.float64).reshape(-1)
    n = np.asarray(events[0]).shape[0]
    w = np.ones(n) if weights is None else np.asarray(weights, np.float64)
    mask = s > 0
    lam = uniform_start(s, w.sum()) if init is None else np.asarray(init, np.float64).reshape(-1).copy()
    history = []
    for _ in range(n_iter):
        for lo, hi in subset_ranges(n, n_subsets):
            ev_b = [np.asarray(e)[lo:hi] for e in events]
            w_b = w[lo:hi]
            p = forward(grid, ev_b, lam, sigma, K, threads)
            valid = p > 0
            r = np.zeros(hi - lo)
            r[valid] = w_b[valid] / p[valid]
            Cimg = backproject(grid, ev_b, r, sigma, K, threads)
            new = np.zeros_like(lam)
            new[mask] = lam[mask] * Cimg[mask] / (s[mask] / n_subsets)
            lam = new
            history.append((float(w_b[valid].sum()), float(np.sum(s * lam))))
    return lam, history
