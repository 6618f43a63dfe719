"""Shared inputs and comparison helpers of the GPU parity tests.

Inputs come from the seeded generator (paper_1706_07075_b300.synth); the
expected values come from the FP64 oracle on the same inputs.
"""
import functools

import numpy as np

import oracle
from oracle import Grid
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

TOF_FWHM_PS = 300.0
SIGMA = oracle.tof_sigma_mm(TOF_FWHM_PS)


def grid_tuple(g):
    return (g.nx, g.ny, g.nz, g.vx, g.vy, g.vz, g.ox, g.oy, g.oz)


def workload_grid(name):
    return Grid(*synth.grid_of(name))


def geometry(name):
    sc = synth.WORKLOADS[name]().scanner
    return (sc.radius_mm, sc.axial_len_mm, sc.max_axial_angle_deg)


@functools.lru_cache(maxsize=None)
def tiny_inputs(n_events=200_000, n_lors=2_000_000, seed=1706):
    ev = synth.events("tiny", n_events, seed)
    lors = synth.sensitivity_lors("tiny", n_lors, seed)
    return ev, lors


@functools.lru_cache(maxsize=None)
def oracle_sensitivity(name, n_lors, seed):
    g = workload_grid(name)
    lors = synth.sensitivity_lors(name, n_lors, seed)
    return oracle.sensitivity(g, lors)


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_rel_above(a, b, frac=0.01):
    """Largest per-voxel relative error over voxels above frac * max(b)."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    sel = b > frac * b.max()
    return float(np.max(np.abs(a[sel] - b[sel]) / b[sel])) if sel.any() else 0.0


def new_context(name, **kw):
    return B.Context(geometry(name), grid_tuple(workload_grid(name)), kw.get("fwhm", TOF_FWHM_PS))


def lut_unambiguous(g, ev, n_samples):
    """The events of ev ((7, n) float32) none of whose n_samples samples lies within
    oracle.LUT_EPS_VOXELS of a voxel plane (oracle.lut_ambiguous): on those the
    kernel's FP32 voxel decisions equal the oracle's FP64 ones."""
    mask = oracle.lut_ambiguous(g, ev.astype(np.float64), n_samples, SIGMA) == 0
    return np.ascontiguousarray(ev[:, mask])
