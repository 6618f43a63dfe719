"""ctypes wrappers over the FP64 C oracle (oracle.c).  Test infrastructure.

Events are passed as seven FP64 planes (x1, y1, z1, x2, y2, z2, d) in mm; FP32
inputs are widened exactly.  Work over many events is split into contiguous
event ranges run on Python threads (ctypes releases the GIL); backprojection
gives each range its own accumulator and sums them in range order, so a run
is deterministic for a fixed thread count.
"""
import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None
_lock = threading.Lock()


class _OgGrid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("vx", C.c_double), ("vy", C.c_double), ("vz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


@dataclass(frozen=True)
class Grid:
    """nx*ny*nz voxels of (vx, vy, vz) mm; (ox, oy, oz) is the low corner."""
    nx: int
    ny: int
    nz: int
    vx: float
    vy: float
    vz: float
    ox: float
    oy: float
    oz: float

    @staticmethod
    def centred(nx, ny, nz, vx, vy=None, vz=None):
        vy = vx if vy is None else vy
        vz = vx if vz is None else vz
        return Grid(nx, ny, nz, vx, vy, vz, -0.5 * nx * vx, -0.5 * ny * vy, -0.5 * nz * vz)

    @property
    def shape_zyx(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_vox(self):
        return self.nx * self.ny * self.nz

    def c(self):
        return _OgGrid(self.nx, self.ny, self.nz, self.vx, self.vy, self.vz, self.ox, self.oy, self.oz)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int64)
            gp = C.POINTER(_OgGrid)
            planes = C.POINTER(C.c_void_p)
            lib.oracle_tof_sigma_mm.argtypes = [C.c_double]
            lib.oracle_tof_sigma_mm.restype = C.c_double
            lib.oracle_tof_weight.argtypes = [C.c_double] * 5
            lib.oracle_tof_weight.restype = C.c_double
            lib.oracle_trace.argtypes = [gp, dp, dp, C.c_double, C.c_double, C.c_int64, ip, dp, dp]
            lib.oracle_trace.restype = C.c_int64
            lib.oracle_system_row.argtypes = [gp, planes, C.c_int64, C.c_double, C.c_double, C.c_int64, ip, dp]
            lib.oracle_system_row.restype = C.c_int64
            lib.oracle_forward.argtypes = [gp, planes, C.c_int64, C.c_int64, C.c_double, C.c_double, dp, dp]
            lib.oracle_forward.restype = C.c_int
            lib.oracle_backproject.argtypes = [gp, planes, C.c_int64, C.c_int64, C.c_double, C.c_double, dp, dp]
            lib.oracle_backproject.restype = C.c_int
            lib.oracle_count_visits.argtypes = [gp, planes, C.c_int64, C.c_int64, C.c_double, C.c_double]
            lib.oracle_count_visits.restype = C.c_int64
            lib.oracle_sensitivity.argtypes = [gp, planes, C.c_int64, C.c_int64, dp]
            lib.oracle_sensitivity.restype = C.c_int
            lib.oracle_region_codes.argtypes = [planes, C.c_int64, C.c_int64, C.c_int32, dp, C.c_double,
                                                C.POINTER(C.c_uint8), dp]
            lib.oracle_region_codes.restype = C.c_int64
            lib.oracle_preprocess.argtypes = [gp, planes, C.c_int64, C.c_int64, dp, C.c_double, C.c_double, dp,
                                              C.POINTER(C.c_uint8)]
            lib.oracle_preprocess.restype = C.c_int64
            lib.oracle_lut_samples.argtypes = [C.c_int32, C.c_double, C.c_double, dp, dp]
            lib.oracle_lut_samples.restype = None
            lib.oracle_forward_lut.argtypes = [gp, planes, C.c_int64, C.c_int64, C.c_int32, dp, dp, dp, dp]
            lib.oracle_forward_lut.restype = C.c_int
            lib.oracle_backproject_lut.argtypes = [gp, planes, C.c_int64, C.c_int64, C.c_int32, dp, dp, dp, dp]
            lib.oracle_backproject_lut.restype = C.c_int
            lib.oracle_lut_ambiguous.argtypes = [gp, planes, C.c_int64, C.c_int64, C.c_int32, dp, C.c_double,
                                                 C.POINTER(C.c_int32)]
            lib.oracle_lut_ambiguous.restype = C.c_int
            _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _planes(arrs):
    """Pack FP64 contiguous planes into a void* array; keep the arrays alive."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
    ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    return arrs, ptrs


def _event_planes(events):
    """events: (7, n) array-like or sequence of 7 planes."""
    if isinstance(events, np.ndarray) and events.ndim == 2:
        planes = [events[k] for k in range(events.shape[0])]
    else:
        planes = list(events)
    return _planes(planes)


def threads_used(n_items=None):
    """Threads the oracle spreads work over: all host cores (capped by items)."""
    t = os.cpu_count() or 1
    env = os.environ.get("ORACLE_THREADS")
    if env:
        t = max(1, int(env))
    if n_items is not None:
        t = max(1, min(t, int(n_items)))
    return t


def _ranges(n, parts):
    edges = np.linspace(0, n, parts + 1).astype(np.int64)
    return [(int(edges[k]), int(edges[k + 1])) for k in range(parts)]


def _run_threads(fn, ranges):
    out = [None] * len(ranges)

    def work(k, r):
        out[k] = fn(*r)

    ths = [threading.Thread(target=work, args=(k, r)) for k, r in enumerate(ranges)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    return out


# ------------------------------------------------------------------ constants

def tof_sigma_mm(fwhm_ps):
    """sigma along the LOR for a coincidence timing FWHM (Sec. 2.5)."""
    return _load().oracle_tof_sigma_mm(float(fwhm_ps))


def tof_weight(ta, tb, d, sigma, K):
    return _load().oracle_tof_weight(float(ta), float(tb), float(d), float(sigma), float(K))


# ------------------------------------------------------------------ tracing

def trace(grid, p1, p2, t_lo=-np.inf, t_hi=np.inf):
    """Siddon segments of the LOR P1-P2 in [t_lo, t_hi]: (vox, t_a, t_b)."""
    lib = _load()
    cap = grid.nx + grid.ny + grid.nz + 8
    vox = np.zeros(cap, np.int64)
    ta = np.zeros(cap)
    tb = np.zeros(cap)
    a = np.ascontiguousarray(p1, np.float64)
    b = np.ascontiguousarray(p2, np.float64)
    g = grid.c()
    n = lib.oracle_trace(C.byref(g), _dptr(a), _dptr(b), float(t_lo), float(t_hi), cap,
                         vox.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(ta), _dptr(tb))
    if n < 0:
        raise RuntimeError(f"oracle_trace failed ({n})")
    return vox[:n].copy(), ta[:n].copy(), tb[:n].copy()


def system_row(grid, events, i, sigma, K=3.0):
    """Sparse row of event i: (voxel indices, a_ij)."""
    lib = _load()
    keep, ptrs = _event_planes(events)
    cap = grid.nx + grid.ny + grid.nz + 8
    vox = np.zeros(cap, np.int64)
    a = np.zeros(cap)
    g = grid.c()
    n = lib.oracle_system_row(C.byref(g), ptrs, int(i), float(sigma), float(K), cap,
                              vox.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(a))
    if n < 0:
        raise RuntimeError(f"oracle_system_row failed ({n})")
    return vox[:n].copy(), a[:n].copy()


def forward(grid, events, lam, sigma, K=3.0, threads=None):
    """p_i = sum_j a_ij lambda_j for every event (FP64)."""
    lib = _load()
    keep, ptrs = _event_planes(events)
    n = keep[0].shape[0]
    lam = np.ascontiguousarray(lam, np.float64).reshape(-1)
    assert lam.size == grid.n_vox
    p = np.zeros(n)
    g = grid.c()
    if n == 0:
        return p

    def part(i0, i1):
        return lib.oracle_forward(C.byref(g), ptrs, i0, i1, float(sigma), float(K), _dptr(lam), _dptr(p))

    rcs = _run_threads(part, _ranges(n, threads or threads_used(n)))
    if any(rc != 0 for rc in rcs):
        raise RuntimeError(f"oracle_forward failed {rcs}")
    return p


def backproject(grid, events, r, sigma, K=3.0, threads=None):
    """C_j = sum_i a_ij r_i (FP64)."""
    lib = _load()
    keep, ptrs = _event_planes(events)
    n = keep[0].shape[0]
    r = np.ascontiguousarray(r, np.float64).reshape(-1)
    assert r.size == n
    g = grid.c()
    ranges = _ranges(n, threads or threads_used(n)) if n else []
    accs = [np.zeros(grid.n_vox) for _ in ranges]

    def part(i0, i1, k):
        return lib.oracle_backproject(C.byref(g), ptrs, i0, i1, float(sigma), float(K), _dptr(r), _dptr(accs[k]))

    rcs = _run_threads(part, [(a, b, k) for k, (a, b) in enumerate(ranges)])
    if any(rc != 0 for rc in rcs):
        raise RuntimeError(f"oracle_backproject failed {rcs}")
    total = np.zeros(grid.n_vox)
    for acc in accs:
        total += acc
    return total


def count_visits(grid, events, sigma, K=3.0, threads=None):
    """Total number of voxel segments inside the TOF windows of all events."""
    lib = _load()
    keep, ptrs = _event_planes(events)
    n = keep[0].shape[0]
    if n == 0:
        return 0
    g = grid.c()

    def part(i0, i1):
        return lib.oracle_count_visits(C.byref(g), ptrs, i0, i1, float(sigma), float(K))

    return int(sum(_run_threads(part, _ranges(n, threads or threads_used(n)))))


def sensitivity(grid, lors, threads=None):
    """s_j = sum_l L_lj over LORs given as six planes (full chord, mm, FP64)."""
    lib = _load()
    if isinstance(lors, np.ndarray) and lors.ndim == 2:
        planes = [lors[k] for k in range(6)]
    else:
        planes = list(lors)
    keep, ptrs = _planes(planes)
    n = keep[0].shape[0]
    g = grid.c()
    ranges = _ranges(n, threads or threads_used(n)) if n else []
    accs = [np.zeros(grid.n_vox) for _ in ranges]

    def part(l0, l1, k):
        return lib.oracle_sensitivity(C.byref(g), ptrs, l0, l1, _dptr(accs[k]))

    rcs = _run_threads(part, [(a, b, k) for k, (a, b) in enumerate(ranges)])
    if any(rc != 0 for rc in rcs):
        raise RuntimeError(f"oracle_sensitivity failed {rcs}")
    total = np.zeros(grid.n_vox)
    for acc in accs:
        total += acc
    return total


# ------------------------------------------------------- pre-processing

def preprocess(grid, events, mu, sigma, z=1.96, threads=None):
    """Attenuation weights and TOF scatter rejection (Sec. 2.4, Sec. 2.2).

    Returns (w, keep, kept): w_i = exp(sum_j mu_j L_ij) for kept events and 0
    for rejected ones; keep_i = 1 iff [d - z sigma, d + z sigma] meets a voxel
    with mu > 0 (z <= 0: keep all).
    """
    lib = _load()
    keep_planes, ptrs = _event_planes(events)
    n = keep_planes[0].shape[0]
    mu = np.ascontiguousarray(mu, np.float64).reshape(-1)
    assert mu.size == grid.n_vox
    w = np.zeros(n)
    keep = np.zeros(n, np.uint8)
    if n == 0:
        return w, keep, 0
    g = grid.c()

    def part(i0, i1):
        r = lib.oracle_preprocess(C.byref(g), ptrs, i0, i1, _dptr(mu), float(sigma), float(z), _dptr(w),
                                  keep.ctypes.data_as(C.POINTER(C.c_uint8)))
        if r < 0:
            raise MemoryError("oracle_preprocess buffer error")
        return r

    kept = int(sum(_run_threads(part, _ranges(n, threads or threads_used(n)))))
    return w, keep, kept


# --------------------------------------------------- sampled TOF kernel

def lut_samples(n_samples, sigma, K=3.0):
    """Offsets t_k (mm) and unit-sum Gaussian weights w_k of the sampled kernel."""
    t = np.zeros(n_samples)
    w = np.zeros(n_samples)
    _load().oracle_lut_samples(int(n_samples), float(sigma), float(K), _dptr(t), _dptr(w))
    return t, w


# Samples within this many voxels of a voxel plane are "ambiguous": an FP32
# evaluation of the sample position may put them in the neighbouring voxel.
# Bound on that FP32 error for one IEEE rounding per operation (unit roundoff
# 2^-24 = 6e-8), with coordinates up to 1.2 m, |d| up to 1 m and |t| up to 3
# sigma = 57 mm: the TOF point c = M + d u carries |M| 2^-24 + |d| 6 2^-24
# <= 4e-4 mm, c - o another 1.2e-4 mm, the voxel-unit scaling and the final
# fused multiply-add ~6e-5 voxel each, so the voxel coordinate of a sample is off
# by at most ~2e-4 voxel on the 4 mm full-body grid (less on smaller grids; the
# FP32 rounding of t_k adds 5e-7 voxel).  1e-3 voxel leaves a factor of five.
LUT_EPS_VOXELS = 1e-3


def _lut_args(n_samples, sigma, K):
    t, w = lut_samples(n_samples, sigma, K)
    return np.ascontiguousarray(w), np.ascontiguousarray(t)


def forward_lut(grid, events, lam, n_samples, sigma, K=3.0, threads=None):
    """p_i with the sampled kernel: sum_k w_k lambda(voxel of sample k), voxels
    decided in FP64 from the exact sample positions c + t_k u."""
    lib = _load()
    keep, ptrs = _event_planes(events)
    n = keep[0].shape[0]
    lam = np.ascontiguousarray(lam, np.float64).reshape(-1)
    p = np.zeros(n)
    if n == 0:
        return p
    w, t = _lut_args(n_samples, sigma, K)
    g = grid.c()

    def part(i0, i1):
        return lib.oracle_forward_lut(C.byref(g), ptrs, i0, i1, int(n_samples), _dptr(w), _dptr(t), _dptr(lam),
                                      _dptr(p))

    _run_threads(part, _ranges(n, threads or threads_used(n)))
    return p


def backproject_lut(grid, events, r, n_samples, sigma, K=3.0, threads=None):
    """C_j = sum over samples in voxel j of w_k r_i (sampled kernel)."""
    lib = _load()
    keep, ptrs = _event_planes(events)
    n = keep[0].shape[0]
    r = np.ascontiguousarray(r, np.float64).reshape(-1)
    w, t = _lut_args(n_samples, sigma, K)
    g = grid.c()
    ranges = _ranges(n, threads or threads_used(n)) if n else []
    accs = [np.zeros(grid.n_vox) for _ in ranges]

    def part(i0, i1, k):
        return lib.oracle_backproject_lut(C.byref(g), ptrs, i0, i1, int(n_samples), _dptr(w), _dptr(t), _dptr(r),
                                          _dptr(accs[k]))

    _run_threads(part, [(a, b, k) for k, (a, b) in enumerate(ranges)])
    total = np.zeros(grid.n_vox)
    for acc in accs:
        total += acc
    return total


def lut_ambiguous(grid, events, n_samples, sigma, K=3.0, eps=LUT_EPS_VOXELS, threads=None):
    """Per event, how many of its samples lie within eps voxels of a voxel plane
    (or of the grid boundary), where a lower-precision evaluation of the sample
    position may choose the neighbouring voxel."""
    lib = _load()
    keep, ptrs = _event_planes(events)
    n = keep[0].shape[0]
    out = np.zeros(n, np.int32)
    if n == 0:
        return out
    _, t = _lut_args(n_samples, sigma, K)
    g = grid.c()

    def part(i0, i1):
        return lib.oracle_lut_ambiguous(C.byref(g), ptrs, i0, i1, int(n_samples), _dptr(t), float(eps),
                                        out.ctypes.data_as(C.POINTER(C.c_int32)))

    _run_threads(part, _ranges(n, threads or threads_used(n)))
    return out


# ---------------------------------------------------------- region division

def region_codes(events, z_bounds, shell_mm, return_z=False):
    """Per-event region code (0xFF: none; r; r | 0x80: regions r and r+1)."""
    lib = _load()
    keep, ptrs = _event_planes(events)
    n = keep[0].shape[0]
    zb = np.ascontiguousarray(z_bounds, np.float64)
    codes = np.zeros(n, np.uint8)
    z = np.zeros(n)
    bad = lib.oracle_region_codes(ptrs, 0, n, len(zb) - 1, _dptr(zb), float(shell_mm),
                                  codes.ctypes.data_as(C.POINTER(C.c_uint8)), _dptr(z))
    if bad:
        raise ValueError(f"{bad} events fall in three or more regions: cores narrower than 2*shell")
    return (codes, z) if return_z else codes


def region_members(codes, n_regions):
    """Stable per-region event lists (ascending index) and their offsets."""
    codes = np.asarray(codes, np.uint8)
    first = (codes & 0x7F).astype(np.int64)
    two = (codes & 0x80) != 0
    valid = codes != 0xFF
    lists = []
    for r in range(n_regions):
        member = valid & ((first == r) | (two & (first + 1 == r)))
        lists.append(np.nonzero(member)[0].astype(np.int32))
    offsets = np.zeros(n_regions + 1, np.int64)
    offsets[1:] = np.cumsum([len(x) for x in lists])
    idx = np.concatenate(lists) if lists else np.zeros(0, np.int32)
    return offsets, idx
