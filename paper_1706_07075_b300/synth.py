"""Seeded synthetic list-mode data shaped like the paper's workloads.

This module only simulates inputs: phantoms, annihilation points, photon
paths, detector hits, timing blur and sensitivity lines.  It holds none of
the reconstruction's arithmetic (no ray tracing through voxels, no TOF
kernel, no MLEM) and is the one piece shared by the CUDA library's callers
and the FP64 oracle's callers.

The paper's inputs (GEANT4 simulations of the NCAT phantom, Sec. 2 and 2.1)
are not available; these stand in for them:

* tiny: cylindrical detector R = 150 mm, axial 200 mm; a uniform cylinder
  (r = 50 mm, |z| <= 80 mm) with two hot spheres (r = 8 mm, 4:1); true
  coincidences only.
* full body: detector R = 400 mm, axial 2400 mm, axial acceptance below 45
  degrees (Sec. 2.1.2); nested ellipsoids for trunk, neck, head, legs, lungs
  (0.3x), liver (2x), heart (3x), bladder (8x), brain (2.5x) and ten 10-20 mm
  lesions (4-8x); 33% of the events are scattered once (deflection uniform
  along the in-body path, polar angle uniform in 0-60 degrees).
* small FOV: detector R = 60 mm, axial 100 mm; a 64 mm field of view.

Every event: emission point drawn from the activity, isotropic back-to-back
photons, endpoints on the cylinder's lateral surface, 0.4 mm FWHM Gaussian
blur per endpoint coordinate (the intrinsic resolution quoted in Sec. 1),
and a TOF offset from the true photon path lengths plus a 300 ps FWHM
Gaussian timing error on t2 - t1.  Event layout: FP32 SoA, seven planes
x1, y1, z1, x2, y2, z2, d (mm; d > 0 toward P1, d = c (t2 - t1) / 2).

Randomness: chunk k of a draw uses its own Philox stream keyed by
(seed, stream id, k), so results do not depend on the number of worker
processes.
"""
import math
import multiprocessing as mp
import os
from dataclasses import dataclass, field, replace
from multiprocessing import shared_memory

import numpy as np

C_MM_PER_PS = 0.299792458
FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))
CHUNK = 1 << 20
MU_WATER = 0.0096   # 1/mm at 511 keV: soft tissue
MU_LUNG = 0.0029    # 1/mm: lung (density ~0.3)


@dataclass(frozen=True)
class Shape:
    kind: str          # "ellipsoid" or "zcylinder"
    centre: tuple      # mm
    axes: tuple        # ellipsoid semi-axes; zcylinder (radius, radius, half length)
    activity: float
    body: bool = False  # part of the body outline (used for the scatter path)
    mu: float = -1.0    # attenuation coefficient (1/mm) inside the shape; < 0: that of the enclosing body

    def volume(self):
        a, b, c = self.axes
        if self.kind == "ellipsoid":
            return 4.0 / 3.0 * math.pi * a * b * c
        return math.pi * a * b * 2.0 * c

    def bbox(self):
        return (np.array(self.centre) - np.array(self.axes), np.array(self.centre) + np.array(self.axes))

    def contains(self, p):
        q = (p - np.array(self.centre)[:, None]) / np.array(self.axes)[:, None]
        if self.kind == "ellipsoid":
            return (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) <= 1.0
        return ((q[0] * q[0] + q[1] * q[1]) <= 1.0) & (np.abs(q[2]) <= 1.0)


@dataclass(frozen=True)
class Scanner:
    radius_mm: float
    axial_len_mm: float
    max_axial_angle_deg: float = 90.0
    tof_fwhm_ps: float = 300.0
    blur_fwhm_mm: float = 0.4


@dataclass(frozen=True)
class Workload:
    name: str
    scanner: Scanner
    shapes: tuple
    grid: tuple               # (nx, ny, nz, voxel_mm), centred on the origin
    scatter_fraction: float = 0.0
    max_scatter_deg: float = 60.0
    extra: dict = field(default_factory=dict)


def tiny_workload():
    shapes = (
        Shape("zcylinder", (0.0, 0.0, 0.0), (50.0, 50.0, 80.0), 1.0, body=True),
        Shape("ellipsoid", (20.0, 0.0, 20.0), (8.0, 8.0, 8.0), 4.0),
        Shape("ellipsoid", (-20.0, 10.0, -30.0), (8.0, 8.0, 8.0), 4.0),
    )
    return Workload("tiny", Scanner(150.0, 200.0), shapes, (32, 32, 48, 4.0))


def fullbody_workload():
    e = lambda c, a, act, body=False: Shape("ellipsoid", c, a, act, body)  # noqa: E731
    shapes = [
        e((0, 0, 150), (170, 110, 330), 1.0, True),     # trunk
        e((0, 0, 510), (55, 55, 50), 1.0, True),        # neck
        e((0, 0, 650), (80, 95, 110), 1.0, True),       # head
        e((90, 0, -600), (75, 75, 430), 1.0, True),     # left leg
        e((-90, 0, -600), (75, 75, 430), 1.0, True),    # right leg
        Shape("ellipsoid", (85, 0, 300), (60, 70, 120), 0.3, False, MU_LUNG),    # lungs
        Shape("ellipsoid", (-85, 0, 300), (60, 70, 120), 0.3, False, MU_LUNG),
        e((-70, 0, 140), (90, 70, 70), 2.0),            # liver
        e((30, -20, 260), (50, 45, 55), 3.0),           # heart
        e((0, -30, -140), (35, 30, 30), 8.0),           # bladder
        e((0, 0, 660), (65, 80, 75), 2.5),              # brain
    ]
    # ten lesions, 10-20 mm diameter, 4-8x: neck, subclavicular, axillary,
    # lung, liver, abdomen, inguinal, thigh, knee, calf
    # (every lesion lies inside the body outline, away from the organ edges)
    lesions = [((20, 10, 520), 5.0, 6.0), ((-60, -40, 400), 6.0, 5.0), ((-150, 0, 250), 7.0, 4.0),
               ((95, 10, 290), 8.0, 6.0), ((-60, 20, 120), 10.0, 4.0), ((40, -40, 20), 9.0, 5.0),
               ((60, -30, -120), 5.0, 8.0), ((90, 0, -400), 6.0, 7.0), ((-90, -20, -640), 7.5, 6.0),
               ((90, 10, -850), 5.5, 8.0)]
    for c, r, act in lesions:
        shapes.append(e(c, (r, r, r), act))
    return Workload("fullbody", Scanner(400.0, 2400.0, 45.0), tuple(shapes), (150, 150, 600, 4.0),
                    scatter_fraction=0.33, extra={"lesions": lesions})


def fullbody_background_workload():
    """The full-body phantom without its lesions: the background data set of the
    contrast recovery coefficient, reconstructed independently of the data with
    lesions (Sec. 2.6)."""
    w = fullbody_workload()
    return replace(w, name="fullbody_background", shapes=w.shapes[:-len(w.extra["lesions"])])


def smallfov_workload():
    shapes = (
        Shape("zcylinder", (0.0, 0.0, 0.0), (14.0, 14.0, 30.0), 1.0, body=True),
        Shape("ellipsoid", (4.0, 2.0, 8.0), (3.0, 3.0, 3.0), 5.0),
        Shape("ellipsoid", (-5.0, -3.0, -10.0), (2.0, 2.0, 2.0), 6.0),
    )
    return Workload("smallfov", Scanner(60.0, 100.0), shapes, (128, 128, 128, 0.5))


WORKLOADS = {"tiny": tiny_workload, "fullbody": fullbody_workload, "fullbody_background": fullbody_background_workload,
             "smallfov": smallfov_workload}


def grid_of(w):
    """(nx, ny, nz, v, v, v, ox, oy, oz) of a workload's centred image grid."""
    if isinstance(w, str):
        w = WORKLOADS[w]()
    nx, ny, nz, v = w.grid
    return (nx, ny, nz, v, v, v, -0.5 * nx * v, -0.5 * ny * v, -0.5 * nz * v)


# Nine body regions of the full-body workload (Sec. 2.5), as core slice ranges
# [z_lo, z_hi) of its 150x150x600 grid of 4 mm.  Eight cores of 50 slices
# (200 mm, the core length of the paper's regions 2-9) run from the feet
# (slice 42, z = -1032 mm) up the body; the ninth takes the 68 slices up to
# z = 840 mm, above the head.  With the 6 mm shell the regions take 6.7 M to
# 34.4 M of the 146 M events each, and slabs widened by 3 sigma + shell span
# 82 to 100 slices; the 0.09% of events whose TOF point lies below the feet or
# above the head join no region.
FULLBODY_REGIONS = [(42, 92), (92, 142), (142, 192), (192, 242), (242, 292), (292, 342), (342, 392),
                    (392, 442), (442, 510)]


# ----------------------------------------------------------------- sampling

def _rng(seed, stream, chunk):
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(stream), int(chunk)])))


def _unit_vectors(rng, n):
    cz = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([sz * np.cos(phi), sz * np.sin(phi), cz])


def _uniform_in(shape, rng, n):
    a = np.array(shape.axes)[:, None]
    c = np.array(shape.centre, dtype=np.float64)[:, None]
    if shape.kind == "ellipsoid":
        d = _unit_vectors(rng, n)
        r = np.cbrt(rng.uniform(0.0, 1.0, n))
        return c + a * d * r
    r = np.sqrt(rng.uniform(0.0, 1.0, n))
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    z = rng.uniform(-1.0, 1.0, n)
    return c + a * np.stack([r * np.cos(phi), r * np.sin(phi), z])


def _overlaps(shapes):
    """For each shape, the later shapes whose bounding box meets its own."""
    out = []
    for i, s in enumerate(shapes):
        lo, hi = s.bbox()
        later = []
        for t in shapes[i + 1:]:
            lo2, hi2 = t.bbox()
            if np.all(lo <= hi2) and np.all(lo2 <= hi):
                later.append(t)
        out.append(later)
    return out


def sample_emissions(shapes, rng, n):
    """n points with density proportional to the painter-ordered activity.

    A shape is picked with probability proportional to activity x volume, a
    point is drawn uniformly inside it, and kept only when no later shape
    (which would paint over it) contains it; the kept points then have the
    density of the topmost shape's activity.
    """
    weights = np.array([s.activity * s.volume() for s in shapes])
    prob = weights / weights.sum()
    later = _overlaps(shapes)
    out = np.empty((3, 0))
    while out.shape[1] < n:
        m = int(1.3 * (n - out.shape[1])) + 64
        pick = rng.choice(len(shapes), size=m, p=prob)
        pts = np.empty((3, m))
        keep = np.ones(m, bool)
        for i, s in enumerate(shapes):
            sel = np.nonzero(pick == i)[0]
            if sel.size == 0:
                continue
            p = _uniform_in(s, rng, sel.size)
            ok = np.ones(sel.size, bool)
            for t in later[i]:
                ok &= ~t.contains(p)
            pts[:, sel] = p
            keep[sel] = ok
        out = np.concatenate([out, pts[:, keep]], axis=1)
    return out[:, :n]


def _cylinder_exit(p, v, R):
    """Distance t >= 0 from p (inside radius R) along v to the lateral surface."""
    a = v[0] * v[0] + v[1] * v[1]
    b = 2.0 * (p[0] * v[0] + p[1] * v[1])
    c = p[0] * p[0] + p[1] * p[1] - R * R
    disc = np.maximum(b * b - 4.0 * a * c, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (-b + np.sqrt(disc)) / (2.0 * a)
    return np.where(a > 1e-12, t, np.inf)


def _ellipsoid_exit(p, v, shape):
    """Distance from p (inside) along v to the surface of an ellipsoid."""
    a = np.array(shape.axes)[:, None]
    c = np.array(shape.centre, dtype=np.float64)[:, None]
    q = (p - c) / a
    w = v / a
    A = np.sum(w * w, axis=0)
    B = 2.0 * np.sum(q * w, axis=0)
    Cc = np.sum(q * q, axis=0) - 1.0
    disc = np.maximum(B * B - 4.0 * A * Cc, 0.0)
    return np.maximum((-B + np.sqrt(disc)) / (2.0 * A), 0.0)


def _body_exit(p, v, shapes):
    """In-body path length from p along v: exit of the body part holding p."""
    t = np.zeros(p.shape[1])
    found = np.zeros(p.shape[1], bool)
    for s in shapes:
        if not s.body:
            continue
        inside = s.contains(p) & ~found
        if not inside.any():
            continue
        if s.kind == "ellipsoid":
            t[inside] = _ellipsoid_exit(p[:, inside], v[:, inside], s)
        else:
            t[inside] = np.minimum(_cylinder_exit(p[:, inside] - np.array(s.centre)[:, None], v[:, inside],
                                                  s.axes[0]), 1e9)
        found |= inside
    return t


def _deflect(v, rng, max_deg):
    """Rotate unit vectors v by a polar angle ~ U(0, max) and uniform azimuth."""
    n = v.shape[1]
    theta = rng.uniform(0.0, math.radians(max_deg), n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    helper = np.where(np.abs(v[2]) < 0.9, np.array([[0.0], [0.0], [1.0]]), np.array([[1.0], [0.0], [0.0]]))
    e1 = np.cross(v.T, helper.T).T
    e1 /= np.linalg.norm(e1, axis=0)
    e2 = np.cross(v.T, e1.T).T
    return np.cos(theta) * v + np.sin(theta) * (np.cos(phi) * e1 + np.sin(phi) * e2)


def _events_chunk(w, rng, n):
    """n accepted events of workload w as a (7, n) float32 array."""
    sc = w.scanner
    R, half = sc.radius_mm, 0.5 * sc.axial_len_mm
    tan_cut = math.tan(math.radians(sc.max_axial_angle_deg)) if sc.max_axial_angle_deg < 90.0 else np.inf
    blur_sigma = sc.blur_fwhm_mm / FWHM_PER_SIGMA
    timing_sigma_ps = sc.tof_fwhm_ps / FWHM_PER_SIGMA
    parts, have = [], 0
    while have < n:
        m = int(1.6 * (n - have)) + 256
        e = sample_emissions(w.shapes, rng, m)
        v = _unit_vectors(rng, m)
        o1, o2 = e.copy(), e.copy()       # photon 1 goes along +v, photon 2 along -v
        v1, v2 = v.copy(), -v
        l1 = np.zeros(m)
        l2 = np.zeros(m)
        if w.scatter_fraction > 0.0:
            scat = rng.uniform(0.0, 1.0, m) < w.scatter_fraction
            which = rng.uniform(0.0, 1.0, m) < 0.5          # True: photon 1 scatters
            vs = np.where(which, v1, v2)
            t_in = _body_exit(e, vs, w.shapes)
            s = rng.uniform(0.0, 1.0, m) * t_in
            q = e + vs * s
            vn = _deflect(vs, rng, w.max_scatter_deg)
            s1 = scat & which
            s2 = scat & ~which
            o1[:, s1], v1[:, s1], l1[s1] = q[:, s1], vn[:, s1], s[s1]
            o2[:, s2], v2[:, s2], l2[s2] = q[:, s2], vn[:, s2], s[s2]
        t1 = _cylinder_exit(o1, v1, R)
        t2 = _cylinder_exit(o2, v2, R)
        p1 = o1 + v1 * t1
        p2 = o2 + v2 * t2
        l1 += t1
        l2 += t2
        ok = np.isfinite(t1) & np.isfinite(t2) & (np.abs(p1[2]) <= half) & (np.abs(p2[2]) <= half)
        if np.isfinite(tan_cut):
            dxy = np.hypot(p1[0] - p2[0], p1[1] - p2[1])
            ok &= np.abs(p1[2] - p2[2]) < tan_cut * dxy
        k = int(ok.sum())
        p1 = p1[:, ok] + rng.normal(0.0, blur_sigma, (3, k))
        p2 = p2[:, ok] + rng.normal(0.0, blur_sigma, (3, k))
        dt_ps = (l2[ok] - l1[ok]) / C_MM_PER_PS + rng.normal(0.0, timing_sigma_ps, k)  # t2 - t1
        d = 0.5 * C_MM_PER_PS * dt_ps
        parts.append(np.concatenate([p1, p2, d[None, :]]).astype(np.float32))
        have += k
    return np.concatenate(parts, axis=1)[:, :n]


def _lors_chunk(sc, rng, n):
    """n kinematically uniform LORs meeting the lateral surface at |z| <= L/2."""
    R, half = sc.radius_mm, 0.5 * sc.axial_len_mm
    tan_cut = math.tan(math.radians(sc.max_axial_angle_deg)) if sc.max_axial_angle_deg < 90.0 else np.inf
    rho = math.sqrt(R * R + half * half)
    parts, have = [], 0
    while have < n:
        m = int(2.5 * (n - have)) + 256
        u = _unit_vectors(rng, m)
        helper = np.where(np.abs(u[2]) < 0.9, np.array([[0.0], [0.0], [1.0]]), np.array([[1.0], [0.0], [0.0]]))
        e1 = np.cross(u.T, helper.T).T
        e1 /= np.linalg.norm(e1, axis=0)
        e2 = np.cross(u.T, e1.T).T
        r = rho * np.sqrt(rng.uniform(0.0, 1.0, m))
        phi = rng.uniform(0.0, 2.0 * math.pi, m)
        q = r * np.cos(phi) * e1 + r * np.sin(phi) * e2
        a = u[0] * u[0] + u[1] * u[1]
        b = 2.0 * (q[0] * u[0] + q[1] * u[1])
        c = q[0] * q[0] + q[1] * q[1] - R * R
        disc = b * b - 4.0 * a * c
        ok = (a > 1e-12) & (disc > 0.0)
        sq = np.sqrt(np.where(ok, disc, 0.0))
        aa = np.where(ok, a, 1.0)
        ta = (-b - sq) / (2.0 * aa)
        tb = (-b + sq) / (2.0 * aa)
        p1 = q + u * tb
        p2 = q + u * ta
        ok &= (np.abs(p1[2]) <= half) & (np.abs(p2[2]) <= half)
        if np.isfinite(tan_cut):
            dxy = np.hypot(p1[0] - p2[0], p1[1] - p2[1])
            ok &= np.abs(p1[2] - p2[2]) < tan_cut * dxy
        parts.append(np.concatenate([p1[:, ok], p2[:, ok]]).astype(np.float32))
        have += int(ok.sum())
    return np.concatenate(parts, axis=1)[:, :n]


# ------------------------------------------------------------ parallel driver

def _fill(kind, w, seed, n, k, out):
    lo = k * CHUNK
    m = min(CHUNK, n - lo)
    if kind == "events":
        out[:, lo:lo + m] = _events_chunk(w, _rng(seed, 1, k), m)
    else:
        out[:, lo:lo + m] = _lors_chunk(w.scanner, _rng(seed, 2, k), m)


def _worker(args):
    kind, wname, seed, n, chunks, shm_name, rows = args
    w = WORKLOADS[wname]()
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        out = np.ndarray((rows, n), np.float32, buffer=shm.buf)
        for k in chunks:
            _fill(kind, w, seed, n, k, out)
        del out
    finally:
        shm.close()
    return 0


def _draw(kind, wname, n, seed, rows, workers, out=None):
    n = int(n)
    if out is None:
        out = np.empty((rows, n), np.float32)
    if n == 0:
        return out
    n_chunks = (n + CHUNK - 1) // CHUNK
    w = WORKLOADS[wname]()
    if workers is None:
        workers = min(os.cpu_count() or 1, n_chunks)
    if workers <= 1 or n_chunks == 1:
        for k in range(n_chunks):
            _fill(kind, w, seed, n, k, out)
        return out
    shm = shared_memory.SharedMemory(create=True, size=rows * n * 4)
    try:
        view = np.ndarray((rows, n), np.float32, buffer=shm.buf)
        jobs = [(kind, wname, seed, n, list(range(p, n_chunks, workers)), shm.name, rows) for p in range(workers)]
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_worker, jobs)
        out[...] = view
        del view
    finally:
        shm.close()
        shm.unlink()
    return out


def events(wname, n, seed, workers=None, out=None):
    """(7, n) float32 SoA events x1,y1,z1,x2,y2,z2,d of a named workload."""
    return _draw("events", wname, n, seed, 7, workers, out)


def sensitivity_lors(wname, n, seed, workers=None, out=None):
    """(6, n) float32 SoA kinematically uniform LORs of a workload's scanner."""
    return _draw("lors", wname, n, seed, 6, workers, out)


# ------------------------------------------------------------------ packing

LATTICE_MM = 0.05


def pack_events(ev):
    """int16 endpoints on a 0.05 mm lattice plus an FP16 TOF offset.

    Returns an (n, 8) int16 array: x1, y1, z1, x2, y2, z2 as lattice counts,
    the FP16 bits of d, and a zero pad (16 bytes per event).
    """
    ev = np.asarray(ev)
    n = ev.shape[1]
    q = np.rint(ev[:6].astype(np.float64) / LATTICE_MM)
    if np.any(np.abs(q) > 32767):
        raise ValueError("endpoint outside the int16 lattice range (+-1638.35 mm)")
    rec = np.zeros((n, 8), np.int16)
    rec[:, :6] = q.T.astype(np.int16)
    rec[:, 6] = ev[6].astype(np.float16).view(np.int16)
    return rec


def phantom_image(wname, grid=None, oversample=2):
    """Activity phantom averaged over voxels, (nz, ny, nx), for reporting only."""
    w = WORKLOADS[wname]()
    nx, ny, nz, v, _, _, ox, oy, oz = grid if grid is not None else grid_of(w)
    img = np.zeros((nz, ny, nx))
    offs = (np.arange(oversample) + 0.5) / oversample
    for a in offs:
        for b in offs:
            for c in offs:
                zz, yy, xx = np.meshgrid(oz + (np.arange(nz) + a) * v, oy + (np.arange(ny) + b) * v,
                                         ox + (np.arange(nx) + c) * v, indexing="ij")
                p = np.stack([xx.ravel(), yy.ravel(), zz.ravel()])
                img += activity_at(w, p).reshape(nz, ny, nx)
    return img / oversample ** 3


def activity_at(w, points):
    """Activity of a workload's phantom at points (3, n) in mm (painter order: a
    later shape overrides an earlier one where they overlap)."""
    if isinstance(w, str):
        w = WORKLOADS[w]()
    p = np.asarray(points, np.float64).reshape(3, -1)
    act = np.zeros(p.shape[1])
    for sh in w.shapes:
        act[sh.contains(p)] = sh.activity
    return act


def mu_image(wname, grid=None):
    """Attenuation map (1/mm) at the voxel centres, flat x-fastest: MU_WATER inside
    the body outline, a shape's own mu where it sets one, 0 outside the body."""
    w = WORKLOADS[wname]()
    nx, ny, nz, v, _, _, ox, oy, oz = grid if grid is not None else grid_of(w)
    out = np.zeros(nz * ny * nx, np.float32)
    xs = ox + (np.arange(nx) + 0.5) * v
    ys = oy + (np.arange(ny) + 0.5) * v
    for z0 in range(0, nz, 16):
        z1 = min(nz, z0 + 16)
        zz, yy, xx = np.meshgrid(oz + (np.arange(z0, z1) + 0.5) * v, ys, xs, indexing="ij")
        p = np.stack([xx.ravel(), yy.ravel(), zz.ravel()])
        m = np.zeros(p.shape[1], np.float32)
        for s in w.shapes:
            if s.body:
                m[s.contains(p)] = MU_WATER
        for s in w.shapes:
            if s.mu >= 0:
                m[s.contains(p)] = s.mu
        out[z0 * ny * nx:z1 * ny * nx] = m
    return out
