"""Parity at the full benchmark size: 146 M full-body events on the 150 x 150 x 600
grid of 4 mm voxels, events resident on the device, in the launch and event order
that the benchmark times (the library's autotuned default).

The benchmark's own reconstruction is compared whole: the sensitivity image from
its 50 M LORs element by element, and the image after its three MLEM iterations
from the uniform start over every voxel, against the FP64 oracle run over all
146 M events (a few minutes on the host cores).

The other tests recompute sampled outputs one by one, which lets them cover the
projector variants, the region form and the sieve at this size without an oracle
reconstruction each.  One MLEM iteration (Sec. 2.4) from a seeded random
start image lam0 gives, at voxel j,

    lam1_j = lam0_j / s_j * sum_i a_ij w_i / p_i,      p_i = sum_k a_ik lam0_k,

and only events whose TOF window passes within half a voxel diagonal of the
centre of voxel j have a_ij > 0.  A conservative prefilter over all events (the
TOF point within 3 sigma plus a voxel diagonal of the centre, then the line's
distance and window position in FP64 with a 1 mm margin) finds them; the oracle
computes p_i and a_ij for those events exactly.  The sampled voxels are the
voxels of the TOF points of seeded random events, the ten lesion centres, and
voxels at every region core boundary and slab edge.

Properties that hold at any size are checked on the whole output:
sum_j s_j lambda_j = N_eff after every iteration, nonnegativity, N_eff against
an FP64 count of the events whose TOF window meets the grid, and the region
codes, offsets and member lists bit-exact against the oracle over all events.

lam0 takes values k/128 (k = 64..192), exact in BF16, so that the BF16-gather
run of the packed form is compared with the same p_i as the FP32 runs.
"""
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from gpu_common import SIGMA, geometry, grid_tuple, max_rel_above, rel_l2, workload_grid
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

pytestmark = pytest.mark.gpu

N_EVENTS = 146_000_000          # the full-body benchmark workload
SEED = 1708                     # the benchmark's event seed (rank 0)
N_LORS = 50_000_000             # the benchmark's sensitivity LORs (same seed)
N_ITER = 3                      # MLEM iterations of a benchmark step
K = 3.0
MARGIN_MM = 1.0                 # prefilter margin (covers the int16/FP16 packing error)
FULLBODY_REGIONS = synth.FULLBODY_REGIONS   # the benchmark's nine body regions
SHELL_MM = 6.0
CHUNK = 8_000_000
THREADS = min(16, os.cpu_count() or 1)   # numpy releases the GIL in the array work


def smooth_s(g):
    z = g.oz + (np.arange(g.nz) + 0.5) * g.vz
    y = g.oy + (np.arange(g.ny) + 0.5) * g.vy
    x = g.ox + (np.arange(g.nx) + 0.5) * g.vx
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    return (3000.0 * (1.2 + np.cos(zz / 700.0)) * (1.0 + 0.2 * np.cos(xx / 200.0) * np.cos(yy / 200.0))).ravel()


def tof_points(ev):
    """c = M + d u with u = (P1 - P2)/|P1 - P2| (FP32, chunked)."""
    n = ev.shape[1]
    c = np.empty((3, n), np.float32)
    for lo in range(0, n, CHUNK):
        hi = min(n, lo + CHUNK)
        p1 = ev[0:3, lo:hi]
        p2 = ev[3:6, lo:hi]
        u = p1 - p2
        u /= np.sqrt((u * u).sum(axis=0))
        c[:, lo:hi] = 0.5 * (p1 + p2) + ev[6, lo:hi] * u
    return c


def voxel_centre(g, j):
    iz, rem = divmod(int(j), g.ny * g.nx)
    iy, ix = divmod(rem, g.nx)
    return np.array([g.ox + (ix + 0.5) * g.vx, g.oy + (iy + 0.5) * g.vy, g.oz + (iz + 0.5) * g.vz])


def voxel_of(g, p):
    ix = int(math.floor((p[0] - g.ox) / g.vx))
    iy = int(math.floor((p[1] - g.oy) / g.vy))
    iz = int(math.floor((p[2] - g.oz) / g.vz))
    if not (0 <= ix < g.nx and 0 <= iy < g.ny and 0 <= iz < g.nz):
        return None
    return (iz * g.ny + iy) * g.nx + ix


def sample_voxels(g, ev, c, rng):
    """Voxels of random TOF points, the lesion centres, and voxels at each region
    core boundary and slab edge (x, y of a TOF point near that slice)."""
    vox = []
    pick = rng.choice(ev.shape[1], 48, replace=False)
    for i in pick:
        vox.append(voxel_of(g, c[:, i].astype(np.float64)))
    for centre, _, _ in synth.WORKLOADS["fullbody"]().extra["lesions"]:
        vox.append(voxel_of(g, np.asarray(centre, np.float64)))
    slabs = oracle.region_slabs(g, FULLBODY_REGIONS, K * SIGMA + SHELL_MM)
    slices = set()
    for lo, _ in FULLBODY_REGIONS[1:]:
        slices.update((lo - 1, lo))
    for lo, hi in slabs:
        slices.update((lo, hi - 1))
    sub = rng.choice(ev.shape[1], min(ev.shape[1], 2_000_000), replace=False)
    cz = c[2, sub].astype(np.float64)
    for k in sorted(slices):
        zc = g.oz + (k + 0.5) * g.vz
        near = np.nonzero(np.abs(cz - zc) < 0.5 * g.vz)[0]
        if near.size:
            p = c[:, sub[near[0]]].astype(np.float64)
            p[2] = zc
            vox.append(voxel_of(g, p))
    vox = [v for v in vox if v is not None]
    return np.array(sorted(set(vox)), np.int64)


def prefilter(g, ev, c, vox):
    """Per sampled voxel, the events whose TOF window can reach it (a superset)."""
    H = 0.5 * math.sqrt(g.vx ** 2 + g.vy ** 2 + g.vz ** 2)
    along = K * SIGMA + H + MARGIN_MM
    perp = H + MARGIN_MM
    reach = math.hypot(along, perp)
    dz = int(math.ceil(reach / g.vz)) + 1
    iz = np.clip(np.floor((c[2] - g.oz) / g.vz), -2, g.nz + 1).astype(np.int16)
    order = np.argsort(iz, kind="stable")
    iz_sorted = iz[order]
    cs = c[:, order]

    def one(j):
        v = voxel_centre(g, j)
        kz = int(math.floor((v[2] - g.oz) / g.vz))
        a = np.searchsorted(iz_sorted, kz - dz, "left")
        b = np.searchsorted(iz_sorted, kz + dz, "right")
        blk = cs[:, a:b]
        d2 = (blk[0] - v[0]) ** 2 + (blk[1] - v[1]) ** 2 + (blk[2] - v[2]) ** 2
        idx = order[a:b][d2 <= (reach + 0.5) ** 2]
        e = ev[:, idx].astype(np.float64)
        u = e[0:3] - e[3:6]
        u /= np.sqrt((u * u).sum(axis=0))
        w = v[:, None] - (0.5 * (e[0:3] + e[3:6]) + e[6] * u)
        s_al = (w * u).sum(axis=0)
        p2 = (w * w).sum(axis=0) - s_al ** 2
        keep = (np.abs(s_al) <= along) & (p2 <= perp ** 2)
        return np.sort(idx[keep])

    with ThreadPoolExecutor(THREADS) as pool:
        return list(pool.map(one, vox))


def window_meets_grid(g, ev):
    """FP64 count of events whose TOF window [d - K sigma, d + K sigma] meets the
    grid box in a piece longer than 1e-3 mm (sure), and of those within 1e-3 mm
    of touching it (either way)."""
    lo = np.array([g.ox, g.oy, g.oz])[:, None]
    hi = lo + np.array([g.nx * g.vx, g.ny * g.vy, g.nz * g.vz])[:, None]
    half = K * SIGMA

    def one(a):
        e = ev[:, a:a + CHUNK].astype(np.float64)
        u = e[0:3] - e[3:6]
        u /= np.sqrt((u * u).sum(axis=0))
        c = 0.5 * (e[0:3] + e[3:6]) + e[6] * u
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (lo - c) / u
            t2 = (hi - c) / u
        inside = (c >= lo) & (c < hi)
        tmin = np.where(u == 0, np.where(inside, -np.inf, np.inf), np.minimum(t1, t2))
        tmax = np.where(u == 0, np.where(inside, np.inf, -np.inf), np.maximum(t1, t2))
        L = np.minimum(tmax.min(axis=0), half) - np.maximum(tmin.max(axis=0), -half)
        return int(np.count_nonzero(L > 1e-3)), int(np.count_nonzero(np.abs(L) <= 1e-3))

    with ThreadPoolExecutor(THREADS) as pool:
        parts = list(pool.map(one, range(0, ev.shape[1], CHUNK)))
    return sum(p[0] for p in parts), sum(p[1] for p in parts)


def oracle_lam1(g, events64, cand, vox, lam0, s, lut=None, weights=None):
    """lam1 at the sampled voxels from the candidate events (FP64 oracle)."""
    union = np.unique(np.concatenate(cand))
    e = events64(union)
    lam = lam0.astype(np.float64)
    if lut:
        p = oracle.forward_lut(g, e, lam, lut, SIGMA)
    else:
        p = oracle.forward(g, e, lam, SIGMA)
    w = np.ones(union.size) if weights is None else weights[union]
    r = np.where(p > 0, w / np.where(p > 0, p, 1.0), 0.0)
    C = oracle.backproject_lut(g, e, r, lut, SIGMA) if lut else oracle.backproject(g, e, r, SIGMA)
    return lam[vox] * C[vox] / s[vox]


def oracle_region_lam1(g, ev, s, vox, cand, codes, offs, idx, slabs):
    """Region form after one iteration from each region's uniform start, at every
    (sampled voxel, slab containing it): positions in the concatenated slab
    images and the FP64 values.  Region r reconstructs its members (weight 1/2
    for events fed to two regions) on its slab grid; lam0_r = sum w / sum_slab s."""
    w_all = np.where((codes & 0x80) != 0, 0.5, 1.0)
    s3 = np.asarray(s, np.float64).reshape(g.nz, g.ny, g.nx)
    iz_vox = vox // (g.ny * g.nx)
    pos, ref = [], []
    base = 0
    for r, (lo, hi) in enumerate(slabs):
        members = idx[offs[r]:offs[r + 1]]
        s_slab = s3[lo:hi].reshape(-1)
        lam0_r = w_all[members].sum() / s_slab.sum()
        inside = np.nonzero((iz_vox >= lo) & (iz_vox < hi))[0]
        if inside.size:
            union = np.intersect1d(np.unique(np.concatenate([cand[k] for k in inside])), members)
            e = ev[:, union].astype(np.float64)
            g_r = oracle.slab_grid(g, lo, hi)
            p = lam0_r * oracle.forward(g_r, e, np.ones(s_slab.size), SIGMA)
            rr = np.where(p > 0, w_all[union] / np.where(p > 0, p, 1.0), 0.0)
            C = oracle.backproject(g_r, e, rr, SIGMA)
            jl = vox[inside] - lo * g.ny * g.nx
            ref.append(lam0_r * C[jl] / s_slab[jl])
            pos.append(base + jl)
        base += s_slab.size
    return np.concatenate(pos), np.concatenate(ref)


def check_voxels(got, ref, label):
    got = np.asarray(got, np.float64)
    big = ref >= 0.01 * ref.max()
    rel = np.abs(got[big] - ref[big]) / ref[big]
    l2 = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    print(f"\n{label}: {ref.size} sampled voxels, max rel {rel.max():.2e}, median rel "
          f"{np.median(rel):.2e}, rel L2 {l2:.2e}")
    assert rel.max() <= 1e-3
    assert l2 <= 1e-4
    if (~big).any():
        assert np.abs(got[~big] - ref[~big]).max() <= 1e-5 * ref.max()


@pytest.fixture(scope="module")
def full():
    g = workload_grid("fullbody")
    ev = synth.events("fullbody", N_EVENTS, SEED)
    rng = np.random.default_rng(1706_07075)
    lam0 = (rng.integers(64, 193, g.n_vox) / 128.0).astype(np.float32)
    s = smooth_s(g)
    c = tof_points(ev)
    vox = sample_voxels(g, ev, c, rng)
    cand = prefilter(g, ev, c, vox)
    del c
    return {"g": g, "ev": ev, "lam0": lam0, "s": s, "vox": vox, "cand": cand}


@pytest.fixture(scope="module")
def ctx(full):
    g = full["g"]
    with B.Context(geometry("fullbody"), grid_tuple(g), 300.0) as c:
        c.set_sensitivity(full["s"])
        c.load_events(B.make_events(full["ev"]))
        yield c


def events64_of(ev):
    return lambda idx: ev[:, idx].astype(np.float64)


def test_fullsize_candidates_cover_every_sampled_voxel(full):
    # the prefilter found events for every sampled voxel (the dense body gives
    # hundreds of TOF windows per voxel)
    counts = np.array([c.size for c in full["cand"]])
    print(f"\n{counts.size} sampled voxels, candidate events per voxel: min {counts.min()}, "
          f"median {int(np.median(counts))}, max {counts.max()}")
    assert counts.size >= 60
    assert np.median(counts) >= 100


def test_fullsize_exact_projector(full, ctx):
    g, lam0, s, vox = full["g"], full["lam0"], full["s"], full["vox"]
    img = np.zeros(g.n_vox, np.float32)
    cons = np.zeros((1, 2))
    ctx.mlem(None, 1, lam0, img, cons)
    ref = oracle_lam1(g, events64_of(full["ev"]), full["cand"], vox, lam0, s)
    check_voxels(img[vox], ref, "exact projector, 1 iteration, 146 M events")
    # properties over the whole image: nonnegative, finite, count conservation,
    # and N_eff equal to the FP64 count of TOF windows that meet the grid
    assert np.isfinite(img).all() and img.min() >= 0.0
    sure, maybe = window_meets_grid(g, full["ev"])
    print(f"N_eff {cons[0, 0]:.0f}; FP64 windows meeting the grid {sure} (+{maybe} within 1e-3 mm)")
    assert sure <= cons[0, 0] <= sure + maybe
    assert cons[0, 1] == pytest.approx(cons[0, 0], rel=1e-5)
    # the benchmark's step: three iterations, conservation after each
    img3 = np.zeros(g.n_vox, np.float32)
    cons3 = np.zeros((3, 2))
    ctx.mlem(None, 3, lam0, img3, cons3)
    assert np.isfinite(img3).all() and img3.min() >= 0.0
    for k in range(3):
        assert cons3[k, 0] == cons[0, 0]
        assert cons3[k, 1] == pytest.approx(cons3[k, 0], rel=1e-5)


def test_fullsize_sampled_projector(full):
    # the paper's 32-sample projector over the events none of whose samples lies
    # within oracle.LUT_EPS_VOXELS of a voxel plane (the oracle decides voxels in
    # FP64, the kernel in FP32; they can differ only nearer a plane than that)
    g, lam0, s, vox, ev = full["g"], full["lam0"], full["s"], full["vox"], full["ev"]
    n = ev.shape[1]
    keep = np.empty(n, bool)
    for a in range(0, n, CHUNK):
        keep[a:a + CHUNK] = oracle.lut_ambiguous(g, ev[:, a:a + CHUNK].astype(np.float64), 32, SIGMA) == 0
    sub = np.ascontiguousarray(ev[:, keep])
    print(f"\nsampled projector: {sub.shape[1]} of {n} events have no sample within "
          f"{oracle.LUT_EPS_VOXELS} voxel of a plane")
    img = np.zeros(g.n_vox, np.float32)
    cons = np.zeros((1, 2))
    with B.Context(geometry("fullbody"), grid_tuple(g), 300.0) as c:
        c.set_sensitivity(s)
        c.load_events(B.make_events(sub))
        c.set_projector(B.PROJ_SAMPLED, 32)
        c.mlem(None, 1, lam0, img, cons)
    del sub
    cand = [cj[keep[cj]] for cj in full["cand"]]
    ref = oracle_lam1(g, events64_of(ev), cand, vox, lam0, s, lut=32)
    check_voxels(img[vox], ref, "sampled 32-point projector, 1 iteration, 146 M events")
    assert np.isfinite(img).all() and img.min() >= 0.0
    assert cons[0, 1] == pytest.approx(cons[0, 0], rel=1e-5)


def test_fullsize_packed_bf16_gather(full):
    g, lam0, s, vox = full["g"], full["lam0"], full["s"], full["vox"]
    rec = synth.pack_events(full["ev"])

    def dequantized(idx):
        r = rec[idx]
        q = r[:, :6].astype(np.float64).T * synth.LATTICE_MM
        d = r[:, 6].view(np.float16).astype(np.float64)
        return np.concatenate([q, d[None, :]])

    img = np.zeros(g.n_vox, np.float32)
    cons = np.zeros((1, 2))
    with B.Context(geometry("fullbody"), grid_tuple(g), 300.0) as c:
        c.set_sensitivity(s)
        c.load_events(B.make_events(rec, packed=True, lattice_mm=synth.LATTICE_MM))
        c.set_gather_bf16(1)
        c.mlem(None, 1, lam0, img, cons)
    ref = oracle_lam1(g, dequantized, full["cand"], vox, lam0, s)
    check_voxels(img[vox], ref, "packed int16/FP16 events, BF16 gather, 1 iteration, 146 M events")
    assert cons[0, 1] == pytest.approx(cons[0, 0], rel=1e-5)


def test_fullsize_osem_subset_counts(full, ctx):
    # OSEM with 5 subsets (consecutive blocks of the list) at full size.  The first
    # sub-iteration starts from lam0 > 0, so its N_eff equals the FP64 count of its
    # block's TOF windows that meet the grid.  A voxel that one block does not reach
    # gets lambda = 0 and keeps it (multiplicative update), so later blocks lose the
    # events whose every voxel some earlier block missed: a few 1e-5 of a block per
    # sub-iteration on this workload (measured 0.7, 3.0, 6.0, 9.4e-5 for blocks 1-4),
    # bounded here by 1e-3.  sum s lambda = B N_eff after each sub-iteration.
    g, lam0, ev = full["g"], full["lam0"], full["ev"]
    B_SUB = 5
    n = ev.shape[1]
    img = np.zeros(g.n_vox, np.float32)
    cons = np.zeros((B_SUB, 2))
    ctx.set_subsets(B_SUB)
    try:
        ctx.mlem(None, 1, lam0, img, cons)
    finally:
        ctx.set_subsets(1)
    assert np.isfinite(img).all() and img.min() >= 0.0
    for b in range(B_SUB):
        lo, hi = b * n // B_SUB, (b + 1) * n // B_SUB
        sure, maybe = window_meets_grid(g, ev[:, lo:hi])
        print(f"\nsubset {b}: N_eff {cons[b, 0]:.0f}, FP64 windows meeting the grid {sure} (+{maybe})")
        if b == 0:
            assert sure <= cons[b, 0] <= sure + maybe
        else:
            assert sure - 1e-3 * (hi - lo) <= cons[b, 0] <= sure + maybe
        assert cons[b, 1] == pytest.approx(B_SUB * cons[b, 0], rel=1e-5)


def test_fullsize_preprocess_sampled_events(full, ctx):
    # attenuation weights and TOF scatter rejection over all 146 M resident events;
    # the oracle recomputes every 1009th event
    from test_gpu_preprocess import Z95, check_against_oracle
    g, ev = full["g"], full["ev"]
    mu = synth.mu_image("fullbody")
    n = ev.shape[1]
    w = np.zeros(n, np.float32)
    keep = np.zeros(n, np.uint8)
    kept = ctx.preprocess(None, mu, Z95, 0, w, keep)
    assert kept == int(keep.sum())
    print(f"\npre-processing, 146 M events: {kept / n:.4f} kept")
    pick = np.arange(0, n, 1009)
    check_against_oracle(g, np.ascontiguousarray(ev[:, pick]), mu, w[pick], keep[pick], int(keep[pick].sum()))


def test_fullsize_median_sieve(full, ctx):
    # one iteration with the median sieve of Sec. 2.4 at full size: the filtered
    # image at a voxel is the 3x3x3 median of lam1, which the oracle recomputes from
    # lam1 at the 27 neighbours (each from its own prefiltered events)
    g, lam0, s, ev = full["g"], full["lam0"], full["s"], full["ev"]
    plane = g.ny * g.nx
    centres = []
    for j in full["vox"]:
        iz, rem = divmod(int(j), plane)
        iy, ix = divmod(rem, g.nx)
        if 0 < ix < g.nx - 1 and 0 < iy < g.ny - 1 and 0 < iz < g.nz - 1:
            centres.append(int(j))
    centres = np.array(centres[:16], np.int64)
    offs = np.array([dz * plane + dy * g.nx + dx for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
    nb = (centres[:, None] + offs[None, :]).ravel()
    c = tof_points(ev)
    cand = prefilter(g, ev, c, nb)
    del c
    lam1_nb = oracle_lam1(g, events64_of(ev), cand, nb, lam0, s).reshape(centres.size, 27)
    ref = np.array([oracle.median3_at(row.reshape(3, 3, 3), (3, 3, 3), [13])[0] for row in lam1_nb])
    img = np.zeros(g.n_vox, np.float32)
    ctx.set_median_filter(1)
    try:
        ctx.mlem(None, 1, lam0, img)
    finally:
        ctx.set_median_filter(0)
    check_voxels(img[centres], ref, "median sieve after 1 iteration, 146 M events")
    assert np.isfinite(img).all() and img.min() >= 0.0


@pytest.fixture(scope="module")
def regions_ref(full):
    """Oracle region codes over all events (FP64, chunked), members and offsets."""
    g, ev = full["g"], full["ev"]
    zb = oracle.region_bounds(g, FULLBODY_REGIONS)
    codes = np.empty(ev.shape[1], np.uint8)
    for a in range(0, ev.shape[1], CHUNK):
        codes[a:a + CHUNK] = oracle.region_codes(ev[:, a:a + CHUNK], zb, SHELL_MM)
    offs, idx = oracle.region_members(codes, len(FULLBODY_REGIONS))
    return codes, offs, idx


def test_fullsize_region_split_bitexact(full, ctx, regions_ref):
    codes_ref, offs_ref, idx_ref = regions_ref
    n = full["ev"].shape[1]
    codes = np.zeros(n, np.uint8)
    offs = np.zeros(len(FULLBODY_REGIONS) + 1, np.int64)
    ctx.split_regions(None, FULLBODY_REGIONS, 0.0, SHELL_MM, codes, offs, None)
    idx = np.zeros(int(offs[-1]), np.int32)
    ctx.split_regions(None, FULLBODY_REGIONS, 0.0, SHELL_MM, None, None, idx)
    assert np.array_equal(codes, codes_ref)
    assert np.array_equal(offs, offs_ref)
    assert np.array_equal(idx, idx_ref)
    counts = np.diff(offs)
    print(f"\nregion event counts (M): {np.round(counts / 1e6, 1).tolist()}")
    assert counts.min() > 0


def test_fullsize_region_mlem(full, ctx, regions_ref):
    # the nine-region form as the benchmark runs it (all regions in one launch per
    # iteration, margin 3 sigma + shell); per-region uniform start
    g, s, vox, cand, ev = full["g"], full["s"], full["vox"], full["cand"], full["ev"]
    codes, offs, idx = regions_ref
    margin = K * SIGMA + SHELL_MM
    slabs = oracle.region_slabs(g, FULLBODY_REGIONS, margin)
    nslab = ctx.region_slab_voxels(FULLBODY_REGIONS, margin)
    assert nslab == sum((hi - lo) * g.ny * g.nx for lo, hi in slabs)
    img = np.zeros(g.n_vox, np.float32)
    slab_img = np.zeros(nslab, np.float32)
    cons = np.zeros((1, len(slabs), 2))
    ctx.mlem_regions(None, FULLBODY_REGIONS, margin, SHELL_MM, 1, img, slab_img, cons)

    w_all = np.where((codes & 0x80) != 0, 0.5, 1.0)
    pos, ref = oracle_region_lam1(g, ev, s, vox, cand, codes, offs, idx, slabs)
    got = slab_img[pos]
    for r in range(len(slabs)):
        members = idx[offs[r]:offs[r + 1]]
        assert cons[0, r, 1] == pytest.approx(cons[0, r, 0], rel=1e-5)
        assert cons[0, r, 0] <= w_all[members].sum() + 1e-6
    check_voxels(got, ref, "nine TOF regions, 1 iteration, 146 M events")
    assert np.isfinite(img).all() and img.min() >= 0.0
    # the whole-body image is the sum of the slabs at their places
    starts = np.cumsum([0] + [(hi - lo) * g.ny * g.nx for lo, hi in slabs])
    parts = [slab_img[starts[r]:starts[r + 1]] for r in range(len(slabs))]
    assert np.allclose(img, oracle.stitch(g, slabs, parts), rtol=1e-6, atol=0.0)


@pytest.fixture(scope="module")
def whole(full):
    """The benchmark's reconstruction end to end: the sensitivity image from the
    50 M LORs, then three MLEM iterations from the uniform start over the resident
    146 M events in the autotuned default launch and event order (graphs on), on
    the GPU; and the same from the FP64 oracle over all events and LORs."""
    import time
    g, ev = full["g"], full["ev"]
    lors = synth.sensitivity_lors("fullbody", N_LORS, SEED)
    s_gpu = np.zeros(g.n_vox)
    img = np.zeros(g.n_vox, np.float32)
    cons = np.zeros((N_ITER, 2))
    with B.Context(geometry("fullbody"), grid_tuple(g), 300.0) as c:
        c.sensitivity(lors, s_gpu)
        c.load_events(B.make_events(ev))
        c.mlem(None, N_ITER, None, img, cons)
        launch = c.get_launch()
    t = time.perf_counter()
    s_ref = oracle.sensitivity(g, lors)
    t_sens = time.perf_counter() - t
    del lors
    evd = ev.astype(np.float64)
    t = time.perf_counter()
    lam_ref, hist = oracle.mlem(g, evd, s_ref, N_ITER, SIGMA)
    t_mlem = time.perf_counter() - t
    del evd
    print(f"\noracle over the whole workload: sensitivity {t_sens:.0f} s, {N_ITER} MLEM iterations "
          f"{t_mlem:.0f} s ({oracle.threads_used()} threads); GPU launch {launch}")
    return {"s": s_gpu, "s_ref": s_ref, "img": img, "cons": cons, "lam_ref": lam_ref, "hist": hist}


def test_fullsize_sensitivity_whole_image(full, whole):
    # every voxel of the full-body sensitivity image from the benchmark's 50 M LORs.
    # The GPU walks the LORs in FP64 (an FP32 walk on this 2.4 m grid moved up to
    # ~1 mm of chord between neighbouring voxels for lines nearly parallel to a
    # plane, 1.1e-2 of s_j at low-sensitivity voxels); an FP64 crossing is off by
    # ulp_64(|X - c|) / |u_k|, ~1e-5 mm only for |u_k| ~ 1e-8
    s, s_ref = whole["s"], whole["s_ref"]
    mask_diff = int(np.sum((s > 0) != (s_ref > 0)))
    l2 = rel_l2(s, s_ref)
    mx = max_rel_above(s, s_ref, 0.01)
    print(f"\nsensitivity, 50 M LORs, {s.size} voxels: rel L2 {l2:.2e}, max rel above 1% {mx:.2e}, "
          f"support differs at {mask_diff} voxels")
    assert mask_diff <= 1e-6 * s.size + 2
    assert l2 < 1e-9
    assert mx < 1e-6


def test_fullsize_mlem_whole_image(full, whole):
    # the benchmark's step, compared over the whole 150 x 150 x 600 image with the
    # plain gates: relative L2 <= 1e-4 and per-voxel relative error <= 1e-3 on the
    # voxels above 1% of the maximum
    img, lam_ref, cons, hist = whole["img"], whole["lam_ref"], whole["cons"], whole["hist"]
    l2 = rel_l2(img, lam_ref)
    mx = max_rel_above(img, lam_ref, 0.01)
    big = lam_ref > 0.01 * lam_ref.max()
    print(f"\n{N_ITER} MLEM iterations, 146 M events, whole image: rel L2 {l2:.2e}, max rel {mx:.2e} over "
          f"{int(big.sum())} voxels above 1% of max; N_eff {cons[:, 0].tolist()} vs oracle "
          f"{[h[0] for h in hist]}")
    rel = np.where(big, np.abs(img - lam_ref) / np.where(big, lam_ref, 1.0), 0.0)
    g = full["g"]
    for j in np.argsort(rel)[-5:][::-1]:
        iz, rem = divmod(int(j), g.ny * g.nx)
        iy, ix = divmod(rem, g.nx)
        print(f"  voxel ({ix},{iy},{iz}): GPU {img[j]:.6g}, oracle {lam_ref[j]:.6g}, rel {rel[j]:.2e}, "
              f"s {whole['s_ref'][j]:.6g}")
    assert np.isfinite(img).all() and img.min() >= 0.0
    assert l2 <= 1e-4
    assert mx <= 1e-3
    for k in range(N_ITER):
        # events whose window only touches the grid may fall either way in FP32
        assert abs(cons[k, 0] - hist[k][0]) <= 1e-6 * N_EVENTS
        assert cons[k, 1] == pytest.approx(cons[k, 0], rel=1e-5)
