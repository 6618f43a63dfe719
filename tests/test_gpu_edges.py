"""Edge cases of the GPU path: empty and one-event inputs, events that miss
the grid, rays lying in voxel planes, axis-parallel rays, the one-voxel grid,
zero iterations, launch configurations, device-resident buffers and call
order errors."""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import SIGMA, geometry, grid_tuple, max_rel_above, rel_l2, tiny_inputs, workload_grid
from oracle import Grid
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

pytestmark = pytest.mark.gpu


def odd_events():
    """Hand-built events on voxel planes, along axes, missing the grid, degenerate."""
    g = workload_grid("tiny")           # 32x32x48 voxels of 4 mm from (-64, -64, -96)
    rows = []
    xp = g.ox + 10 * g.vx               # the plane between columns 9 and 10
    rows.append([xp, -150.0, 3.0, xp, 150.0, -7.0, 12.0])        # in the x-plane
    rows.append([xp, g.oy + 7 * g.vy, -200.0, xp, g.oy + 7 * g.vy, 200.0, -30.0])  # on an edge
    rows.append([-150.0, 2.0, 2.0, 150.0, 2.0, 2.0, 5.0])        # along x
    rows.append([1.0, 1.0, -200.0, 1.0, 1.0, 200.0, 20.0])       # along z
    rows.append([-150.0, 90.0, 0.0, 150.0, 90.0, 0.0, 0.0])      # misses the grid (y = 90 > 64)
    rows.append([-150.0, 0.0, 0.0, 150.0, 0.0, 0.0, 500.0])      # TOF point far outside
    rows.append([5.0, 5.0, 5.0, 5.0, 5.0, 5.0, 0.0])             # P1 == P2
    rows.append([g.ox + 32 * g.vx, -150.0, 0.0, g.ox + 32 * g.vx, 150.0, 1.0, 0.0])  # on the upper face
    rows.append([g.ox, -150.0, 0.0, g.ox, 150.0, 1.0, 0.0])      # on the lower face
    rows.append([100.0, 80.0, 60.0, -90.0, -70.0, -50.0, 17.0])  # oblique through the corner region
    return np.array(rows, np.float32).T.copy()


@pytest.fixture(scope="module")
def ctx_tiny():
    ev, lors = tiny_inputs()
    g = workload_grid("tiny")
    ctx = B.Context(geometry("tiny"), grid_tuple(g), 300.0)
    ctx.sensitivity(lors)
    yield ctx, g
    ctx.close()


def test_odd_rays_forward_match_oracle(ctx_tiny):
    ctx, g = ctx_tiny
    ev = odd_events()
    rng = np.random.default_rng(5)
    lam = rng.uniform(0.5, 1.5, g.n_vox).astype(np.float32)
    p = np.zeros(ev.shape[1], np.float32)
    ctx.forward(B.make_events(ev), lam, p)
    p_ref = oracle.forward(g, ev.astype(np.float64), lam.astype(np.float64), SIGMA)
    assert np.allclose(p, p_ref, rtol=2e-5, atol=1e-7)
    assert p[4] == 0 and p[5] == 0 and p[6] == 0 and p[7] == 0
    assert p[0] > 0 and p[1] > 0 and p[8] > 0


def test_odd_rays_row_mass_is_one_inside(ctx_tiny):
    ctx, g = ctx_tiny
    ev = odd_events()
    p = np.zeros(ev.shape[1], np.float32)
    ctx.forward(B.make_events(ev), np.ones(g.n_vox, np.float32), p)
    # rows 2 and 3 have their whole +-3 sigma window inside the grid: unit mass
    assert p[2] == pytest.approx(1.0, abs=2e-6)
    assert p[3] == pytest.approx(1.0, abs=2e-6)


def test_empty_events_and_zero_iterations(ctx_tiny):
    ctx, g = ctx_tiny
    ev = np.zeros((7, 0), np.float32)
    img = np.full(g.n_vox, -1.0, np.float32)
    cons = np.full((2, 2), -1.0)
    ctx.mlem(B.make_events(ev), 2, None, img, cons)
    assert np.all(img == 0) and np.all(cons == 0)
    ev1, _ = tiny_inputs()
    init = np.random.default_rng(1).uniform(0, 1, g.n_vox).astype(np.float32)
    ctx.mlem(B.make_events(ev1[:, :1000].copy()), 0, init, img, None)
    assert np.array_equal(img, init)


def test_single_event_and_ragged_counts(ctx_tiny):
    ctx, g = ctx_tiny
    ev_all, _ = tiny_inputs()
    s = np.zeros(g.n_vox)
    for n in [1, 31, 33, 257, 4099]:
        ev = ev_all[:, :n].copy()
        img = np.zeros(g.n_vox, np.float32)
        cons = np.zeros((1, 2))
        ctx.mlem(B.make_events(ev), 1, None, img, cons)
        assert cons[0, 0] <= n and cons[0, 1] == pytest.approx(cons[0, 0], rel=1e-5)


def test_one_voxel_grid_closed_form():
    with B.Context((100.0, 100.0, 90.0), (1, 1, 1, 10.0, 10.0, 10.0, -5.0, -5.0, -5.0), 300.0) as ctx:
        ctx.set_sensitivity(np.array([12.5]))
        rng = np.random.default_rng(8)
        n = 37
        u = rng.normal(size=(n, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        ev = np.ascontiguousarray(np.concatenate([(50 * u).T, (-50 * u).T, rng.uniform(-3, 3, (1, n))]), np.float32)
        img = np.zeros(1, np.float32)
        ctx.mlem(B.make_events(ev), 1, None, img, None)
        assert img[0] == pytest.approx(n / 12.5, rel=1e-6)


@pytest.mark.parametrize("cfg", [(64, 0, 0, 0, 0), (128, 0, 0, 0, 0), (256, 4, 32, 0, 0), (128, 16, 256, 0, 0),
                                 (256, 1, 1024, 0, 0), (128, 0, 0, 64, 0), (64, 6, 64, 64, 0), (128, 0, 0, 8, 0),
                                 (256, 2, 64, 96, 0), (128, 0, 0, 0, 1), (64, 4, 64, 32, 1), (192, 0, 0, 0, 2),
                                 (128, 0, 0, 32, 2), (256, 4, 64, 0, 2), (128, 0, 0, 0, 2, 1), (192, 0, 0, 0, 0, 1),
                                 (256, 0, 0, 0, 1, 1), (128, 0, 0, 0, 3), (192, 0, 0, 0, 3, 1)])
def test_launch_configurations_agree(ctx_tiny, cfg):
    # (128, 0, 0, 8) caches fewer pieces than most walks have: those events walk twice.
    # The fifth field selects the piece-mass form: fitted tails (0), CUDA's erfcf tails
    # (1), the midpoint Taylor series (2); a sixth field of 1 the brick-layout
    # reductions.
    ctx, g = ctx_tiny
    ev, _ = tiny_inputs()
    ctx.set_launch(None)
    ref = np.zeros(g.n_vox, np.float32)
    ctx.set_launch(256, 0, 0, 0, 0)
    ctx.mlem(B.make_events(ev), 2, None, ref, None)
    ctx.set_launch(*cfg)
    img = np.zeros(g.n_vox, np.float32)
    ctx.mlem(None, 2, None, img, None)
    assert ctx.get_launch() == (cfg[0], cfg[1], cfg[2] if cfg[1] else 0, cfg[3], cfg[4], cfg[5] if len(cfg) > 5 else 0)
    ctx.set_launch(None)
    assert rel_l2(img, ref) < {0: 1e-6, 1: 2e-6, 2: 5e-6, 3: 5e-6}[cfg[4]]


def test_device_buffers_match_host_buffers(ctx_tiny):
    ctx, g = ctx_tiny
    ev, lors = tiny_inputs()
    img_h = np.zeros(g.n_vox, np.float32)
    ctx.mlem(B.make_events(ev), 2, None, img_h, None)
    evd = torch.from_numpy(ev).cuda()
    img_d = torch.zeros(g.n_vox, dtype=torch.float32, device="cuda")
    cons_d = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    ctx.mlem(B.make_events(evd), 2, None, img_d, cons_d)
    torch.cuda.synchronize()
    assert rel_l2(img_d.cpu().numpy(), img_h) < 1e-6
    s_d = torch.zeros(g.n_vox, dtype=torch.float64, device="cuda")
    ctx.sensitivity(torch.from_numpy(lors).cuda(), s_d)
    s_h = np.zeros(g.n_vox)
    ctx.sensitivity(lors, s_h)
    assert rel_l2(s_d.cpu().numpy(), s_h) < 1e-12


def test_call_order_and_argument_errors():
    g = workload_grid("tiny")
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx:
        ev = synth.events("tiny", 100, 3)
        with pytest.raises(B.ReconError) as e:
            ctx.mlem(B.make_events(ev), 1)
        assert e.value.status == B.RECON_ESTATE
        with pytest.raises(B.ReconError) as e:
            ctx.mlem(None, -1)
        assert e.value.status == B.RECON_EINVAL
        with pytest.raises(B.ReconError):
            ctx.set_launch(100, 0, 0)
        with pytest.raises(B.ReconError):
            ctx.set_launch(256, 4, 48)
        with pytest.raises(B.ReconError):
            ctx.set_launch(256, 0, 0, 128)          # 256 KB of shared memory
        with pytest.raises(B.ReconError):
            ctx.set_launch(128, 0, 0, 4)            # fewer than 8 pieces
        with pytest.raises(B.ReconError):
            ctx.set_kernel_window(0.1)
        bad = B.make_events(ev)
        bad.fmt = 7
        with pytest.raises(B.ReconError):
            ctx.load_events(bad)
        rec = np.zeros((4, 8), np.int16)
        pk = B.make_events(rec, packed=True, lattice_mm=0.0)
        with pytest.raises(B.ReconError):
            ctx.load_events(pk)
        # the failed calls left the context usable: a valid reconstruction runs and
        # matches a fresh context's
        lors = synth.sensitivity_lors("tiny", 20_000, 3)
        ctx.sensitivity(lors)
        img = np.zeros(g.n_vox, np.float32)
        ctx.mlem(B.make_events(ev), 2, None, img)
        with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as fresh:
            fresh.sensitivity(lors)
            ref = np.zeros(g.n_vox, np.float32)
            fresh.mlem(B.make_events(ev), 2, None, ref)
        assert img.max() > 0 and rel_l2(img, ref) < 1e-6
    with B.Context(geometry("tiny"), grid_tuple(g), 300.0) as ctx2:
        with pytest.raises(B.ReconError) as e:
            ctx2.forward(None, None, np.zeros(4, np.float32))
        assert e.value.status == B.RECON_ESTATE


def test_kernel_window_changes_the_projector(ctx_tiny):
    ctx, g = ctx_tiny
    ev, _ = tiny_inputs()
    sub = ev[:, :5000].copy()
    lam = np.random.default_rng(3).uniform(0.5, 1.5, g.n_vox).astype(np.float32)
    p = np.zeros(sub.shape[1], np.float32)
    ctx.set_kernel_window(2.0)
    ctx.forward(B.make_events(sub), lam, p)
    ctx.set_kernel_window(3.0)
    p_ref = oracle.forward(g, sub.astype(np.float64), lam.astype(np.float64), SIGMA, K=2.0)
    sel = p_ref > 1e-3 * p_ref.max()
    # per-event bound of the FP32 walk (the same as test_forward_matches_oracle): a
    # plane crossing tau = (X - c_k) / u_k carries ~ulp(|X - c_k|) / |u_k| of rounding,
    # 3.8e-6 mm / 1e-3 = 3.8e-3 mm for a line with |u_k| = 1e-3, which moves that much
    # chord between two voxels whose lambda differ by up to 1 (lambda in [0.5, 1.5]) at
    # a TOF density of at most 1/(sigma sqrt(2 pi)) = 0.021 / mm: ~8e-5 of p_i ~ 1.
    # Among 5000 isotropic lines about 15 have some |u_k| < 1e-3.
    assert np.max(np.abs(p[sel] - p_ref[sel]) / p_ref[sel]) < 1e-4
    assert np.linalg.norm(p - p_ref) / np.linalg.norm(p_ref) < 2e-6


def test_largest_grid_unit_mass():
    # 1290^3 voxels (just below the 2^31 limit) of 0.5 mm: the 64-bit voxel offsets of the
    # walk and of the image kernels at the largest grid the API accepts.  A forward
    # projection of the constant image 1 gives p_i = 1 (unit TOF mass) for every event
    # whose +-3 sigma window lies inside the grid, whatever the grid's size.
    import torch
    n = 1290
    g = (n, n, n, 0.5, 0.5, 0.5, -n * 0.25, -n * 0.25, -n * 0.25)
    rng = np.random.default_rng(44)
    m = 2000
    u = rng.normal(size=(m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    c = rng.uniform(-100, 100, (m, 3))
    d = rng.uniform(-50, 50, m)
    ev = np.concatenate([(c + 500 * u).T, (c - 500 * u).T, d[None, :]]).astype(np.float32)
    with B.Context((400.0, 2400.0, 90.0), g, 300.0) as ctx:
        ones = torch.ones(n ** 3, dtype=torch.float32, device="cuda")
        p = torch.zeros(m, dtype=torch.float32, device="cuda")
        ctx.forward(B.make_events(ev), ones, p)
        del ones
        p = p.cpu().numpy()
    np.testing.assert_allclose(p, 1.0, atol=2e-5)


def test_coarse_voxels_use_tail_masses():
    # 12 mm voxels: a piece can be 20.8 mm = 1.09 sigma long, beyond the midpoint
    # series' range, so the library's own launch evaluates the masses from the tails;
    # the result still matches the oracle
    ev, lors = tiny_inputs()
    ev = np.ascontiguousarray(ev[:, :60_000])
    g = Grid(11, 11, 16, 12.0, 12.0, 12.0, -66.0, -66.0, -96.0)
    s_ref = oracle.sensitivity(g, lors)
    lam_ref, _ = oracle.mlem(g, ev.astype(np.float64), s_ref, 3, SIGMA)
    with B.Context(geometry("tiny"), (g.nx, g.ny, g.nz, g.vx, g.vy, g.vz, g.ox, g.oy, g.oz), 300.0) as ctx:
        ctx.set_sensitivity(s_ref)
        lam = np.zeros(g.n_vox, np.float32)
        ctx.mlem(B.make_events(ev), 3, None, lam)
        assert ctx.get_launch()[4] != 2
    assert rel_l2(lam, lam_ref) <= 1e-4
    assert max_rel_above(lam, lam_ref, 0.01) <= 1e-3


def test_lines_a_few_ulps_from_a_voxel_plane():
    # Transaxial and axial lines nearly parallel to a voxel plane, their endpoints a
    # few FP32 ulps from it at |coordinate| up to 1 m: the side of the plane the TOF
    # window runs on is decided by ~1e-5 mm.  The image takes another value on each
    # side of every plane, so a window put on the wrong side changes p_i by tens of
    # percent.  The kernel keeps the TOF point as a pair of FP32 numbers; every
    # event must match the FP64 oracle.  Planes at least 100 mm from the origin: at
    # the plane through 0 "a few ulps" are denormals (~1e-45 mm), a side that the
    # FP64 oracle itself cannot resolve (-2.8e-45 + 1200 rounds to 1200).
    g = workload_grid("fullbody")
    rng = np.random.default_rng(71)
    iz = np.arange(g.nz)[:, None, None]
    iy = np.arange(g.ny)[None, :, None]
    ix = np.arange(g.nx)[None, None, :]
    lam = (1.0 + 0.5 * (iz % 2) + 0.25 * (iy % 2) + 0.125 * (ix % 2)).astype(np.float32).reshape(-1)
    events = []
    for _ in range(3000):
        axis = int(rng.integers(0, 3))
        lo = (g.ox, g.oy, g.oz)[axis]
        v = (g.vx, g.vy, g.vz)[axis]
        n = (g.nx, g.ny, g.nz)[axis]
        Z = np.float32(0.0)
        while abs(float(Z)) < 100.0:                                 # a plane away from the origin
            Z = np.float32(lo + v * int(rng.integers(n // 4, n)))
        m1, m2 = rng.integers(-3, 4, 2)
        zs = []
        for m in (m1, m2):
            z = Z
            for _ in range(abs(int(m))):
                z = np.nextafter(z, np.float32(np.inf if m > 0 else -np.inf), dtype=np.float32)
            zs.append(z)
        phi = rng.uniform(0, 2 * np.pi)
        half = rng.uniform(150.0, 280.0)
        a, b = [k for k in range(3) if k != axis]
        p1 = np.zeros(3, np.float32)
        p2 = np.zeros(3, np.float32)
        p1[axis], p2[axis] = zs
        off = rng.uniform(-40, 40, 2)
        p1[a], p1[b] = off[0] + half * np.cos(phi), off[1] + half * np.sin(phi)
        p2[a], p2[b] = off[0] - half * np.cos(phi), off[1] - half * np.sin(phi)
        events.append(np.concatenate([p1, p2, [np.float32(rng.uniform(-60, 60))]]))
    ev = np.ascontiguousarray(np.array(events, np.float32).T)
    with B.Context(geometry("fullbody"), grid_tuple(g), 300.0) as ctx:
        p = np.zeros(ev.shape[1], np.float32)
        ctx.forward(B.make_events(ev), lam, p)
    p_ref = oracle.forward(g, ev.astype(np.float64), lam.astype(np.float64), SIGMA)
    sel = p_ref > 0
    assert sel.sum() > 0.9 * ev.shape[1]
    assert np.array_equal(p > 0, p_ref > 0)
    rel = np.abs(p[sel] - p_ref[sel]) / p_ref[sel]
    assert rel.max() < 1e-4, f"{int(np.sum(rel > 1e-4))} events off, worst {rel.max():.3e}"
