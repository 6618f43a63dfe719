"""Host-side helpers that need no GPU: the synthetic attenuation map, the
binding's buffer-size check, the bench's shared workload description."""
import os
import sys
import types

import numpy as np
import pytest

from paper_1706_07075_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_mu_image_values_and_outline():
    g = synth.grid_of("tiny")
    mu = synth.mu_image("tiny")
    assert mu.shape == (g[0] * g[1] * g[2],) and mu.dtype == np.float32
    assert set(np.unique(mu).tolist()) <= {0.0, np.float32(synth.MU_WATER)}
    # the tiny body is a cylinder r = 50 mm, |z| <= 80 mm: a voxel centre at the origin is
    # inside, the grid corner outside
    nx, ny, nz, v = g[0], g[1], g[2], g[3]
    a = mu.reshape(nz, ny, nx)
    assert a[nz // 2, ny // 2, nx // 2] == np.float32(synth.MU_WATER)
    assert a[0, 0, 0] == 0.0
    # fraction inside ~ cylinder volume / grid volume
    frac = (mu > 0).mean()
    expect = np.pi * 50.0 ** 2 * 160.0 / (nx * v * ny * v * nz * v)
    assert frac == pytest.approx(expect, rel=0.1)


def test_mu_image_lungs_in_fullbody_outline():
    mu = synth.mu_image("fullbody")
    vals = set(np.unique(mu).tolist())
    assert vals == {0.0, np.float32(synth.MU_LUNG), np.float32(synth.MU_WATER)}


def test_binding_size_check():
    from paper_1706_07075_b300 import binding as B
    B._check_size("x", np.zeros(10), 10)
    with pytest.raises(ValueError):
        B._check_size("x", np.zeros(9), 10)
    B._check_size("x", None, 10)


def test_bench_arms_share_the_workload_config():
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(iters=3, lors=50_000_000, samples=0, events=146_000_000)
    a = bench.workload_config(args, args.events, 1)
    b = bench.workload_config(args, args.events, 1)
    assert a == b and a["events"] == 146_000_000 and a["parallelism"] == "single"
    assert bench.workload_config(args, args.events, 4)["parallelism"] == "replicas4"


def test_bench_reference_arm_prints_one_json_line():
    # the oracle arm of bench.py on a small sample: one JSON line with the keys
    # of the benchmark contract and the same workload description as the CUDA arm
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--cpu-sample", "20000"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600, check=True).stdout.strip().splitlines()
    line = json.loads(out[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["unit"] == "events*iters/s" and line["steps"] == 1 and line["warmup"] == 1
    assert line["config"]["workload"] == "fullbody-146M-150x150x600-4mm"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert "20000" in line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_bench_roofline_terms_and_fraction():
    # the roofline arithmetic of bench.py on the figures of a measured full-body run:
    # 146 M events x 44.25 pieces, pass 31.2 ms, live probes as measured
    sys.path.insert(0, ROOT)
    import bench
    n, visits, pass_ms = 146_000_000, 146_000_000 * 44.25, 31.22
    probes = {"l2_red_gops": 230.8, "gather_gops": 299.1, "l2_stream_gbs": 12862.0, "mixed_gsteps": 99.9}
    r = bench.roofline(n, visits, pass_ms, probes, 6506.9, 2032.0, 49.3 * n)
    t = r["terms_ms"]
    assert t["hbm"] == pytest.approx(32.0 * n / 6506.9e9 * 1e3)
    assert t["l2_reductions"] == pytest.approx(visits / 230.8e9 * 1e3)
    assert t["l2_gathers"] == pytest.approx(visits / 299.1e9 * 1e3)
    assert t["alu"] == pytest.approx(visits * bench.ALU_OPS_PER_PIECE / (148 * 128 * 2032e6) * 1e3)
    # the sector term (an L2 sector per gather, although a third of the gathers hit
    # L1) is reported but is not a lower bound, so it stays out of the maximum
    assert "l2_sectors" not in t
    assert r["l2_sectors_ms_not_a_bound"] == pytest.approx(visits * 64.0 / 12862.0e9 * 1e3)
    # the bound is the largest term, and frac = t_min / t_measured in any unit
    assert r["bound"] == max(t, key=t.get) == "l2_reductions"
    assert r["frac"] == pytest.approx(t["l2_reductions"] / pass_ms)
    assert r["frac"] < 1.0
    assert r["achieved"] == pytest.approx(visits / (pass_ms / 1e3) / 1e9)
    assert r["unit"] == "Gred/s" and r["peak"] == 230.8
    assert r["secondary"]["hbm_frac"] == pytest.approx(32.0 * n / (pass_ms / 1e3) / 6506.9e9)
    # with a slower gather rate the gather term becomes the bound
    slow = dict(probes, gather_gops=150.0)
    r2 = bench.roofline(n, visits, pass_ms, slow, 6506.9, 2032.0, None)
    assert r2["bound"] == "l2_gathers" and r2["unit"] == "Ggather/s" and r2["traffic"] is None
    assert r2["frac"] == pytest.approx(r2["terms_ms"]["l2_gathers"] / pass_ms)
    # request level: the layout's ncu requests per event over the same probe rate; no
    # note while the element rate stays below the scattered rate
    q = r["l2_requests"]
    assert q["achieved_greq_s"] == pytest.approx(bench.NCU_PER_EVENT[0]["l2_requests"] * n / (pass_ms / 1e3) / 1e9)
    assert q["frac"] == pytest.approx(q["achieved_greq_s"] / 230.8) and r["note"] is None
    # the brick layout at 26.6 ms: more reductions per second than the scattered probe
    # (frac above 1, with the note), while its requests stay below the request rate
    rb = bench.roofline(n, visits, 26.57, probes, 6506.9, 2032.0, None, layout=1)
    assert rb["frac"] > 1.0 and rb["note"] and rb["image_layout"] == "2x2x2-brick copies"
    assert rb["l2_requests"]["frac"] < 1.0


def test_fullsize_sampled_voxel_references_match_brute_force():
    """The full-size GPU test recomputes sampled voxels from prefiltered events.
    On 200 k full-body events the prefilter must miss no contributing event:
    lam1 at the sampled voxels from the candidates equals lam1 from all events
    (exact and sampled projectors), the window count brackets the oracle's
    p_i > 0 count, the per-voxel region reference equals the oracle's whole
    region reconstruction at those voxels, and the median-sieve reference its
    whole iteration with the sieve."""
    import oracle
    import test_gpu_fullsize as F
    g = F.workload_grid("fullbody")
    ev = synth.events("fullbody", 200_000, 77)
    rng = np.random.default_rng(5)
    lam0 = (rng.integers(64, 193, g.n_vox) / 128.0).astype(np.float32)
    s = F.smooth_s(g)
    c = F.tof_points(ev)
    vox = F.sample_voxels(g, ev, c, rng)
    cand = F.prefilter(g, ev, c, vox)
    assert vox.size >= 60
    every = [np.arange(ev.shape[1])]
    for lut in (None, 32):
        a = F.oracle_lam1(g, F.events64_of(ev), cand, vox, lam0, s, lut=lut)
        b = F.oracle_lam1(g, F.events64_of(ev), every, vox, lam0, s, lut=lut)
        assert np.count_nonzero(b) >= 0.9 * vox.size
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=0.0)
    p = oracle.forward(g, ev.astype(np.float64), lam0.astype(np.float64), F.SIGMA)
    sure, maybe = F.window_meets_grid(g, ev)
    assert sure <= np.count_nonzero(p > 0) <= sure + maybe

    zb = oracle.region_bounds(g, F.FULLBODY_REGIONS)
    codes = oracle.region_codes(ev, zb, F.SHELL_MM)
    offs, idx = oracle.region_members(codes, len(F.FULLBODY_REGIONS))
    margin = F.K * F.SIGMA + F.SHELL_MM
    slabs = oracle.region_slabs(g, F.FULLBODY_REGIONS, margin)
    pos, ref = F.oracle_region_lam1(g, ev, s, vox, cand, codes, offs, idx, slabs)
    _, images, _, _, _, _ = oracle.mlem_regions(g, ev.astype(np.float64), s, F.FULLBODY_REGIONS, F.SHELL_MM,
                                                margin, 1, F.SIGMA)
    whole = np.concatenate(images)
    assert np.count_nonzero(whole[pos]) >= 0.5 * pos.size      # slab-edge voxels see few windows
    np.testing.assert_allclose(ref, whole[pos], rtol=1e-12, atol=1e-300)

    # the median-sieve reference: the 3x3x3 median of lam1 from the 27 neighbours'
    # prefiltered events equals the oracle's whole iteration with the sieve
    plane = g.ny * g.nx
    centres = np.array([j for j in vox if 0 < j % g.nx < g.nx - 1 and 0 < (j // g.nx) % g.ny < g.ny - 1
                        and 0 < j // plane < g.nz - 1][:16])
    offs27 = np.array([dz * plane + dy * g.nx + dx for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
    nb = (centres[:, None] + offs27[None, :]).ravel()
    lam1_nb = F.oracle_lam1(g, F.events64_of(ev), F.prefilter(g, ev, c, nb), nb, lam0, s).reshape(centres.size, 27)
    med = np.array([oracle.median3_at(row.reshape(3, 3, 3), (3, 3, 3), [13])[0] for row in lam1_nb])
    sieved, _ = oracle.mlem(g, ev.astype(np.float64), s, 1, F.SIGMA, init=lam0.astype(np.float64), median=True)
    assert np.count_nonzero(med) >= centres.size - 2   # slab-edge voxels below the feet see few windows
    np.testing.assert_allclose(med, sieved[centres], rtol=1e-12, atol=0.0)


def test_fullbody_lesions_sit_inside_the_body_on_a_uniform_background():
    # Eq. 1 needs a background VOI for each lesion: the lesion-free phantom must
    # be uniform over the lesion sphere and every lesion inside the body outline
    w = synth.WORKLOADS["fullbody"]()
    bkg = synth.WORKLOADS["fullbody_background"]()
    assert len(bkg.shapes) == len(w.shapes) - len(w.extra["lesions"])
    rng = np.random.default_rng(3)
    ratios = []
    for c, r, act in w.extra["lesions"]:
        d = rng.normal(size=(3, 4000))
        d /= np.linalg.norm(d, axis=0)
        pts = np.asarray(c, np.float64)[:, None] + d * r * rng.uniform(0.0, 1.0, 4000) ** (1.0 / 3.0)
        b = synth.activity_at(bkg, pts)
        assert np.unique(b).size == 1 and b[0] > 0
        assert np.all(synth.activity_at(w, pts) == act)
        body = np.zeros(pts.shape[1], bool)
        for s in bkg.shapes:
            if s.body:
                body |= s.contains(pts)
        assert body.all()
        ratios.append(act / b[0])
    assert ratios[3] == pytest.approx(6.0 / 0.3)      # the lung lesion
    assert ratios[4] == pytest.approx(4.0 / 2.0)      # the liver lesion
    assert min(ratios) > 1.0


def test_fullbody_regions_cover_the_body_in_nine_uneven_regions():
    """The nine body regions of the full-body workload (Sec. 2.5): consecutive
    cores, eight of 200 mm; slabs widened by 3 sigma + 6 mm shell of 60 to 110
    slices; on a seeded sample every region takes between 4 M and 35 M of 146 M
    events, and fewer than 0.5% of the events join no region."""
    import oracle
    regions = synth.FULLBODY_REGIONS
    g = oracle.Grid(*synth.grid_of("fullbody"))
    assert len(regions) == 9
    assert all(regions[r][1] == regions[r + 1][0] for r in range(8))
    assert 0 <= regions[0][0] and regions[-1][1] <= g.nz
    assert [hi - lo for lo, hi in regions[:8]] == [50] * 8 and 50 * g.vz == 200.0
    sigma = oracle.tof_sigma_mm(300.0)
    slabs = oracle.region_slabs(g, regions, 3.0 * sigma + 6.0)
    widths = [hi - lo for lo, hi in slabs]
    assert min(widths) >= 60 and max(widths) <= 110
    ev = synth.events("fullbody", 400_000, 1708).astype(np.float64)
    codes = oracle.region_codes(ev, oracle.region_bounds(g, regions), 6.0)
    offs, _ = oracle.region_members(codes, 9)
    share = np.diff(offs) / ev.shape[1]
    assert share.min() >= 4.0 / 146.0 and share.max() <= 35.0 / 146.0
    assert np.count_nonzero(codes == 0xFF) < 0.005 * ev.shape[1]


def test_synthetic_draws_do_not_depend_on_the_worker_count():
    # chunk k of a draw comes from its own Philox stream keyed by (seed, kind, k):
    # the same events with one worker or several, and whole chunks of a longer
    # draw equal a shorter draw of those chunks
    n = 2 * synth.CHUNK + 1000
    one = synth.events("tiny", n, 11, workers=1)
    two = synth.events("tiny", n, 11, workers=2)
    assert np.array_equal(one, two)
    assert np.array_equal(synth.events("tiny", synth.CHUNK, 11, workers=1), one[:, :synth.CHUNK])
    lors1 = synth.sensitivity_lors("tiny", n, 11, workers=1)
    assert np.array_equal(lors1, synth.sensitivity_lors("tiny", n, 11, workers=3))
    assert not np.array_equal(one[:, :1000], synth.events("tiny", 1000, 12, workers=1))
