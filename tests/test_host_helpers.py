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
