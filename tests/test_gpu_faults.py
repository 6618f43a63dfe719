"""Failure handling under an exhausted device, made on the host
(recon_debug_fail_alloc): the n-th device allocation the library attempts fails
as if the device were out of memory.  Nothing is allocated for it and no kernel
runs for it, so no GPU faults.

For n = 1, 2, ... every allocation that a sequence of calls makes on a fresh
context fails in turn: the call that needed it (or recon_create) must return
RECON_ENOMEM with a message, and the same context must then run the whole
sequence again with the results of an undisturbed run: sensitivity, event
upload, region split and region MLEM, pre-processing, forward and back
projection, the median filter, MLEM with BF16 gathers, with brick reductions
and with streamed host events.  The sweep ends at the first n past the
sequence's last allocation."""
import numpy as np
import pytest

from gpu_common import geometry, grid_tuple, rel_l2, workload_grid
from paper_1706_07075_b300 import binding as B
from paper_1706_07075_b300 import synth

pytestmark = pytest.mark.gpu

REGIONS = [(0, 16), (16, 32), (32, 48)]


@pytest.fixture(scope="module")
def data():
    g = workload_grid("tiny")
    rng = np.random.default_rng(9)
    return {
        "g": g,
        "ev": synth.events("tiny", 30_000, 91),
        "lors": synth.sensitivity_lors("tiny", 100_000, 91),
        "mu": synth.mu_image("tiny"),
        "lam": rng.uniform(0.5, 1.5, g.n_vox).astype(np.float32),
        "r": rng.uniform(0.0, 2.0, 30_000).astype(np.float32),
    }


def steps(d):
    g, ev = d["g"], d["ev"]
    n, nv = ev.shape[1], g.n_vox
    margin = 3.0 * 19.0965 + 6.0

    def sensitivity(ctx, out):
        out["s"] = np.zeros(nv)
        ctx.sensitivity(d["lors"], out["s"])

    def load(ctx, out):
        ctx.load_events(B.make_events(ev))

    def split(ctx, out):
        out["codes"] = np.zeros(n, np.uint8)
        out["offs"] = np.zeros(len(REGIONS) + 1, np.int64)
        ctx.split_regions(None, REGIONS, margin, 6.0, out["codes"], out["offs"], None)

    def regions(ctx, out):
        out["img_r"] = np.zeros(nv, np.float32)
        ctx.mlem_regions(None, REGIONS, margin, 6.0, 2, out["img_r"])

    def preprocess(ctx, out):
        out["w"] = np.zeros(n, np.float32)
        out["keep"] = np.zeros(n, np.uint8)
        ctx.preprocess(None, d["mu"], 1.96, 0, out["w"], out["keep"])

    def forward(ctx, out):
        out["p"] = np.zeros(n, np.float32)
        ctx.forward(None, d["lam"], out["p"])

    def backproject(ctx, out):
        out["C"] = np.zeros(nv, np.float32)
        ctx.backproject(None, d["r"], out["C"])

    def median(ctx, out):
        out["med"] = np.zeros(nv, np.float32)
        ctx.median_filter(d["lam"], out["med"])

    def mlem_bf16(ctx, out):
        ctx.set_gather_bf16(1)
        try:
            out["img_bf16"] = np.zeros(nv, np.float32)
            ctx.mlem(None, 2, None, out["img_bf16"])
        finally:
            ctx.set_gather_bf16(0)

    def mlem_bricks(ctx, out):
        ctx.set_launch(128, 0, 0, 0, 2, 1)
        try:
            out["img_brick"] = np.zeros(nv, np.float32)
            ctx.mlem(None, 2, None, out["img_brick"])
        finally:
            ctx.set_launch(None)

    def mlem_streamed(ctx, out):
        out["img"] = np.zeros(nv, np.float32)
        out["cons"] = np.zeros((3, 2))
        ctx.mlem(B.make_events(ev), 3, None, out["img"], out["cons"])

    return {f.__name__: f for f in [sensitivity, load, split, regions, preprocess, forward, backproject, median,
                                    mlem_bf16, mlem_bricks, mlem_streamed]}


# Two call orders: a buffer allocated by an earlier call is reused by later ones, so
# the second order puts the projectors and the streamed MLEM where they allocate.
SEQUENCES = {
    "all entry points": (["sensitivity", "load", "split", "regions", "preprocess", "forward", "backproject", "median",
                          "mlem_bf16", "mlem_bricks", "mlem_streamed"],
                         ["recon_create", "sensitivity", "load", "split", "regions", "preprocess", "median",
                          "mlem_bf16", "mlem_bricks"]),
    "projectors and streamed MLEM first": (["sensitivity", "load", "forward", "backproject", "mlem_streamed"],
                                           ["forward", "mlem_streamed"]),
}


def new_context(d):
    return B.Context(geometry("tiny"), grid_tuple(d["g"]), 300.0)


def run_all(ctx, d, names):
    out = {}
    fns = steps(d)
    for name in names:
        fns[name](ctx, out)
    return out


def same_results(got, ref):
    for k in ("codes", "offs", "keep"):
        if k in ref:
            assert np.array_equal(got[k], ref[k]), k
    for k in ("s", "w", "p", "med"):
        if k in ref:
            np.testing.assert_allclose(got[k], ref[k], rtol=1e-6, atol=0.0, err_msg=k)
    for k in ("img_r", "C", "img_bf16", "img_brick", "img"):       # FP32 reductions in another order
        if k in ref:
            assert rel_l2(got[k], ref[k]) <= 1e-5, k
    np.testing.assert_allclose(got["cons"][:, 0], ref["cons"][:, 0], rtol=0, atol=0.5)


@pytest.mark.parametrize("sequence", list(SEQUENCES))
def test_every_allocation_failure_returns_enomem_and_the_context_recovers(data, sequence):
    names, must_fail = SEQUENCES[sequence]
    fns = steps(data)
    with new_context(data) as ctx:
        ref = run_all(ctx, data, names)
    failures = {}
    n = 0
    try:
        for n in range(1, 400):
            B.recon_debug_fail_alloc(n)
            where = None
            ctx = None
            try:
                ctx = new_context(data)
            except B.ReconError as e:
                assert e.status == B.RECON_ENOMEM, e
                assert "out of memory" in str(e)
                where = "recon_create"
            if ctx is not None:
                for name in names:
                    try:
                        fns[name](ctx, {})
                    except B.ReconError as e:
                        assert e.status == B.RECON_ENOMEM, (name, e)
                        assert "out of memory" in str(e), (name, e)
                        where = name
                        break
            B.recon_debug_fail_alloc(0)
            if where is None:
                ctx.close()
                break
            failures[where] = failures.get(where, 0) + 1
            if ctx is None:
                ctx = new_context(data)
            try:
                same_results(run_all(ctx, data, names), ref)
            finally:
                ctx.close()
    finally:
        B.recon_debug_fail_alloc(0)
    print(f"\n{sequence}: {n - 1} allocations failed in turn; calls that returned RECON_ENOMEM: {failures}")
    assert n > 1 and n < 399
    for name in must_fail:
        assert failures.get(name, 0) >= 1, name


def test_fail_alloc_argument_check():
    with pytest.raises(B.ReconError) as e:
        B.recon_debug_fail_alloc(-1)
    assert e.value.status == B.RECON_EINVAL
    B.recon_debug_fail_alloc(0)
