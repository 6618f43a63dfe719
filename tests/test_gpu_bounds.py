"""The bounds-checked build (librecon_check.so, RECON_BOUNDS_CHECK): every voxel
index that a walk produces (event passes of both projectors and both reduction
forms, the tiled pass, pre-processing, the sensitivity) is checked against its
image before use, and an index outside is counted instead of being accessed.
A spread of workloads runs in a fresh process on that build (grids with odd
extents, lines a few ulps from voxel planes, rays along grid faces, regions,
tiles, packed events) and must count no out-of-range index.  This stands in for
a memory sanitizer: nothing traps and nothing faults."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
from paper_1706_07075_b300 import binding as B, synth
from gpu_common import geometry, grid_tuple, workload_grid
import oracle
assert B.library_path().endswith("librecon_check.so")
assert B.recon_debug_bounds_violations() == 0            # checks compiled in, nothing counted yet
total = 0

def run(geo, g, ev, lors, extra=None):
    global total
    with B.Context(geo, grid_tuple(g), 300.0) as ctx:
        ctx.sensitivity(lors)
        ctx.load_events(B.make_events(ev))
        for launch in [(128, 0, 0, 0, 2, 0), (128, 0, 0, 0, 3, 0), (128, 0, 0, 0, 3, 1), (96, 0, 0, 0, 0, 0),
                       (128, 4, 64, 32, 1, 0)]:
            ctx.set_launch(*launch)
            ctx.mlem(None, 2)
        ctx.set_launch(None)
        ctx.set_projector(B.PROJ_SAMPLED, 32)
        ctx.mlem(None, 2)
        ctx.set_brick_layout(1)
        ctx.mlem(None, 2)
        ctx.set_brick_layout(0)
        ctx.set_projector(B.PROJ_EXACT)
        ctx.set_tiled_pass(1, 8)
        ctx.mlem(None, 2)
        ctx.set_tiled_pass(1, 1)
        ctx.mlem(None, 2)
        ctx.set_tiled_pass(0, 1)
        nz = g.nz
        regions = [(0, nz // 3), (nz // 3, 2 * nz // 3), (2 * nz // 3, nz)]
        ctx.mlem_regions(None, regions, 3 * 19.0965 + 6.0, 6.0, 2)
        ctx.set_launch(128, 0, 0, 0, 3, 1)            # every slab over its own brick copies
        ctx.mlem_regions(None, regions, 3 * 19.0965 + 6.0, 6.0, 2)
        ctx.set_launch(None)
        ctx.preprocess(None, np.full(g.n_vox, 0.0096, np.float32), 1.96, 0)
        if extra:
            extra(ctx)
    n = B.recon_debug_bounds_violations()
    print(f"{{g}}: {{n}} out-of-range indices")
    total += n

tiny = workload_grid("tiny")
run(geometry("tiny"), tiny, synth.events("tiny", 60_000, 5), synth.sensitivity_lors("tiny", 200_000, 5))
odd = oracle.Grid.centred(33, 31, 47, 4.0)
run(geometry("tiny"), odd, synth.events("tiny", 60_000, 6), synth.sensitivity_lors("tiny", 200_000, 6))
fb = workload_grid("fullbody")
run(geometry("fullbody"), fb, synth.events("fullbody", 1_500_000, 7), synth.sensitivity_lors("fullbody", 500_000, 7))
# rays along the grid's faces and edges, both directions, and in voxel planes
h = 0.5 * tiny.nx * tiny.vx
face = []
for x in (-h, h, 0.0, 4.0):
    for y in (-h, h, 0.0):
        face.append([x, y, -300.0, x, y, 300.0, 10.0])
        face.append([x, -300.0, y, x, 300.0, y, -5.0])
        face.append([-300.0, x, y, 300.0, x, y, 0.0])
face = np.ascontiguousarray(np.array(face, np.float32).T)
run(geometry("tiny"), tiny, np.concatenate([synth.events("tiny", 5000, 8), face], axis=1),
    synth.sensitivity_lors("tiny", 50_000, 8))
print("TOTAL", total)
'''


def test_checked_build_counts_no_out_of_range_index():
    env = dict(os.environ, RECON_BOUNDS_CHECK="1")
    code = SCRIPT.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    print(r.stdout[-3000:], r.stderr[-3000:])
    assert r.returncode == 0
    assert "TOTAL 0" in r.stdout
