"""FP64 CPU oracle for list-mode TOF-weighted MLEM (arXiv:1706.07075).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import this package.  It shares no code with
the CUDA library (paper_1706_07075_b300): the per-event arithmetic is plain C
(oracle.c, FP64, one rounding per operation), the iteration is plain numpy
(mlem.py), and the two sides meet only at seeded inputs.

Parity status of each function (what pins it is in tests/test_oracle_*.py):
  tof_sigma_mm ........ pinned (Sec. 2.5 prints sigma = 19.11 mm for 300 ps)
  trace ............... pinned (brute-force per-voxel box intersection;
                        analytic chord through the grid box)
  system_row .......... pinned (closed-form truncated-Gaussian mass of the
                        clipped window; unit sum inside the grid)
  forward/backproject . pinned (dense matrix built by brute force; adjointness)
  count_visits ........ pinned (brute-force count of the positive-length
                        pieces inside the TOF windows; axis-parallel closed form)
  sensitivity ......... pinned (chord sums; brute force)
  mlem ................ pinned (dense textbook MLEM on an 8x8x8 grid; the
                        one-voxel closed form; conservation; monotone
                        likelihood; nonnegativity)
  region_codes ........ pinned (hand-built events at the boundaries; the
                        one-or-two-regions property of Sec. 2.5)
  region_slabs ........ pinned (the paper's 176-slice extended regions)
  mlem_regions ........ pinned through mlem and region_codes; the stitched
                        image's count total is a closed form (N events)
  lut_samples ......... pinned (unit sum, symmetry, spacing; second moment
                        converges to the truncated-normal variance)
  forward_lut /
  backproject_lut ..... pinned (brute-force sample positions on axis lines;
                        unit mass inside the grid; adjointness; convergence
                        to the exact Siddon x Phi projector as N grows)
  lut_ambiguous ....... pinned (samples placed by hand at known distances
                        from voxel planes and from the grid boundary)
  preprocess .......... pinned (closed-form line integrals through uniform
                        boxes and a sphere; rejection decided by hand-built
                        events inside, outside and at the 1.96 sigma edge)
  start_backprojection  pinned (equals one MLEM iteration from a uniform
                        image when every event's window lies in the mask;
                        dense-matrix form A^T w / s)
  osem ................ pinned (dense textbook OSEM on an 8x8x8 grid built
                        by brute force; sum s lambda = B N_eff per
                        sub-iteration; B = 1 is MLEM)
  median3 / sieve ..... pinned (scipy.ndimage.median_filter; closed forms on
                        constant images at faces, edges and corners;
                        impulse removal; ramps preserved)
"""
from .core import (  # noqa: F401
    Grid,
    backproject,
    backproject_lut,
    count_visits,
    forward,
    forward_lut,
    LUT_EPS_VOXELS,
    lut_ambiguous,
    lut_samples,
    preprocess,
    region_codes,
    region_members,
    sensitivity,
    system_row,
    threads_used,
    tof_sigma_mm,
    tof_weight,
    trace,
)
from .filters import median3, median3_at, sieve  # noqa: F401
from .mlem import (mlem, mlem_regions, osem, region_bounds, region_slabs, slab_grid, start_backprojection,  # noqa
                   stitch, subset_ranges)
