"""Median-filter sieve between MLEM iterations (Sec. 2.4), in plain numpy.

TEST INFRASTRUCTURE (see oracle/__init__.py).

Sec. 2.4 applies a median filter to the image estimate after each iteration
(a sieve: it suppresses high-frequency noise) and Sec. 4 notes that it lowers
voxels at the border of a divided image, where several neighbours are null.
Readings taken where the paper is silent: the neighbourhood is the 3 x 3 x 3
cube around the voxel (27 values, the median is the 14th smallest); a
neighbour outside the grid (or outside a region's slab) counts as zero, which
is the behaviour at the borders that Sec. 4 describes; the filter runs on the
whole grid and voxels outside the mask {s_j > 0} are then set back to zero,
so the mask rule of the update still holds.
"""
import numpy as np


def median3(img, shape_zyx):
    """3x3x3 median of a flat x-fastest image with zero padding; exact selection."""
    a = np.asarray(img, np.float64).reshape(shape_zyx)
    nz, ny, nx = shape_zyx
    pad = np.zeros((nz + 2, ny + 2, nx + 2))
    pad[1:-1, 1:-1, 1:-1] = a
    stack = np.empty((27, nz, ny, nx))
    k = 0
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                stack[k] = pad[dz:dz + nz, dy:dy + ny, dx:dx + nx]
                k += 1
    # 27 values: np.median returns the single middle element of the sorted values
    return np.median(stack, axis=0).reshape(-1)


def sieve(lam, sens, shape_zyx):
    """Median filter, then zero outside the mask {s > 0}."""
    out = median3(lam, shape_zyx)
    out[np.asarray(sens).reshape(-1) <= 0] = 0.0
    return out


def median3_at(img, shape_zyx, vox):
    """median3 at the flat voxel indices vox only (for grids too large for median3)."""
    a = np.asarray(img, np.float64).reshape(shape_zyx)
    nz, ny, nx = shape_zyx
    vox = np.asarray(vox, np.int64)
    z, rem = np.divmod(vox, nx * ny)
    y, x = np.divmod(rem, nx)
    vals = np.zeros((27, vox.size))
    k = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                zz, yy, xx = z + dz, y + dy, x + dx
                inside = (zz >= 0) & (zz < nz) & (yy >= 0) & (yy < ny) & (xx >= 0) & (xx < nx)
                vals[k, inside] = a[zz[inside], yy[inside], xx[inside]]
                k += 1
    return np.median(vals, axis=0)
