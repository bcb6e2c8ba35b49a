"""Distance map of a material grid by its definition (test reference).

D(v) = the largest D <= cap such that every voxel of the grid within
chessboard distance D - 1 of voxel v holds v's material; voxels outside the
grid do not count.  Brute force over growing cubes (small test grids), and
the same map from windowed minimum and maximum filters (any size): the cube
of half-width r around v, clipped to the grid, holds one material iff the
minimum and the maximum of the material over the (2r + 1)^3 window agree
(with edge replication, the window's outside values repeat voxels inside
the clipped cube).
"""
import numpy as np


def distance_map_by_definition(mat, cap=16):
    out = np.zeros(mat.shape, np.int64)
    for z, y, x in np.ndindex(mat.shape):
        d = 1
        while d < cap:
            cube = mat[max(0, z - d):z + d + 1, max(0, y - d):y + d + 1, max(0, x - d):x + d + 1]
            if not np.all(cube == mat[z, y, x]):
                break
            d += 1
        out[z, y, x] = d
    return out


def distance_map_by_filters(mat, cap=16):
    from scipy import ndimage
    d = np.ones(mat.shape, np.int64)
    for r in range(1, cap):
        lo = ndimage.minimum_filter(mat, size=2 * r + 1, mode="nearest")
        hi = ndimage.maximum_filter(mat, size=2 * r + 1, mode="nearest")
        d += (lo == hi) & (d == r)
    return d
