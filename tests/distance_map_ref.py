"""Distance map of a material grid by its definition (test reference).

D(v) = the largest D <= cap such that every voxel of the grid within
chessboard distance D - 1 of voxel v holds v's material; voxels outside the
grid do not count.  Brute force over growing cubes: for test grids only.
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
