"""The distance map's test reference against an independent formulation.

The GPU test of mc_debug_distance_map compares the library with
distance_map_by_definition (brute force over growing cubes); here that
brute force is checked against the windowed minimum/maximum filter
formulation and against values worked out by hand.
"""
import numpy as np
import pytest

from tests.distance_map_ref import distance_map_by_definition, distance_map_by_filters

pytest.importorskip("scipy.ndimage")


@pytest.mark.parametrize("shape,p,seed", [((6, 7, 9), 0.15, 0), ((3, 20, 20), 0.02, 1), ((1, 1, 1), 0.5, 2),
                                          ((2, 5, 40), 0.0, 3), ((9, 9, 9), 0.004, 4)])
def test_brute_force_equals_window_filters(shape, p, seed):
    rng = np.random.default_rng(seed)
    mat = (rng.random(shape) < p).astype(np.uint8)
    mat[rng.random(shape) < p / 2] = 2
    np.testing.assert_array_equal(distance_map_by_definition(mat), distance_map_by_filters(mat))


def test_known_values():
    # a single odd voxel in the middle of a 1 x 1 x 9 row: distances to it
    mat = np.zeros((1, 1, 9), np.uint8)
    mat[0, 0, 4] = 1
    np.testing.assert_array_equal(distance_map_by_definition(mat)[0, 0], [4, 3, 2, 1, 1, 1, 2, 3, 4])
    # a uniform grid reaches the cap
    assert distance_map_by_definition(np.zeros((2, 2, 2), np.uint8)).min() == 16
