"""The cube-step traversal of the float forced-detection path, as an
algorithm, gives the oracle's transmission.

The float path integrates mu along a ray one cube of constant material at a
time: from the current voxel, whose distance map value is D, the ray runs
to the (D - 1)-th face beyond the voxel's own next face on the first axis
to reach it (clamped at the grid's exit), adding mu times that length; then
each axis advances by the faces it crossed.  Restated here step for step in
float64 (a model of the algorithm, not the library's code) and compared on
random rays through the torso phantom with the oracle's voxel walk
(exp(-sum of mu times the length in each voxel)): the two sums are the same
integral, so they agree to rounding.  The library's float kernel itself is
compared with the oracle on the GPU (tests/test_gpu_fd.py).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2105_13324_gb300 import phantoms as P
from tests.distance_map_ref import distance_map_by_filters

pytest.importorskip("scipy.ndimage")


def _cube_step_transmission(mat, dmap, h, mu, p, d, steps=None):
    nz, ny, nx = mat.shape
    n = np.array([nx, ny, nz])
    half = 0.5 * n * h
    i = np.clip(np.floor((np.asarray(p) + half) / h).astype(np.int64), 0, n - 1)
    s = np.sign(d).astype(np.int64)
    t_a = np.full(3, math.inf)
    dt = np.zeros(3)
    per = np.abs(d) / h                      # faces per unit length
    for a in range(3):
        if s[a]:
            t_a[a] = ((i[a] + (s[a] > 0)) * h - half[a] - p[a]) / d[a]
            dt[a] = h / abs(d[a])
    t_grid = min(t_a[a] + (n[a] - 1 - i[a] if s[a] > 0 else i[a]) * dt[a] for a in range(3) if s[a])
    t, tau = 0.0, 0.0
    for it in range(int(n.sum()) + 3):
        if steps is not None:
            steps[0] += 1
        m = mat[i[2], i[1], i[0]]
        D = int(dmap[i[2], i[1], i[0]])
        c = t_a + (D - 1) * dt               # the cube's exit face on each axis
        tc = min(c.min(), t_grid)
        tau += mu[m] * max(tc - t, 0.0)
        t = max(t, tc)
        if tc >= t_grid:
            break
        k = np.zeros(3, np.int64)
        for a in range(3):
            if c[a] == tc:
                k[a] = D
            elif t_a[a] <= tc:
                k[a] = min(int((tc - t_a[a]) * per[a]) + 1, D)
        i = i + s * k
        t_a = t_a + k * dt
        if np.any(i < 0) or np.any(i >= n):
            break
    return math.exp(-tau)


@pytest.fixture(scope="module")
def torso():
    w = P.workload("torso64")
    pr = oracle.Problem(w.phantom, w.geometry)
    mat = np.ascontiguousarray(w.phantom.material)
    return pr, mat, distance_map_by_filters(mat), float(w.phantom.voxel_mm), len(w.phantom.rho)


@pytest.mark.parametrize("e_kev", [140.5, 126.0])
def test_cube_steps_give_the_voxel_walk_transmission(torso, e_kev):
    pr, mat, dmap, h, n_mat = torso
    mu = [oracle.mu_total(pr, m, e_kev) for m in range(n_mat)]
    nz, ny, nx = mat.shape
    half = 0.5 * np.array([nx, ny, nz]) * h
    rng = np.random.default_rng(5)
    for ray in range(600):
        p = (rng.random(3) * 2.0 - 1.0) * half * 0.999
        if ray % 5 == 0:                      # start on a voxel face
            p[0] = (np.floor((p[0] + half[0]) / h)) * h - half[0]
        d = rng.normal(size=3)
        if ray % 11 == 0:
            d[:2] = 0.0                       # along z only
        elif ray % 7 == 0:
            d[2] = 0.0                        # parallel to the z faces
        d /= np.linalg.norm(d)
        got = _cube_step_transmission(mat, dmap, h, mu, p, d)
        want = oracle.transmission(pr, p, d, e_kev)
        assert -math.log(got) == pytest.approx(-math.log(want), rel=1e-10, abs=1e-12), (p, d)


def test_the_map_makes_the_steps_few(torso):
    # the point of the map: with D = 1 everywhere the same loop is the voxel
    # walk; with the map it takes a fraction of the steps, same result
    pr, mat, dmap, h, n_mat = torso
    mu = [oracle.mu_total(pr, m, 140.5) for m in range(n_mat)]
    ones = np.ones_like(dmap)
    nz, ny, nx = mat.shape
    half = 0.5 * np.array([nx, ny, nz]) * h
    rng = np.random.default_rng(6)
    cube, voxel = [0], [0]
    for _ in range(200):
        p = (rng.random(3) * 2.0 - 1.0) * half * 0.999
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        a = _cube_step_transmission(mat, dmap, h, mu, p, d, cube)
        b = _cube_step_transmission(mat, ones, h, mu, p, d, voxel)
        assert a == pytest.approx(b, rel=1e-12)
    assert cube[0] < 0.5 * voxel[0]
