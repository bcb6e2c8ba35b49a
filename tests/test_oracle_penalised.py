"""Pins for the oracle's quadratic prior and penalised Poisson objective:
brute force over voxel pairs, central finite differences, invariances."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import oracle


def test_prior_value_by_brute_force_over_pairs():
    rng = np.random.default_rng(0)
    shape = (3, 4, 5)
    x = rng.normal(size=np.prod(shape))
    img = x.reshape(shape)
    want = 0.0
    for k, j, i in itertools.product(range(3), range(4), range(5)):
        for dk, dj, di in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            if k + dk < 3 and j + dj < 4 and i + di < 5:
                want += (img[k, j, i] - img[k + dk, j + dj, i + di]) ** 2
    val, _ = oracle.prior_quadratic(x, shape, 0.7)
    assert val == pytest.approx(0.35 * want, rel=1e-13)


def test_prior_gradient_by_finite_differences_and_invariances():
    rng = np.random.default_rng(1)
    shape = (4, 3, 5)
    x = rng.normal(size=np.prod(shape))
    _, g = oracle.prior_quadratic(x, shape, 1.3)
    h = 1e-6
    for v in range(x.size):
        e = np.zeros_like(x)
        e[v] = h
        fd = (oracle.prior_quadratic(x + e, shape, 1.3)[0] - oracle.prior_quadratic(x - e, shape, 1.3)[0]) / (2 * h)
        assert g[v] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    v0, g0 = oracle.prior_quadratic(np.full(x.size, 3.0), shape, 2.0)
    assert v0 == 0.0 and np.all(g0 == 0.0)
    assert abs(np.sum(g)) < 1e-12          # the penalty is shift invariant


def test_penalised_gradient_by_finite_differences():
    rng = np.random.default_rng(2)
    shape = (2, 3, 4)
    n = int(np.prod(shape))
    a = sp.csr_matrix(rng.uniform(0, 1, (30, n)) ** 3)
    x = rng.uniform(0.5, 2.0, n)
    y = rng.poisson(a @ x).astype(float)
    g = oracle.penalised_gradient(a, y, x, shape, 0.4)
    h = 1e-6
    for v in range(n):
        e = np.zeros(n)
        e[v] = h
        fd = (oracle.penalised_objective(a, y, x + e, shape, 0.4) -
              oracle.penalised_objective(a, y, x - e, shape, 0.4)) / (2 * h)
        assert g[v] == pytest.approx(fd, rel=1e-5, abs=1e-7)
