"""Pins for the oracle's ML-EM (paper Sec. 5.1, Eq. (MLEM)).

Checked against properties of the EM algorithm for Poisson data that the
paper relies on through its citations (Shepp & Vardi 1982, Lange & Carson
1984): non-negativity, preservation of the total count, monotone
likelihood, one-step convergence for a diagonal system, convergence to the
exact solution of a consistent invertible system, and the Karush-Kuhn-Tucker
conditions of the maximum-likelihood solution on a 4^3 toy whose optimum is
found by an independent bound-constrained optimiser.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy import optimize, stats

import oracle


def _random_system(m, n, density, seed):
    rng = np.random.default_rng(seed)
    a = sp.random(m, n, density=density, random_state=rng, format="csr", dtype=np.float64)
    a = a + sp.csr_matrix((np.full(m, 0.05), (np.arange(m), rng.integers(0, n, m))), shape=(m, n))
    return sp.csr_matrix(a), rng


def test_loglik_is_poisson_log_pmf_up_to_constant():
    a, rng = _random_system(40, 25, 0.3, 1)
    x = rng.uniform(0.5, 2.0, 25)
    q = a @ x
    y = rng.poisson(q).astype(np.float64)
    want = stats.poisson.logpmf(y, q).sum() + np.sum([np.sum(np.log(np.arange(1, k + 1))) for k in y])
    assert oracle.loglik(a, x, y) == pytest.approx(want, rel=1e-12)


def test_nonnegative_count_preserving_monotone():
    a, rng = _random_system(300, 120, 0.05, 2)
    x_true = rng.uniform(0.0, 3.0, 120)
    y = rng.poisson(a @ x_true).astype(np.float64)
    x = oracle.mlem_init(a, y)
    s = oracle.sensitivity(a)
    x, ll = oracle.mlem(a, y, x, 60, with_loglik=True)
    assert np.all(x >= 0)
    assert float(s @ x) == pytest.approx(float(y.sum()), rel=1e-12)
    ll = np.asarray(ll)
    assert np.all(np.diff(ll) >= -1e-12 * np.abs(ll[1:]))


def test_each_iterate_preserves_counts():
    a, rng = _random_system(80, 40, 0.1, 3)
    y = rng.poisson(a @ rng.uniform(0, 2, 40)).astype(np.float64)
    s = oracle.sensitivity(a)
    x = oracle.mlem_init(a, y)
    for _ in range(5):
        x = oracle.mlem_step(a, y, x, s)
        assert float(s @ x) == pytest.approx(float(y.sum()), rel=1e-12)


def test_diagonal_system_converges_in_one_step():
    d = np.array([0.5, 2.0, 0.25, 1.0, 3.0])
    a = sp.diags(d).tocsr()
    y = np.array([3.0, 4.0, 0.0, 7.0, 9.0])
    x = oracle.mlem(a, y, np.ones(5), 1)
    np.testing.assert_allclose(x, y / d, rtol=1e-15)


def test_consistent_invertible_system_converges_to_truth():
    rng = np.random.default_rng(4)
    n = 12
    a = np.eye(n) * 2.0 + rng.uniform(0.0, 0.2, (n, n))
    x_true = rng.uniform(0.5, 2.0, n)
    y = a @ x_true
    x = oracle.mlem(sp.csr_matrix(a), y, np.ones(n), 4000)
    np.testing.assert_allclose(x, x_true, rtol=1e-9)


def test_zero_sensitivity_voxels_and_empty_projections():
    a = sp.csr_matrix(np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 0.0]]))
    y = np.array([2.0, 4.0, 5.0])          # last bin sees no voxel: contributes nothing
    x = oracle.mlem(a, y, np.array([1.0, 1.0, 1.0]), 3)
    np.testing.assert_allclose(x, [2.0, 2.0, 0.0])
    x0 = oracle.mlem_init(a, y)
    assert x0[2] == 0.0 and x0[0] == pytest.approx(11.0 / 3.0)


def test_toy_4cubed_reaches_the_ml_optimum():
    # 64 voxels, 96 bins, dense positive system: the ML estimate found by
    # L-BFGS-B on the negative log-likelihood (x >= 0) must satisfy the same
    # KKT conditions as the EM fixed point, and both must agree.
    rng = np.random.default_rng(5)
    m, n = 96, 64
    a_dense = rng.uniform(0.0, 1.0, (m, n)) ** 4
    a = sp.csr_matrix(a_dense)
    x_true = rng.uniform(0.0, 4.0, n)
    x_true[rng.choice(n, 8, replace=False)] = 0.0
    y = rng.poisson(a_dense @ x_true).astype(np.float64)

    x_em = oracle.mlem(a, y, oracle.mlem_init(a, y), 20000)

    def nll(x):
        q = a_dense @ x
        return float(np.sum(q) - np.sum(y[y > 0] * np.log(np.maximum(q[y > 0], 1e-300))))

    def grad(x):
        q = a_dense @ x
        return a_dense.sum(axis=0) - a_dense.T @ np.where(y > 0, y / np.maximum(q, 1e-300), 0.0)

    res = optimize.minimize(nll, np.full(n, y.sum() / a_dense.sum()), jac=grad, method="L-BFGS-B",
                            bounds=[(0, None)] * n, options={"maxiter": 20000, "ftol": 1e-15, "gtol": 1e-12})
    assert nll(x_em) <= nll(res.x) + 1e-6 * abs(nll(res.x))
    # KKT: dL/dx_v = sum_j a_jv (y_j/q_j - 1) is 0 where x_v > 0 and <= 0 where x_v = 0
    q = a_dense @ x_em
    g = a_dense.T @ (y / q - 1.0)
    s = a_dense.sum(axis=0)
    on = x_em > 1e-3
    assert np.max(np.abs(g[on]) / s[on]) < 1e-4
    assert np.max(g[~on] / s[~on]) < 1e-3
    np.testing.assert_allclose(x_em[on], res.x[on], rtol=2e-3, atol=2e-3)


def test_loglik_leaves_out_bins_the_model_cannot_reach():
    # row 2 of A is empty: q_2 = 0 for every image, so its y ln q term is
    # left out (by hand: L = 3 ln 2 + 1 ln 3 - (2 + 3)); ML-EM ignores the
    # bin (r_2 = 0) and increases this L monotonically
    a = sp.csr_matrix(np.array([[1.0, 1.0], [0.0, 3.0], [0.0, 0.0]]))
    y = np.array([3.0, 1.0, 4.0])
    x = np.array([1.0, 1.0])
    assert oracle.loglik(a, x, y) == pytest.approx(3 * np.log(2.0) + np.log(3.0) - 5.0, rel=1e-15)
    x = oracle.mlem_init(a, y)
    ll = [oracle.loglik(a, x, y)]
    for _ in range(20):
        x = oracle.mlem_step(a, y, x)
        ll.append(oracle.loglik(a, x, y))
    assert np.all(np.isfinite(ll)) and np.all(np.diff(ll) >= -1e-12 * np.abs(ll[1:]))
    # a reachable bin with q_j = 0 and y_j > 0 still gives -inf
    assert oracle.loglik(a, np.array([0.0, 0.0]), y) == -np.inf
