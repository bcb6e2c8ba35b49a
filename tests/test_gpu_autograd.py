"""Differentiable projector and penalised reconstruction on the GPU.

Checks, through the C ABI and the autograd binding: the backward of the
projector is Aᵀ (FP32 against the FP64 oracle; FP64 against torch's
finite-difference gradcheck on a 16³ × 8-view × 16² instance), the prior's
value and gradient against the oracle, the penalised objective's gradient
against central finite differences in FP64, and that the gradient solver
with β = 0 and unit step reproduces ML-EM and decreases the objective with
a prior."""
import numpy as np
import pytest

import oracle
from paper_2105_13324_gb300 import phantoms as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2105_13324_gb300 import autograd as AG
    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect
    mcspect.load(B.build())
    # 16^3 torso at 16 mm, 8 views over 180 deg, 16^2 bins of 16 mm
    ph = P.torso_phantom(16, 16.0)
    g = P.spect_geometry(8, 180.0, 16, 16.0, 16, 16.0, hole_len_mm=20.0, hole_diam_mm=4.0, fwhm_mm=8.0)
    pr = oracle.Problem(ph, g)
    H = 4_000_000
    rows, cols, _ = oracle.run(pr, 1, 0, H)
    c = oracle.system_counts(rows, cols, pr.n_rows, pr.n_voxels)
    a = oracle.system_matrix(c, oracle.histories_per_voxel(pr.n_voxels, 0, H))
    sysm = mcspect.mc_system_from_events(pr.n_rows, pr.n_voxels, rows, cols.astype(np.int32), 0, H)
    y = P.poisson_counts(a @ ph.activity.ravel().astype(np.float64), 5e4, 7)
    return mcspect, AG, ph, a, sysm, y


def test_backward_is_the_transpose(env):
    import torch
    mc, AG, ph, a, sysm, y = env
    rng = np.random.default_rng(0)
    x = torch.tensor(rng.uniform(0, 2, a.shape[1]), dtype=torch.float32, device="cuda", requires_grad=True)
    g = rng.uniform(-1, 1, a.shape[0])
    q = AG.project(x, sysm)
    q.backward(torch.tensor(g, dtype=torch.float32, device="cuda"))
    np.testing.assert_allclose(q.detach().cpu().numpy(), a @ x.detach().cpu().numpy().astype(np.float64),
                               rtol=1e-5, atol=1e-6)
    want = a.T @ g
    got = x.grad.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-6
    # FP64: forward and backward against the oracle to rounding
    x64 = x.detach().double().requires_grad_(True)
    q64 = AG.project(x64, sysm)
    np.testing.assert_allclose(q64.detach().cpu().numpy(), a @ x64.detach().cpu().numpy(), rtol=1e-13, atol=1e-15)
    q64.backward(torch.tensor(g, dtype=torch.float64, device="cuda"))
    np.testing.assert_allclose(x64.grad.cpu().numpy(), want, rtol=1e-12, atol=1e-14)


def test_gradcheck_fp64(env):
    import torch
    mc, AG, ph, a, sysm, y = env
    x = torch.rand(a.shape[1], dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: AG.project(t, sysm), (x,), eps=1e-6, atol=1e-7, rtol=1e-5,
                                    fast_mode=True)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_prior_matches_oracle(env, dtype):
    import torch
    mc, AG, ph, a, sysm, y = env
    shape = ph.shape
    rng = np.random.default_rng(1)
    xv = rng.uniform(0, 3, int(np.prod(shape)))
    want_v, want_g = oracle.prior_quadratic(xv, shape, 0.05)
    dt = getattr(torch, dtype)
    x = torch.tensor(xv, dtype=dt, device="cuda")
    g = torch.empty_like(x)
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    mc.mc_prior_quadratic(shape, 0.05, x, g, v)
    tol = 1e-6 if dtype == "float32" else 1e-12
    assert float(v.item()) == pytest.approx(want_v, rel=tol)
    np.testing.assert_allclose(g.cpu().numpy(), want_g, rtol=tol, atol=tol)


def _penalised_objective(AG, x, system, y, shape, beta):
    """Phi(x) = sum_j (q_j - y_j ln q_j) + prior, composed in torch from the
    library's differentiable projector and prior (bins with y_j = 0 add q_j),
    so that autograd differentiates it through the library's A^T."""
    import torch
    q = AG.project(x, system)
    pos = y > 0
    return q.sum() - (y[pos] * torch.log(q[pos])).sum() + AG.quadratic_prior(x, shape, beta)


def test_penalised_gradient_by_central_differences_fp64(env):
    import torch
    mc, AG, ph, a, sysm, y = env
    shape, beta = ph.shape, 0.01
    rng = np.random.default_rng(2)
    x = torch.tensor(rng.uniform(0.5, 2.0, a.shape[1]), dtype=torch.float64, device="cuda", requires_grad=True)
    yd = torch.tensor(y, dtype=torch.float64, device="cuda")
    phi = _penalised_objective(AG, x, sysm, yd, shape, beta)
    (g,) = torch.autograd.grad(phi, x)
    g = g.cpu().numpy()
    np.testing.assert_allclose(g, oracle.penalised_gradient(a, y, x.detach().cpu().numpy(), shape, beta),
                               rtol=1e-9, atol=1e-10)
    # central differences; the objective is ~1e5, so h = 1e-3 keeps the
    # rounding error (~1e-16 * 1e5 / h) below the truncation error (h^2 terms)
    h = 1e-3
    for v in rng.choice(a.shape[1], 40, replace=False):
        e = torch.zeros_like(x)
        e[v] = h
        with torch.no_grad():
            fd = (_penalised_objective(AG, x + e, sysm, yd, shape, beta) -
                  _penalised_objective(AG, x - e, sysm, yd, shape, beta)).item() / (2 * h)
        assert g[v] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_gradient_solver(env):
    import torch
    mc, AG, ph, a, sysm, y = env
    shape = ph.shape
    yd = torch.as_tensor(y).cuda()
    # beta = 0, unit step: exactly the ML-EM update
    x_pgd = AG.penalised_reconstruct(sysm, yd, shape, 0.0, 5)
    x_em = torch.zeros_like(x_pgd)
    mc.mc_mlem_init(sysm, yd, x_em)
    mc.mlem_iterate(sysm, yd, x_em, 5)
    assert float(torch.linalg.norm(x_pgd - x_em) / torch.linalg.norm(x_em)) < 1e-5
    # with a prior (beta relative to the mean sensitivity): non-negative
    # iterates, objective decreasing (checked by the oracle too)
    s_mean = float(oracle.sensitivity(a).mean())
    for rel in (1e-4, 1e-2, 1e-1):
        beta = rel * s_mean
        hist = []
        x = AG.penalised_reconstruct(sysm, yd, shape, beta, 12, history=hist)
        assert torch.all(x >= 0)
        assert all(b <= a_ + 1e-9 * abs(a_) for a_, b in zip(hist, hist[1:]))
        x0 = torch.zeros_like(x)
        mc.mc_mlem_init(sysm, yd, x0)
        o0 = oracle.penalised_objective(a, y, x0.cpu().numpy().astype(np.float64), shape, beta)
        o1 = oracle.penalised_objective(a, y, x.cpu().numpy().astype(np.float64), shape, beta)
        assert o1 < o0
        assert hist[-1] == pytest.approx(o1, rel=1e-5)
