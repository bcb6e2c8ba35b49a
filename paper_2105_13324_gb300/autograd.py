"""Differentiable projector and penalised-likelihood reconstruction.

`project(x, system)` is A·x (Eq. (IMC) of Sec. 5.1) as a torch autograd
function whose backward is the library's Aᵀ kernel (float32 or float64,
following x).  `quadratic_prior` is the 6-neighbour smoothness penalty
computed by the library.  `penalised_reconstruct` minimises
    Φ(x) = Σ_j (q_j − y_j ln q_j) + β/2 Σ_(v,w) (x_v − x_w)²,  q = A x,
by EM-preconditioned projected gradient steps (`mc_pgd_step`); with β = 0
and step 1 each step is one ML-EM update (Eq. (MLEM)).  Every arithmetic
step runs in the CUDA library; torch only holds the device buffers.
"""
from __future__ import annotations

import torch

from . import mcspect as mc


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, system):
        ctx.system = system
        m, _ = system.shape
        q = torch.empty(m, dtype=x.dtype, device=x.device)
        xc = x.contiguous()
        if x.dtype == torch.float64:
            mc.mc_project_f64(system, xc, q)
        else:
            mc.mc_project(system, xc, q)
        return q

    @staticmethod
    def backward(ctx, g):
        _, n = ctx.system.shape
        b = torch.empty(n, dtype=g.dtype, device=g.device)
        gc = g.contiguous()
        if g.dtype == torch.float64:
            mc.mc_backproject_f64(ctx.system, gc, b)
        else:
            mc.mc_backproject(ctx.system, gc, b)
        return b, None


def project(x: torch.Tensor, system) -> torch.Tensor:
    """q = A x, differentiable in x (backward = Aᵀ)."""
    return _Project.apply(x, system)


class _Prior(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, shape, beta):
        grad = torch.empty_like(x)
        value = torch.zeros(1, dtype=torch.float64, device=x.device)
        mc.mc_prior_quadratic(shape, beta, x.contiguous(), grad, value)
        ctx.save_for_backward(grad)
        return value.to(x.dtype)[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None, None


def quadratic_prior(x: torch.Tensor, shape, beta: float) -> torch.Tensor:
    """β/2 Σ over 6-neighbour pairs (x_v − x_w)², differentiable in x."""
    return _Prior.apply(x, tuple(shape), float(beta))


def penalised_reconstruct(system, y, shape, beta: float, n_iter: int, alpha: float = 1.0, x0=None,
                          history: list | None = None):
    """EM-preconditioned projected gradient descent on Φ (float32 images,
    FP64 objective).  Each step starts at `alpha` and halves it until Φ does
    not increase (at most 20 halvings), so Φ decreases monotonically; with
    β = 0 and alpha = 1 the first trial is the ML-EM update, which never
    increases Φ.  `history` (a list) receives Φ after each step."""
    m, n = system.shape
    dev = y.device
    sens = torch.empty(n, dtype=torch.float64, device=dev)
    mc.mc_sensitivity(system, sens)
    x = torch.empty(n, dtype=torch.float32, device=dev)
    if x0 is None:
        mc.mc_mlem_init(system, y, x)
    else:
        x.copy_(x0)
    r = torch.empty(m, dtype=torch.float32, device=dev)
    bp = torch.empty(n, dtype=torch.float32, device=dev)
    gp = torch.empty(n, dtype=torch.float32, device=dev) if beta > 0 else None
    ll = torch.zeros(1, dtype=torch.float64, device=dev)
    pv = torch.zeros(1, dtype=torch.float64, device=dev)

    def phi(img):
        mc.mc_loglik(system, img, y, ll)
        val = -float(ll.item())
        if beta > 0:
            mc.mc_prior_quadratic(shape, beta, img, None, pv)
            val += float(pv.item())
        return val

    cur = phi(x)
    for _ in range(n_iter):
        mc.mc_project_ratio(system, x, y, r)
        mc.mc_backproject(system, r, bp)
        if gp is not None:
            mc.mc_prior_quadratic(shape, beta, x, gp)
        a = alpha
        for _ in range(21):
            xn = x.clone()
            mc.mc_pgd_step(a, sens, bp, xn, gp)
            new = phi(xn)
            if new <= cur or a < alpha * 2.0 ** -19:
                break
            a *= 0.5
        if new <= cur:
            x, cur = xn, new
        if history is not None:
            history.append(cur)
    return x
