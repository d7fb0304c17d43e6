"""Held-out predictions of kernel ridge regression as a differentiable function.

    F(log sigma, log lambda) = K(Xte, X) (K + lambda I)^-1 Y

with the Gaussian kernel of Section 5 and the system of Eq. (1).  The paper
keeps sigma and lambda fixed; this module adds their gradient for any scalar
loss of F.  ``forward`` runs ``krr_pcg_solve`` (Algorithm 1) and
``krr_predict``; ``backward`` runs ``krr_hypergrad`` (the pull-back of dL/dF,
an adjoint solve with the same operator and the (D o K) products).  Every
step runs in the library's CUDA kernels; this file only moves tensors and
scalars across the C boundary.

The random-feature draw ``W, b`` only shapes the preconditioner, which does
not change the converged solution, so it is treated as a constant (draw it
for the current sigma, e.g. ``W = Omega / sigma``).
"""
from __future__ import annotations

import math

import torch

from . import _krr


def _scalar(t) -> float:
    return float(t.detach().cpu()) if torch.is_tensor(t) else float(t)


class KRRPredict(torch.autograd.Function):
    """F = K(Xte, X) (K + lambda I)^-1 Y; differentiable in log sigma and log lambda."""

    @staticmethod
    def forward(ctx, log_sigma, log_lambda, X, Y, Xte, W, b, handle, opts, predict_precision):
        sigma = math.exp(_scalar(log_sigma))
        lam = math.exp(_scalar(log_lambda))
        n, k = Y.shape
        m = Xte.shape[0]
        C = torch.empty((n, k), dtype=torch.float64, device=X.device)
        _krr.krr_pcg_solve(handle, X, sigma, lam, W, b, Y, C, opts)
        F = torch.empty((m, k), dtype=torch.float64, device=X.device)
        _krr.krr_predict(handle, X, Xte, sigma, C, F, predict_precision)
        ctx.save_for_backward(log_sigma, log_lambda, X, Xte, W, b, C)
        ctx.sigma, ctx.lam, ctx.handle, ctx.opts = sigma, lam, handle, opts
        return F

    @staticmethod
    def backward(ctx, gF):
        log_sigma, log_lambda, X, Xte, W, b, C = ctx.saved_tensors
        gF = gF.to(torch.float64).contiguous()
        (dls, dll), _ = _krr.krr_hypergrad(ctx.handle, X, Xte, ctx.sigma, ctx.lam, W, b, C, gF,
                                           ctx.opts)
        g_s = torch.tensor(dls, dtype=log_sigma.dtype, device=log_sigma.device)
        g_l = torch.tensor(dll, dtype=log_lambda.dtype, device=log_lambda.device)
        return g_s, g_l, None, None, None, None, None, None, None, None


def krr_predict_fn(log_sigma, log_lambda, X, Y, Xte, W=None, b=None, handle=None, opts=None,
                   predict_precision="fp64"):
    """Differentiable held-out predictions (m x k float64 on X's device).

    X (n x d) and Xte (m x d) are float32 device tensors, Y (n x k) float64;
    W (d x s) and b (s) the RFF draw for the preconditioner (None together
    with ``opts.precond = 0``).  ``opts`` (a ``krr_opts``) sets the solver
    for both the forward and the adjoint solve.
    """
    h = handle if handle is not None else _krr.Handle()
    o = opts if opts is not None else _krr.default_opts()
    return KRRPredict.apply(log_sigma, log_lambda, X, Y, Xte, W, b, h, o, predict_precision)
