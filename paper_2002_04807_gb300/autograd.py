"""Differentiable FEAST eigenvalues (torch.autograd.Function).

forward: the eigenvalues lambda_1..lambda_M of A x = lambda B x inside
[emin, emax], computed by the GPU FEAST solver (feast_scsr_solve_dev).
backward: for a loss L = sum_k g_k lambda_k the gradient over the stored CSR
values is, for B-orthonormal eigenvectors x_k (first-order perturbation of
simple eigenvalues),
    dL/da_p = sum_k g_k x_k[i_p] x_k[j_p],
    dL/db_p = -sum_k g_k lambda_k x_k[i_p] x_k[j_p],
evaluated by the library's SDDMM kernel (feast_eig_grad_dev).  Each stored
entry gets its own derivative; perturbing a symmetric pair (i,j),(j,i) moves
the loss by the sum of the two entries' derivatives.  Eigenvalues inside the
loss must be simple (distinct): for a degenerate cluster only symmetric
functions of the cluster are differentiable.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib


class FeastEigenvalues(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b, ia, ja, ib, jb, n, emin, emax, m0, fpm, x0):
        x = torch.zeros((m0, n), dtype=torch.float64, device=a.device) if x0 is None else x0.clone()
        f = np.array(fpm, dtype=np.int32, copy=True)
        if x0 is not None:
            f[4] = 1
        r = _lib.feast_scsr_solve_dev(n, ia, ja, a.detach(), ib, jb, None if b is None else b.detach(), fpm=f,
                                      emin=emin, emax=emax, m0=m0, x=x)
        if r.info not in (0, 3):
            raise _lib.FeastError(f"FEAST returned info {r.info}")
        M = r.M
        lam = torch.as_tensor(r.E[:M].copy(), dtype=torch.float64, device=a.device)
        Xr = x[:M].t().contiguous()  # row-major n x M, eigenvectors in columns
        ctx.save_for_backward(Xr, lam, ia, ja, ib if ib is not None else ia, jb if jb is not None else ja)
        ctx.has_b = b is not None
        ctx.n = n
        ctx.nnz = (a.numel(), 0 if b is None else b.numel())
        return lam

    @staticmethod
    def backward(ctx, g):
        Xr, lam, ia, ja, ib, jb = ctx.saved_tensors
        M = lam.numel()
        g = g.to(torch.float64).contiguous()
        grad_a = torch.zeros(ctx.nnz[0], dtype=torch.float64, device=Xr.device)
        grad_b = None
        if M > 0:
            _lib.feast_eig_grad_dev(ctx.n, ia, ja, M, Xr, g, grad_a)
            if ctx.has_b:
                grad_b = torch.zeros(ctx.nnz[1], dtype=torch.float64, device=Xr.device)
                _lib.feast_eig_grad_dev(ctx.n, ib, jb, M, Xr, (-g * lam).contiguous(), grad_b)
        elif ctx.has_b:
            grad_b = torch.zeros(ctx.nnz[1], dtype=torch.float64, device=Xr.device)
        return grad_a, grad_b, None, None, None, None, None, None, None, None, None, None


def feast_eigenvalues(a, ia, ja, n, emin, emax, m0, fpm, b=None, ib=None, jb=None, x0=None):
    """Eigenvalues of (A, B) in [emin, emax] as a differentiable tensor.

    a, b: CUDA float64 CSR values (0-based full storage; ia/ja/ib/jb CUDA
    int32); B omitted means B = I.  x0: optional (m0, n) CUDA float64 start
    subspace (column-major n x m0).  fpm: 64 FEAST parameters."""
    return FeastEigenvalues.apply(a, b, ia, ja, ib, jb, n, emin, emax, m0, fpm, x0)
