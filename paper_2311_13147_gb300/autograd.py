"""torch.autograd.Function wrappers of the EROT value through the reduced problem.

The value is V = N * [sum_ijk C_ijk T_ijk + eps T_ijk (log T_ijk - 1)] for the
cyclic problem (Eq. problem_CROT times N, Sec. 5.1), computed by the C ABI:
soft-min fold (Eq. def_Kij), cyclic Sinkhorn (Algorithm 2) and
ot_value_and_grad.  Gradients come from the same calls (the forward pass
computes them; backward only scales by the incoming gradient):

* unroll = 0: envelope gradients from Theorem 2's dual at the converged
  potentials;
* unroll = T: gradients of the value after exactly T iterations from z = 0,
  by the library's reverse pass through the checkpointed iterations.

Marginal inputs are normalised inside the library, so d/da_base is the exact
gradient of the normalised function (it sums to zero against a_base).
"""
from __future__ import annotations

import torch

from . import cyclicot as cy


def _solve_value_grad(a_base, b_base, eps, N, C_base=None, x=None, y=None, tol=1e-6, max_iter=10000,
                      unroll=0, need=(True, True, True, True)):
    m = a_base.shape[0]
    dev = a_base.device
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, m, N, C_base=C_base, x=x, y=y, eps=eps)
    d_a = torch.empty(m, device=dev) if need[0] else None
    d_b = torch.empty(m, device=dev) if need[1] else None
    d_C = torch.empty((N, m, m), device=dev) if (C_base is not None and need[2]) else None
    d_x = torch.empty((m, 2), device=dev) if (C_base is None and need[2]) else None
    d_y = torch.empty((m, 2), device=dev) if (C_base is None and need[3]) else None
    if unroll:
        out = cy.ot_value_and_grad(m, N, a_base, b_base, C_base=C_base, x=x, y=y, G=G, eps=eps,
                                   adjoint=cy.OT_ADJ_UNROLLED, unroll_iters=unroll, d_a=d_a, d_b=d_b, d_C=d_C,
                                   d_x=d_x, d_y=d_y)
        res = cy.read_result(out)
    else:
        w, z, so = cy.ot_sinkhorn_reduced(m, N, a_base, b_base, G, cy.options(eps, tol=tol, max_iter=max_iter))
        sres = cy.read_result(so)
        if sres["status"] != cy.OT_OK:
            raise cy.OTError(sres["status"], "ot_sinkhorn_reduced")
        out = cy.ot_value_and_grad(m, N, a_base, b_base, C_base=C_base, x=x, y=y, w=w, z=z, eps=eps,
                                   d_a=d_a, d_b=d_b, d_C=d_C, d_x=d_x, d_y=d_y)
        res = cy.read_result(out)
    if res["status"] != cy.OT_OK:
        raise cy.OTError(res["status"], "ot_value_and_grad")
    return res["value"], d_a, d_b, d_C, d_x, d_y


class CyclicEROT(torch.autograd.Function):
    """V(a_base, b_base, C_base): C_base is the first block row [N, m, m] of the block-circulant cost."""

    @staticmethod
    def forward(ctx, a_base, b_base, C_base, eps, tol=1e-6, max_iter=10000, unroll=0):
        N = C_base.shape[0]
        need = (ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2], False)
        value, d_a, d_b, d_C, _, _ = _solve_value_grad(a_base.detach(), b_base.detach(), float(eps), N,
                                                       C_base=C_base.detach(), tol=tol, max_iter=max_iter,
                                                       unroll=int(unroll), need=need)
        ctx.grads = (d_a, d_b, d_C)
        return torch.tensor(value, dtype=torch.float64, device=a_base.device)

    @staticmethod
    def backward(ctx, gv):
        d_a, d_b, d_C = ctx.grads
        s = gv.to(torch.float32)
        return (None if d_a is None else s * d_a, None if d_b is None else s * d_b,
                None if d_C is None else s * d_C, None, None, None, None)


class CyclicEROTPoints(torch.autograd.Function):
    """V(a_base, b_base, x, y) with C_k[i, j] = |x_i - R^k y_j|^2, R the rotation by 2 pi / N."""

    @staticmethod
    def forward(ctx, a_base, b_base, x, y, N, eps, tol=1e-6, max_iter=10000, unroll=0):
        need = (ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2] or ctx.needs_input_grad[3],
                ctx.needs_input_grad[2] or ctx.needs_input_grad[3])
        value, d_a, d_b, _, d_x, d_y = _solve_value_grad(a_base.detach(), b_base.detach(), float(eps), int(N),
                                                         x=x.detach().contiguous(), y=y.detach().contiguous(),
                                                         tol=tol, max_iter=max_iter, unroll=int(unroll), need=need)
        ctx.grads = (d_a, d_b, d_x, d_y)
        return torch.tensor(value, dtype=torch.float64, device=a_base.device)

    @staticmethod
    def backward(ctx, gv):
        d_a, d_b, d_x, d_y = ctx.grads
        s = gv.to(torch.float32)
        sc = (lambda t: None if t is None else s * t)
        return sc(d_a), sc(d_b), sc(d_x), sc(d_y), None, None, None, None, None


def cyclic_erot_value(a_base, b_base, eps, C_base=None, x=None, y=None, N=None, tol=1e-6, max_iter=10000, unroll=0):
    """Differentiable EROT value of the cyclic problem (blocks or points)."""
    if C_base is not None:
        return CyclicEROT.apply(a_base, b_base, C_base, eps, tol, max_iter, unroll)
    return CyclicEROTPoints.apply(a_base, b_base, x, y, N, eps, tol, max_iter, unroll)
