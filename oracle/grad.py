"""Gradients of the EROT value (float64).

Oracle code: test infrastructure only (see ``oracle/__init__.py``).

The paper motivates EROT by its differentiability (Sec. 5) but prints no
gradient; the formulas here follow from Theorem 2's dual by the envelope
theorem.  With V = N * D(w*, z*) the full-problem optimum (Sec. 5.1's 1/N
relation) and D the dual objective of Eq. dual_problem_cyclic_ROT:

* dV/dalpha = N w*,  dV/dbeta = N z*;
* dV/dC_ijk = N * T_ijk with T_ijk = exp((w*_i + z*_j - C_ijk)/lam)
  (differentiating -lam * exp((w_i + z_j - C_ijk)/lam));
* for C_ijk = |x_i - R^k y_j|^2:  dV/dx_i = 2N sum_jk T_ijk (x_i - R^k y_j)
  and dV/dy_j = 2N sum_ik T_ijk (y_j - R^-k x_i).

The library normalises its marginal inputs, alpha = a_base / (N * sum a_base),
so the gradient with respect to a_base is the chain rule through that map:
dV/da_base_l = (w_l - <w, a_base>/s) / s with s = sum(a_base) (the constant
that leaves V unchanged on the simplex is thereby fixed).

The unrolled gradient differentiates the value after a fixed number of
iterations, V_T = N(<w_T, alpha> + <z_T, beta>) - lam, through the iterations
themselves (torch float64 autograd on CPU: plain library differentiation of
the plain loop).
"""
from __future__ import annotations

import numpy as np

from .sinkhorn import base_marginals, cyclic_sinkhorn, unfold_erot, sinkhorn_full, normalise


def rot2(theta):
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, -s], [s, c]])


def cost_from_points(x, y, N):
    """C_base[k, i, j] = |x_i - R^k y_j|^2 with R the rotation by 2*pi/N (float64)."""
    out = np.empty((N, x.shape[0], y.shape[0]))
    for k in range(N):
        yk = y @ rot2(2 * np.pi * k / N).T
        out[k] = ((x[:, None, :] - yk[None, :, :]) ** 2).sum(-1)
    return out


def _marginal_chain(w, v_base):
    v = np.asarray(v_base, np.float64)
    s = v.sum()
    return (w - (w @ v) / s) / s


def envelope_grad(a_base, b_base, C_base, lam, tol=1e-13, max_iter=200000, x=None, y=None):
    """Value and envelope gradients of the EROT value through the reduced problem.

    Returns dict with value (dual, full scale), d_a, d_b (gradients w.r.t. the
    un-normalised base marginals), d_C ([N, m, m] = N * T_k) and, when points
    x, y are given, d_x, d_y.
    """
    C_base = np.asarray(C_base, np.float64)
    N = C_base.shape[0]
    sol = cyclic_sinkhorn(a_base, b_base, C_base, lam, tol=tol, max_iter=max_iter)
    w, z = sol["w"], sol["z"]
    alpha, beta = sol["alpha"], sol["beta"]
    T = unfold_erot(w, z, C_base, lam)
    out = {
        "value": float(N * (w @ alpha + z @ beta - lam * T.sum())),
        "d_a": _marginal_chain(w, a_base),
        "d_b": _marginal_chain(z, b_base),
        "d_C": N * T,
        "w": w, "z": z, "iters": sol["iters"], "err": sol["err"],
    }
    if x is not None:
        dx = np.zeros_like(x, dtype=np.float64)
        dy = np.zeros_like(y, dtype=np.float64)
        for k in range(N):
            R = rot2(2 * np.pi * k / N)
            yk = y @ R.T
            Tk = T[k]
            dx += 2 * N * (Tk.sum(1)[:, None] * x - Tk @ yk)
            # y_j - R^-k x_i  summed with weights T_ijk
            xk = x @ R               # rows are R^-k x_i  (R^T = R^-1)
            dy += 2 * N * (Tk.sum(0)[:, None] * y - Tk.T @ xk)
        out["d_x"], out["d_y"] = dx, dy
    return out


def full_problem_grad(a_full, b_full, X, Y, lam, tol=1e-13, max_iter=200000):
    """Value and envelope gradients of the FULL n x n EROT with C_rs = |X_r - Y_s|^2.

    Independent of the reduction: solves the plain problem (Algorithm 3 Stage 2)
    and differentiates it (dV/da = f - <f,a>, dV/dX_r = 2 sum_s T_rs (X_r - Y_s), ...).
    """
    C = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    a, b = normalise(a_full), normalise(b_full)
    sol = sinkhorn_full(a, b, C, lam, tol=tol, max_iter=max_iter)
    f, g = sol["f"], sol["g"]
    T = np.exp((f[:, None] + g[None, :] - C) / lam)
    return {
        "value": float(f @ a + g @ b - lam * T.sum()),
        "d_a": _marginal_chain(f, a_full),
        "d_b": _marginal_chain(g, b_full),
        "d_X": 2 * (T.sum(1)[:, None] * X - T @ Y),
        "d_Y": 2 * (T.sum(0)[:, None] * Y - T.T @ X),
        "T": T, "f": f, "g": g, "iters": sol["iters"],
    }


def chain_full_to_base(d_X, N):
    """dV/dx_i = sum_k R^-k dV/dX_{k m + i} for X_{k m + i} = R^k x_i."""
    m = d_X.shape[0] // N
    out = np.zeros((m, 2))
    for k in range(N):
        R = rot2(2 * np.pi * k / N)
        out += d_X[k * m:(k + 1) * m] @ R   # (R^T g) as a row vector is g @ R
    return out


def unrolled_value_and_grad(a_base, b_base, lam, iters, C_base=None, x=None, y=None):
    """V_T and its gradient through ``iters`` log-domain iterations from z = 0 (torch float64, CPU).

    Either C_base [N, m, m] or points x, y (with N from C_base or given via
    ``x``/``y`` and the ``N`` key of C_base=None -> pass C_base or points).
    """
    import torch

    a = torch.tensor(np.asarray(a_base, np.float64), requires_grad=True)
    b = torch.tensor(np.asarray(b_base, np.float64), requires_grad=True)
    if C_base is not None:
        C = torch.tensor(np.asarray(C_base, np.float64), requires_grad=True)
        N = C.shape[0]
        leaves = {"d_a": a, "d_b": b, "d_C": C}
    else:
        raise ValueError("use unrolled_value_and_grad_points for point inputs")
    return _unrolled(a, b, C, N, lam, iters, leaves)


def unrolled_value_and_grad_points(a_base, b_base, x, y, N, lam, iters):
    import torch

    a = torch.tensor(np.asarray(a_base, np.float64), requires_grad=True)
    b = torch.tensor(np.asarray(b_base, np.float64), requires_grad=True)
    X = torch.tensor(np.asarray(x, np.float64), requires_grad=True)
    Yv = torch.tensor(np.asarray(y, np.float64), requires_grad=True)
    blocks = []
    for k in range(N):
        th = 2 * np.pi * k / N
        R = torch.tensor([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]], dtype=torch.float64)
        yk = Yv @ R.T
        blocks.append(((X[:, None, :] - yk[None, :, :]) ** 2).sum(-1))
    C = torch.stack(blocks)
    return _unrolled(a, b, C, N, lam, iters, {"d_a": a, "d_b": b, "d_x": X, "d_y": Yv})


def _unrolled(a, b, C, N, lam, iters, leaves):
    import torch

    alpha = a / (N * a.sum())
    beta = b / (N * b.sum())
    G = -lam * torch.logsumexp(-C / lam, dim=0)            # Eq. def_Kij in log form
    z = torch.zeros(C.shape[2], dtype=torch.float64)
    w = torch.zeros(C.shape[1], dtype=torch.float64)
    for _ in range(iters):
        w = lam * torch.log(alpha) - lam * torch.logsumexp((z[None, :] - G) / lam, dim=1)
        z = lam * torch.log(beta) - lam * torch.logsumexp((w[:, None] - G) / lam, dim=0)
    V = N * (w @ alpha + z @ beta) - lam
    V.backward()
    out = {"value": float(V.detach()), "w": w.detach().numpy(), "z": z.detach().numpy()}
    for k, t in leaves.items():
        out[k] = t.grad.detach().numpy().copy()
    return out


def central_difference(fun, x0, direction, h=1e-6) -> float:
    """(fun(x0 + h d) - fun(x0 - h d)) / (2h)."""
    x0 = np.asarray(x0, np.float64)
    return (fun(x0 + h * direction) - fun(x0 - h * direction)) / (2 * h)


def reduced_value(a_base, b_base, C_base, lam, tol=1e-13, max_iter=200000) -> float:
    """EROT value of the full problem computed through the reduced solve (dual, full scale)."""
    C_base = np.asarray(C_base, np.float64)
    N = C_base.shape[0]
    sol = cyclic_sinkhorn(a_base, b_base, C_base, lam, tol=tol, max_iter=max_iter)
    alpha, beta = base_marginals(a_base, b_base, N)
    T = unfold_erot(sol["w"], sol["z"], C_base, lam)
    return float(N * (sol["w"] @ alpha + sol["z"] @ beta - lam * T.sum()))
