"""C-SROT with the squared-L2 regulariser: plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
bench.py's CPU baseline; never by the product path.

Problem (Eq. problem_CROT with a strongly convex regulariser, Sec. 5.3):

    min_{T_0..T_{N-1}}  sum_k <C_k, T_k> + sum_{k,i,j} phi(T_ijk)
    s.t.  sum_k T_k 1 = alpha,  sum_k T_k^T 1 = beta,

with phi(x) = (lam/2) x^2 for x >= 0 and +inf otherwise (the non-negativity of
Eq. problem_ROT), alpha = a_base / N and beta = b_base / N (mass 1/N).

phi*(y) = max(y, 0)^2 / (2 lam), (phi*)'(y) = max(y, 0) / lam.  The dual of
Theorem 2 (Eq. dual_problem_cyclic_ROT) is maximised by alternating
minimisation over w and z: each coordinate w_i solves
sum_{k,j} max(w_i + z_j - C_ijk, 0) / lam = alpha_i (Eq.
derivative_of_objective_function set to zero), a monotone piecewise-linear
equation solved here exactly by sorting its breakpoints.  The optimal plan is
T_ijk = (phi*)'(w_i + z_j - C_ijk) (Eq. optimality_condition).

Potentials follow the reduced problem's mass-1/N convention; the full-scale
objective is N times the reduced one (the remark after Eq. problem_CROT).
"""
from __future__ import annotations

import numpy as np


def phistar(y: np.ndarray, lam: float) -> np.ndarray:
    y = np.maximum(y, 0.0)
    return y * y / (2.0 * lam)


def phistar_prime(y: np.ndarray, lam: float) -> np.ndarray:
    return np.maximum(y, 0.0) / lam


def coordinate_root(d: np.ndarray, target: float) -> float:
    """The unique w with sum_l max(w - d_l, 0) = target (target > 0).

    The left side is 0 up to min d and then piecewise linear with slope p
    (the number of d_l below w) between consecutive sorted breakpoints, so on
    the piece with p active terms w = (target + sum of the p smallest d) / p.
    """
    ds = np.sort(np.asarray(d, dtype=np.float64).ravel())
    w = (target + np.cumsum(ds)) / np.arange(1, ds.size + 1)     # candidate root on each piece
    below_next = np.append(w[:-1] <= ds[1:], True)               # it lies on its piece
    return float(w[int(np.argmax(below_next))])


def srot_plan(w, z, C_base, lam) -> np.ndarray:
    """T_k[i, j] = max(w_i + z_j - C_k[i, j], 0) / lam (Eq. optimality_condition), shape [N, m, m]."""
    C = np.asarray(C_base, dtype=np.float64)
    return phistar_prime(np.asarray(w)[None, :, None] + np.asarray(z)[None, None, :] - C, lam)


def row_error_l1(w, z, C_base, alpha, lam) -> float:
    """Full-scale row marginal L1: N sum_i |sum_{k,j} T_ijk - alpha_i|."""
    T = srot_plan(w, z, C_base, lam)
    N = T.shape[0]
    return float(N * np.abs(T.sum(axis=(0, 2)) - alpha).sum())


def srot_reduced(a_base, b_base, C_base, lam, tol=1e-9, max_iter=100000, w0=None, z0=None):
    """Alternating minimisation of the dual (Theorem 2) on the reduced problem.

    One iteration updates every w_i exactly for the current z, then every z_j
    for the new w.  Stops when the full-scale row L1 of the state after the z
    update is <= tol (the column marginals then hold exactly).  For N = 1 this
    is the plain alternating minimisation of the full problem.
    """
    C = np.asarray(C_base, dtype=np.float64)
    N, m, _ = C.shape
    a = np.asarray(a_base, dtype=np.float64)
    b = np.asarray(b_base, dtype=np.float64)
    alpha = a / a.sum() / N
    beta = b / b.sum() / N
    w = np.zeros(m) if w0 is None else np.array(w0, dtype=np.float64)   # (the first w update overwrites it)
    z = np.zeros(m) if z0 is None else np.array(z0, dtype=np.float64)
    err = np.inf
    it = 0
    while it < max_iter:
        for i in range(m):
            w[i] = coordinate_root((C[:, i, :] - z[None, :]).ravel(), lam * alpha[i])
        for j in range(m):
            z[j] = coordinate_root((C[:, :, j] - w[None, :]).ravel(), lam * beta[j])
        it += 1
        err = row_error_l1(w, z, C, alpha, lam)
        if err <= tol:
            break
    return {"w": w, "z": z, "iters": it, "err": err, "alpha": alpha, "beta": beta,
            "converged": err <= tol}


def primal_value(T_blocks, C_base, lam) -> dict:
    """Full-scale primal objective N sum_k [<C_k, T_k> + sum phi(T_k)] and transport cost N sum_k <C_k, T_k>."""
    T = np.asarray(T_blocks, dtype=np.float64)
    C = np.asarray(C_base, dtype=np.float64)
    N = T.shape[0]
    tc = float((C * T).sum())
    return {"value": N * (tc + 0.5 * lam * float((T * T).sum())), "transport_cost": N * tc}


def dual_value(w, z, alpha, beta, C_base, lam) -> float:
    """Full-scale dual objective N [<w, alpha> + <z, beta> - sum phi*(w_i + z_j - C_ijk)] (Eq. dual_problem_cyclic_ROT)."""
    C = np.asarray(C_base, dtype=np.float64)
    N = C.shape[0]
    s = phistar(np.asarray(w)[None, :, None] + np.asarray(z)[None, None, :] - C, lam).sum()
    return float(N * (np.dot(w, alpha) + np.dot(z, beta) - s))
