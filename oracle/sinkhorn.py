"""Folds, cyclic Sinkhorn, plain Sinkhorn, unfolds and values -- float64.

Oracle code: test infrastructure only (see ``oracle/__init__.py``).

Notation follows the paper with this library's letters: full size n = N*m,
cyclic order N, block size m, regulariser lam (the paper's lambda).  The
inputs a_base, b_base are the base marginal blocks given with any positive
mass; they are normalised so that alpha = a_base / (N * sum(a_base)) has mass
1/N, which makes the full marginal a = (alpha; ...; alpha) a probability
vector (Assumption 1, Eq. assumption_for_input_vectors).

The iterations are the paper's scaling updates written in the log domain:
with p = exp(w/lam), q = exp(z/lam) and K = exp(-G/lam),
    p <- alpha / (K q)    is    w = lam*log(alpha) - lam*LSE_j((z_j - G_ij)/lam)
    q <- beta / (K^T p)   is    z = lam*log(beta)  - lam*LSE_i((w_i - G_ij)/lam)
(Eq. optimal_f_sinkhorn_logdomain and Eq. optimal_sinkhorn), starting from
q = 1, i.e. z = 0 (Algorithm 2).  LSE is the max-shifted log-sum-exp.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- helpers

def lse(X: np.ndarray, axis: int) -> np.ndarray:
    """log(sum(exp(X), axis)) with the maximum subtracted first."""
    mx = np.max(X, axis=axis, keepdims=True)
    mx = np.where(np.isfinite(mx), mx, 0.0)
    return np.squeeze(mx, axis=axis) + np.log(np.sum(np.exp(X - mx), axis=axis))


def normalise(v: np.ndarray) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    return v / v.sum()


def base_marginals(a_base, b_base, N):
    """alpha, beta with mass 1/N each (Assumption 1 with a, b in the simplex)."""
    return normalise(a_base) / N, normalise(b_base) / N


# ---------------------------------------------------------------- folds

def fold_min(C_base: np.ndarray):
    """Theorem 1: G_ij = min_k C_ijk (Eq. definition_G) and the smallest argmin k*.

    Returns (G, kstar) with kstar = min(argmin_k C_ijk) as Eq.
    optimal_solution_problem_CLOT prescribes (np.argmin returns the first
    occurrence, which is the smallest index).
    """
    C = np.asarray(C_base)
    return C.min(axis=0), np.argmin(C, axis=0).astype(np.uint8)


def fold_kernel(C_base: np.ndarray, lam: float) -> np.ndarray:
    """K_ij = sum_k exp(-C_ijk / lam) (Eq. def_Kij), kernel domain."""
    return np.exp(-np.asarray(C_base, np.float64) / lam).sum(axis=0)


def fold_softmin(C_base: np.ndarray, lam: float) -> np.ndarray:
    """G^eps = -lam * log K with K from Eq. def_Kij, computed as a shifted log-sum-exp.

    G^eps_ij = -lam * LSE_k(-C_ijk / lam).  The reduced EROT problem is then an
    ordinary m x m EROT on cost G^eps with marginals alpha, beta.
    """
    C = np.asarray(C_base, np.float64)
    return -lam * lse(-C / lam, axis=0)


def block_average(v: np.ndarray, N: int) -> np.ndarray:
    """Algorithm 3, Stage 1: alpha_i = (1/N) * sum_k v_{i + m k} (mass of v over N)."""
    v = np.asarray(v, np.float64)
    m = v.shape[0] // N
    return v.reshape(N, m).sum(axis=0) / N


# ---------------------------------------------------------------- Sinkhorn

def row_error_l1(f, g, M, a, lam) -> float:
    """sum_i |sum_j exp((f_i + g_j - M_ij)/lam) - a_i| (row marginal violation)."""
    r = np.exp(f / lam + lse((g[None, :] - M) / lam, axis=1))
    return float(np.abs(r - a).sum())


def _log_sinkhorn(a, b, M, lam, tol, max_iter, z0=None, err_scale=1.0, err_fn=None):
    """Alternate the two closed-form dual updates on cost M until the row L1 error <= tol.

    The error is measured after every full iteration (row update, then column
    update), so column marginals hold up to rounding and the row marginal is
    the remaining violation.  err_scale multiplies the reported error.
    """
    loga, logb = np.log(a), np.log(b)
    z = np.zeros(M.shape[1]) if z0 is None else np.array(z0, dtype=np.float64)
    w = np.zeros(M.shape[0])
    errs = []
    it = 0
    err = np.inf
    for it in range(1, max_iter + 1):
        w = lam * loga - lam * lse((z[None, :] - M) / lam, axis=1)
        z = lam * logb - lam * lse((w[:, None] - M) / lam, axis=0)
        err = err_scale * (row_error_l1(w, z, M, a, lam) if err_fn is None else err_fn(w, z))
        errs.append(err)
        if err <= tol:
            break
    return {"f": w, "g": z, "iters": it, "err": err, "errs": np.array(errs),
            "converged": bool(err <= tol)}


def sinkhorn_full(a, b, C, lam, tol=1e-9, max_iter=100000, f0=None, g0=None):
    """Plain Sinkhorn on the full n x n problem (Algorithm 3 Stage 2; Cuturi).

    a, b are normalised to unit mass; the iteration starts from g0 (default
    g = 0, i.e. q = 1).  f0 is accepted for symmetry with the warm start of
    Algorithm 3 but the first update overwrites it.  Returns potentials f, g
    (the log of the scalings times lam), iteration count and the row L1 error.
    """
    a, b = normalise(a), normalise(b)
    C = np.asarray(C, np.float64)
    return _log_sinkhorn(a, b, C, lam, tol, max_iter, z0=g0)


def cyclic_sinkhorn(a_base, b_base, C_base, lam, tol=1e-9, max_iter=100000, z0=None):
    """Algorithm 2 (cyclic Sinkhorn) in the log domain.

    K from Eq. def_Kij (here G^eps = -lam log K), then the alternating closed
    forms of Eq. optimal_f_sinkhorn_logdomain from z = 0 on marginals alpha,
    beta of mass 1/N.  The reported error is the FULL-scale row L1 error,
    N * sum_i |(S 1)_i - alpha_i|, which equals sum over the n full rows of
    |T 1 - a| for the unfolded plan.
    """
    C_base = np.asarray(C_base, np.float64)
    N = C_base.shape[0]
    alpha, beta = base_marginals(a_base, b_base, N)
    G = fold_softmin(C_base, lam)
    out = _log_sinkhorn(alpha, beta, G, lam, tol, max_iter, z0=z0, err_scale=N)
    out["w"], out["z"] = out["f"], out["g"]
    out["G"] = G
    out["alpha"], out["beta"] = alpha, beta
    return out


def two_stage_sinkhorn(a, b, C, N, lam, stage1_l2=1e-3, tol=1e-9, max_iter=100000):
    """Algorithm 3: cyclic Sinkhorn on block averages, then full Sinkhorn from tiled potentials.

    Stage 1 runs Algorithm 2's updates on alpha, beta = block averages of a, b
    (Algorithm 3's first loop) with K from the first block row of C, and stops
    once the reduced-scale L2 row error of diag(p)K diag(q) is below
    ``stage1_l2`` (App. F uses 1e-3).  Stage 2 starts the plain iteration on
    (a, b, C) from the N-fold concatenated potentials.
    """
    a, b = normalise(a), normalise(b)
    C = np.asarray(C, np.float64)
    n = C.shape[0]
    m = n // N
    alpha, beta = block_average(a, N), block_average(b, N)
    C_base = np.stack([C[0:m, k * m:(k + 1) * m] for k in range(N)])
    G = fold_softmin(C_base, lam)

    def l2_err(w, z):
        r = np.exp(w / lam + lse((z[None, :] - G) / lam, axis=1))
        return float(np.sqrt(((r - alpha) ** 2).sum()))

    s1 = _log_sinkhorn(alpha, beta, G, lam, stage1_l2, max_iter, err_fn=l2_err)
    g0 = np.tile(s1["g"], N)
    s2 = _log_sinkhorn(a, b, C, lam, tol, max_iter, z0=g0)
    s2["stage1_iters"] = s1["iters"]
    s2["stage1"] = s1
    return s2


# ---------------------------------------------------------------- unfolds and values

def unfold_erot(w, z, C_base, lam) -> np.ndarray:
    """T_ijk = exp((w_i + z_j - C_ijk)/lam) = p_i q_j exp(-C_ijk/lam).

    Algorithm 2's reconstruction loop, i.e. Theorem 2's optimality condition
    (Eq. optimality_condition) with (phi*)'(y) = exp(y/lam).  Returns the first
    block row [N, m, m]; assemble with ``rot.assemble_block_circulant``.
    """
    C = np.asarray(C_base, np.float64)
    return np.exp((w[None, :, None] + z[None, None, :] - C) / lam)


def unfold_lot(S, kstar, N) -> np.ndarray:
    """Eq. optimal_solution_problem_CLOT: T_ijk = S_ij if k = k*_ij else 0."""
    S = np.asarray(S, np.float64)
    T = np.zeros((N,) + S.shape)
    for k in range(N):
        T[k] = np.where(kstar == k, S, 0.0)
    return T


def dual_value_reduced(w, z, alpha, beta, C_base, lam) -> float:
    """N times Theorem 2's dual objective (Eq. dual_problem_cyclic_ROT) at (w, z).

    With phi*(y) = lam * exp(y/lam):  N * (<w,alpha> + <z,beta>
    - lam * sum_k sum_ij exp((w_i + z_j - C_ijk)/lam)).  The factor N turns
    the reduced objective into the full one (Sec. 5.1: the objective of Eq.
    problem_CROT is 1/N of that of Eq. problem_ROT).
    """
    N = np.asarray(C_base).shape[0]
    T = unfold_erot(w, z, C_base, lam)
    return float(N * (w @ alpha + z @ beta - lam * T.sum()))


def primal_value_reduced(T_blocks, C_base, lam) -> dict:
    """N times Eq. problem_CROT's objective, and N * sum_k <C_k, T_k> (the transport cost)."""
    from .rot import entropy_phi
    N = T_blocks.shape[0]
    C = np.asarray(C_base, np.float64)
    tc = float((C * T_blocks).sum())
    reg = float(entropy_phi(T_blocks, lam).sum())
    return {"value": N * (tc + reg), "transport_cost": N * tc}

