"""Problem definitions of regularised OT (Sec. 3.2) and Lemma 1 helpers.

Oracle code: test infrastructure only (see ``oracle/__init__.py``).
All arrays float64.
"""
from __future__ import annotations

import numpy as np


def entropy_phi(T: np.ndarray, lam: float) -> np.ndarray:
    """phi(x) = lam * x * (log x - 1) for x >= 0 (Eq. reg_for_entropy_ROT); phi(0) = 0."""
    T = np.asarray(T, dtype=np.float64)
    out = np.zeros_like(T)
    pos = T > 0
    out[pos] = lam * T[pos] * (np.log(T[pos]) - 1.0)
    if np.any(T < 0):
        out[T < 0] = np.inf
    return out


def erot_primal(C: np.ndarray, T: np.ndarray, lam: float) -> float:
    """Objective of Eq. problem_ROT with the entropic phi: <C, T> + sum phi(T_ij)."""
    return float((C * T).sum() + entropy_phi(T, lam).sum())


def transport_cost(C: np.ndarray, T: np.ndarray) -> float:
    """<C, T> (the linear part of Eq. problem_ROT; the LOT objective)."""
    return float((np.asarray(C, np.float64) * np.asarray(T, np.float64)).sum())


def marginal_errors(T: np.ndarray, a: np.ndarray, b: np.ndarray) -> dict:
    """Row / column marginal violations of Eq. problem_ROT's constraints.

    Returns the L1 row error sum_i |(T 1)_i - a_i|, the L1 column error and the
    L2 column error ||T^T 1 - b||_2 that Sec. 7.1 reports.
    """
    r = T.sum(axis=1) - a
    c = T.sum(axis=0) - b
    return {"row_l1": float(np.abs(r).sum()), "col_l1": float(np.abs(c).sum()),
            "col_l2": float(np.sqrt((c * c).sum())), "row_l2": float(np.sqrt((r * r).sum()))}


def assemble_block_circulant(blocks: np.ndarray) -> np.ndarray:
    """Lemma 1, Eq. blkstr_optimal_solution: block (r, c) of the n x n matrix is blocks[(c - r) mod N]."""
    N, m, _ = blocks.shape
    T = np.zeros((N * m, N * m), dtype=np.float64)
    for r in range(N):
        for c in range(N):
            T[r * m:(r + 1) * m, c * m:(c + 1) * m] = blocks[(c - r) % N]
    return T


def first_block_row(T: np.ndarray, N: int) -> np.ndarray:
    """T_k = T[0:m, k*m:(k+1)*m] for k = 0..N-1 (inverse of the assembly on block-circulant T)."""
    m = T.shape[0] // N
    return np.stack([T[0:m, k * m:(k + 1) * m] for k in range(N)])


def cyclic_permutation(m: int, N: int) -> np.ndarray:
    """The block permutation P of App. B (Eq. lemma_definition_P).

    P has identity blocks on the block sub-diagonal and in the top-right
    corner: block (r, c) = I_m iff r = (c + 1) mod N.
    """
    P = np.zeros((N * m, N * m))
    for c in range(N):
        r = (c + 1) % N
        P[r * m:(r + 1) * m, c * m:(c + 1) * m] = np.eye(m)
    return P


def symmetrise(T: np.ndarray, N: int) -> np.ndarray:
    """T* = (1/N) sum_k P^k T (P^k)^T (App. B, Eq. lemma_definition_T*)."""
    m = T.shape[0] // N
    P = cyclic_permutation(m, N)
    acc = np.zeros_like(T, dtype=np.float64)
    Pk = np.eye(N * m)
    for _ in range(N):
        acc += Pk @ T @ Pk.T
        Pk = P @ Pk
    return acc / N


def is_block_circulant(T: np.ndarray, N: int, atol: float = 0.0) -> bool:
    """True when P T P^T == T (up to atol), i.e. T has the structure of Eq. blkstr_optimal_solution."""
    m = T.shape[0] // N
    P = cyclic_permutation(m, N)
    return bool(np.max(np.abs(P @ T @ P.T - T)) <= atol)
