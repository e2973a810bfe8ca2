"""Exact linear OT at tiny sizes: a textbook transportation simplex and brute force.

Oracle code: test infrastructure only (see ``oracle/__init__.py``).

``transport_simplex`` solves  min <C, S>  s.t.  S 1 = a, S^T 1 = b, S >= 0
(Eq. problem_ROT with the regulariser of Eq. reg_for_original_OT, and the
small problem of Eq. small_problem_CLOT).  It is the primal network simplex
on the complete bipartite graph:

1. north-west-corner start: a staircase of M + N - 1 basic cells (a
   spanning tree of the bipartite graph, degenerate zeros kept basic);
2. potentials u_i + v_j = C_ij on basic cells (u_0 = 0);
3. reduced costs d_ij = C_ij - u_i - v_j; stop when all d_ij >= -tol;
4. entering cell: most negative d_ij (Dantzig), switching to Bland's
   smallest-index rule while pivots are degenerate, which excludes cycling;
5. the entering cell closes a unique cycle in the tree; flow theta moves
   round it (+ on the entering cell, alternating signs), theta = the least
   flow on a '-' cell, and one such cell leaves the basis.

It returns the plan and the optimal potentials, so callers can check the
LP certificate (primal feasibility, u_i + v_j <= C_ij, complementary
slackness) independently of the solver.
"""
from __future__ import annotations

import itertools
from collections import deque

import numpy as np


def _tree_potentials(M, N, basis, C):
    adj = [[] for _ in range(M + N)]
    for (i, j) in basis:
        adj[i].append(M + j)
        adj[M + j].append(i)
    u = np.full(M, np.nan)
    v = np.full(N, np.nan)
    u[0] = 0.0
    q = deque([0])
    seen = np.zeros(M + N, bool)
    seen[0] = True
    while q:
        x = q.popleft()
        for y in adj[x]:
            if seen[y]:
                continue
            seen[y] = True
            if x < M:           # x is row i, y is column j: v_j = C_ij - u_i
                v[y - M] = C[x, y - M] - u[x]
            else:               # x is column j, y is row i: u_i = C_ij - v_j
                u[y] = C[y, x - M] - v[x - M]
            q.append(y)
    return u, v, adj


def _tree_path(adj, src, dst, total):
    """Node path src -> dst in the basis tree (BFS parents)."""
    parent = np.full(total, -1)
    parent[src] = src
    q = deque([src])
    while q:
        x = q.popleft()
        if x == dst:
            break
        for y in adj[x]:
            if parent[y] < 0:
                parent[y] = x
                q.append(y)
    path = [dst]
    while path[-1] != src:
        path.append(parent[path[-1]])
    return path[::-1]


def transport_simplex(a, b, C, tol=1e-12, max_pivots=1_000_000, stall=20):
    a = np.asarray(a, np.float64).copy()
    b = np.asarray(b, np.float64).copy()
    C = np.asarray(C, np.float64)
    M, N = C.shape
    b *= a.sum() / b.sum()          # equal masses (feasibility of Eq. problem_ROT)
    scale = max(1.0, float(np.abs(C).max()))

    # 1. north-west corner
    S = np.zeros((M, N))
    basis = []
    s, d = a.copy(), b.copy()
    i = j = 0
    while True:
        x = min(s[i], d[j])
        S[i, j] = x
        basis.append((i, j))
        s[i] -= x
        d[j] -= x
        if i == M - 1 and j == N - 1:
            break
        if (s[i] <= d[j] and i < M - 1) or j == N - 1:
            i += 1
        else:
            j += 1
    assert len(basis) == M + N - 1
    in_basis = np.zeros((M, N), bool)
    for (i, j) in basis:
        in_basis[i, j] = True

    degenerate_run = 0
    pivots = 0
    for pivots in range(max_pivots):
        u, v, adj = _tree_potentials(M, N, basis, C)
        red = C - u[:, None] - v[None, :]
        red[in_basis] = 0.0
        neg = red < -tol * scale
        if not neg.any():
            break
        if degenerate_run >= stall:                       # Bland: smallest index
            flat = np.flatnonzero(neg.ravel())[0]
        else:                                             # Dantzig: most negative
            flat = int(np.argmin(red))
        ei, ej = divmod(int(flat), N)
        # cycle: entering (ei, ej) then the tree path from column ej back to row ei
        path = _tree_path(adj, M + ej, ei, M + N)        # nodes col ej ... row ei
        cells = []
        for k in range(len(path) - 1):
            x, y = path[k], path[k + 1]
            cells.append((y, x - M) if x >= M else (x, y - M))
        minus = cells[0::2]
        plus = cells[1::2]
        flows = np.array([S[c] for c in minus])
        theta = flows.min()
        ties = [c for c, fl in zip(minus, flows) if fl == theta]
        leave = min(ties, key=lambda c: c[0] * N + c[1]) if degenerate_run >= stall else ties[0]
        for c in minus:
            S[c] -= theta
        for c in plus:
            S[c] += theta
        S[ei, ej] += theta
        S[leave] = 0.0
        basis.remove(leave)
        in_basis[leave] = False
        basis.append((ei, ej))
        in_basis[ei, ej] = True
        degenerate_run = degenerate_run + 1 if theta == 0.0 else 0
    u, v, _ = _tree_potentials(M, N, basis, C)
    return {"S": S, "u": u, "v": v, "value": float((C * S).sum()), "pivots": pivots,
            "basis": list(basis)}


def lp_certificate(S, u, v, a, b, C, tol=1e-10) -> dict:
    """Check optimality of S for min <C,S> by LP duality, independently of any solver.

    Primal feasibility (S >= 0, marginals), dual feasibility (u_i + v_j <= C_ij)
    and a zero duality gap <C,S> - (<u,a> + <v,b>).
    """
    S, C = np.asarray(S, np.float64), np.asarray(C, np.float64)
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    b = b * a.sum() / b.sum()
    scale = max(1.0, float(np.abs(C).max()))
    primal = float((C * S).sum())
    dual = float(u @ a + v @ b)
    return {
        "nonneg": bool(S.min() >= -tol),
        "row_err": float(np.abs(S.sum(1) - a).max()),
        "col_err": float(np.abs(S.sum(0) - b).max()),
        "dual_viol": float(max(0.0, (u[:, None] + v[None, :] - C).max())) / scale,
        "gap": abs(primal - dual) / scale,
        "primal": primal,
        "dual": dual,
    }


def brute_force_uniform(C) -> float:
    """LOT with uniform marginals 1/n: by Birkhoff-von Neumann the optimum is (1/n) min_sigma sum_i C_{i sigma(i)}."""
    C = np.asarray(C, np.float64)
    n = C.shape[0]
    best = np.inf
    rows = np.arange(n)
    for perm in itertools.permutations(range(n)):
        best = min(best, C[rows, perm].sum())
    return float(best / n)


def highs_lp(a, b, C) -> dict:
    """min <C, S> s.t. S 1 = a, S^T 1 = b (b rescaled to the mass of a), S >= 0, by HiGHS.

    A library LP solver used as an independent reference for larger problems
    than ``transport_simplex`` handles; the equality constraints are assembled
    sparse (2 M N nonzeros).
    """
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    C = np.asarray(C, np.float64)
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    M, N = C.shape
    idx = np.arange(M * N)
    rows = np.concatenate([idx // N, M + idx % N])
    A = coo_matrix((np.ones(2 * M * N), (rows, np.concatenate([idx, idx]))), shape=(M + N, M * N)).tocsr()
    # solved at mass M (entries of order 1, well inside HiGHS's absolute feasibility tolerance), then rescaled
    scale = M / a.sum()
    res = linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([a * scale, b * (a.sum() * scale / b.sum())]),
                  bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(f"HiGHS: {res.message}")
    return {"value": float(res.fun) / scale, "S": res.x.reshape(M, N) / scale}
