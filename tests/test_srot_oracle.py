"""Pins of the C-SROT oracle (squared-L2 regulariser, Sec. 5.3 / Theorem 2).

Each pin compares the oracle with something other than itself: an
optimality certificate (feasibility plus a zero primal-dual gap), the full
problem solved separately (reduced = full, Lemma 1), and scipy's general
constrained solver on a tiny instance.
"""
import numpy as np
import pytest
from scipy.optimize import minimize

from paper_2311_13147_gb300 import inputs as I
from oracle import rot as OR
from oracle import srot as SR


def test_coordinate_root_solves_its_equation():
    rng = np.random.default_rng(0)
    for _ in range(20):
        d = rng.normal(size=rng.integers(1, 40))
        t = float(rng.uniform(1e-3, 5.0))
        w = SR.coordinate_root(d, t)
        assert np.maximum(w - d, 0).sum() == pytest.approx(t, rel=1e-12)
        # the left side is strictly increasing past min d: a nudge changes it
        assert np.maximum(w + 1e-6 - d, 0).sum() > t > np.maximum(w - 1e-6 - d, 0).sum()


@pytest.mark.parametrize("m,N,seed,lam", [(6, 3, 0, 0.3), (9, 4, 1, 0.05), (5, 2, 2, 2.0)])
def test_srot_optimality_certificate(m, N, seed, lam):
    """Primal feasibility of T = (phi*)'(w + z - C) and a zero duality gap certify optimality."""
    p = I.sector_problem(m, N, seed=seed)
    C = p.C_base.astype(np.float64)
    r = SR.srot_reduced(p.a_base, p.b_base, C, lam, tol=1e-13)
    assert r["converged"]
    T = SR.srot_plan(r["w"], r["z"], C, lam)
    assert (T >= 0).all()
    assert np.abs(T.sum(axis=(0, 2)) - r["alpha"]).max() < 1e-13
    assert np.abs(T.sum(axis=(0, 1)) - r["beta"]).max() < 1e-13
    primal = SR.primal_value(T, C, lam)["value"]
    dual = SR.dual_value(r["w"], r["z"], r["alpha"], r["beta"], C, lam)
    assert primal == pytest.approx(dual, rel=1e-11, abs=1e-13)
    assert (T == 0).any()          # the quadratic regulariser gives a sparse plan


@pytest.mark.parametrize("m,N,seed", [(5, 3, 3), (8, 4, 4)])
def test_srot_reduced_equals_full(m, N, seed):
    """Lemma 1 + Theorem 2: the full problem's unique optimum is the unfolded reduced one."""
    lam = 0.2
    p = I.sector_problem(m, N, seed=seed)
    Cb = p.C_base.astype(np.float64)
    red = SR.srot_reduced(p.a_base, p.b_base, Cb, lam, tol=1e-13)
    Tb = SR.srot_plan(red["w"], red["z"], Cb, lam)
    Cf = I.full_cost_from_blocks(p.C_base).astype(np.float64)
    full = SR.srot_reduced(I.tile_marginal(p.a_base, N), I.tile_marginal(p.b_base, N), Cf[None], lam, tol=1e-13)
    Tf = SR.srot_plan(full["w"], full["z"], Cf[None], lam)[0]
    assert np.abs(OR.assemble_block_circulant(Tb) - Tf).max() < 1e-12
    assert SR.primal_value(Tb, Cb, lam)["value"] == pytest.approx(SR.primal_value(Tf[None], Cf[None], lam)["value"],
                                                                   rel=1e-11)


def test_srot_matches_general_qp_solver():
    """A tiny full problem against scipy's SLSQP on the same quadratic program."""
    lam = 0.5
    p = I.sector_problem(2, 3, seed=5)
    C = I.full_cost_from_blocks(p.C_base).astype(np.float64)
    n = C.shape[0]
    a, b = I.tile_marginal(p.a_base, 3), I.tile_marginal(p.b_base, 3)
    fun = lambda t: float((C.ravel() * t).sum() + 0.5 * lam * (t * t).sum())
    jac = lambda t: C.ravel() + lam * t
    cons = [{"type": "eq", "fun": lambda t, i=i: t.reshape(n, n)[i].sum() - a[i]} for i in range(n)]
    cons += [{"type": "eq", "fun": lambda t, j=j: t.reshape(n, n)[:, j].sum() - b[j]} for j in range(n - 1)]
    qp = minimize(fun, np.outer(a, b).ravel(), jac=jac, bounds=[(0, None)] * (n * n), constraints=cons,
                  method="SLSQP", options={"ftol": 1e-14, "maxiter": 1000})
    assert qp.success
    r = SR.srot_reduced(a, b, C[None], lam, tol=1e-13)
    v = SR.primal_value(SR.srot_plan(r["w"], r["z"], C[None], lam), C[None], lam)["value"]
    assert v == pytest.approx(qp.fun, rel=1e-7)
