"""Pins of the CPU FP64 oracle against what the paper and the mathematics fix.

None of these tests retypes an oracle formula: each compares the oracle with
an independent fact -- a hand-derived value (tests/golden), a closed form,
brute force, an LP certificate, an independent library solver, or an
identity the paper proves (Lemma 1, Theorems 1-2, the 1/N relation of Sec. 5.1).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2311_13147_gb300 import inputs as I
from oracle import grad as OG
from oracle import lot as OL
from oracle import rot as OR
from oracle import sinkhorn as OS

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _full(p):
    C = I.full_cost_from_blocks(p.C_base).astype(np.float64)
    return C, I.tile_marginal(p.a_base, p.N), I.tile_marginal(p.b_base, p.N)


# ------------------------------------------------------------------ folds

def test_fold_min_hand_example():
    g = _gold("lot_hand_2x2_N2.json")
    G, ks = OS.fold_min(np.array(g["C_base"], float))
    assert np.array_equal(G, np.array(g["G"], float))
    assert np.array_equal(ks, np.array(g["kstar"]))


def test_fold_min_ties_take_smallest_index():
    # Theorem 1 picks min(argmin_k); build exact ties in several positions.
    C = np.array([[[2.0, 1.0]], [[2.0, 0.5]], [[1.0, 0.5]], [[1.0, 3.0]]])  # N=4, m=1 x 2
    G, ks = OS.fold_min(C)
    assert G.tolist() == [[1.0, 0.5]]
    assert ks.tolist() == [[2, 1]]


def test_fold_softmin_hand_value():
    # K = 1 + exp(-log 3) = 4/3 for lam = 1 (Eq. def_Kij), so G = -log(4/3).
    C = np.array([[[0.0]], [[math.log(3.0)]]])
    assert OS.fold_softmin(C, 1.0)[0, 0] == pytest.approx(-math.log(4.0 / 3.0), abs=1e-15)
    assert OS.fold_kernel(C, 1.0)[0, 0] == pytest.approx(4.0 / 3.0, abs=1e-15)


def test_fold_softmin_equal_blocks_and_limits():
    rng = np.random.default_rng(1)
    c = rng.uniform(0, 2, size=(5, 7))
    lam = 0.3
    eq = np.stack([c] * 6)
    assert np.allclose(OS.fold_softmin(eq, lam), c - lam * math.log(6), atol=1e-14)
    assert np.allclose(OS.fold_softmin(c[None], lam), c, atol=1e-15)   # N = 1
    blocks = rng.uniform(0, 2, size=(4, 5, 7))
    # lam -> 0: soft-min -> min (error <= lam log N)
    G_small = OS.fold_softmin(blocks, 1e-4)
    assert np.all(G_small <= blocks.min(0) + 1e-15)
    assert np.all(G_small >= blocks.min(0) - 1e-4 * math.log(4) - 1e-15)


# ------------------------------------------------------------------ Sinkhorn pins

def test_m1_closed_form_golden():
    g = _gold("erot_m1_closed_form.json")
    N, lam = g["N"], g["lam"]
    C_base = np.array(g["c"], float).reshape(N, 1, 1)
    C = I.full_cost_from_blocks(C_base)
    a = np.full(N, 1.0 / N)
    sol = OS.sinkhorn_full(a, a, C, lam, tol=1e-14)
    T = np.exp((sol["f"][:, None] + sol["g"][None, :] - C) / lam)
    assert OR.erot_primal(C, T, lam) == pytest.approx(g["value"], abs=1e-12)
    red = OS.cyclic_sinkhorn(np.ones(1), np.ones(1), C_base, lam, tol=1e-14)
    v = OS.dual_value_reduced(red["w"], red["z"], red["alpha"], red["beta"], C_base, lam)
    assert v == pytest.approx(g["value"], abs=1e-12)


def test_tiled_iterates_exact():
    """Full Sinkhorn from q = 1 equals the tiled cyclic iterates at EVERY iteration."""
    p = I.sector_problem(12, 5, seed=3, eps_frac=0.02)
    C, a, b = _full(p)
    for iters in (1, 2, 7, 30):
        full = OS.sinkhorn_full(a, b, C, p.eps, tol=0.0, max_iter=iters)
        red = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=0.0, max_iter=iters)
        assert full["iters"] == red["iters"] == iters
        assert np.abs(full["f"] - np.tile(red["w"], p.N)).max() < 1e-13
        assert np.abs(full["g"] - np.tile(red["z"], p.N)).max() < 1e-13
        assert full["err"] == pytest.approx(red["err"], rel=1e-9, abs=1e-14)


@pytest.mark.parametrize("m,N,seed", [(6, 4, 0), (11, 3, 1), (60, 4, 0)])
def test_reduced_value_equals_full(m, N, seed):
    """Sec. 5.1 + Theorem 2: V_full = N * V_reduced(alpha, beta) = EROT_m(a_base, b_base; G^eps) - lam log N."""
    p = I.sector_problem(m, N, seed=seed, eps_frac=0.05)
    C, a, b = _full(p)
    full = OS.sinkhorn_full(a, b, C, p.eps, tol=1e-13)
    Tf = np.exp((full["f"][:, None] + full["g"][None, :] - C) / p.eps)
    v_full = OR.erot_primal(C, Tf, p.eps)
    red = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=1e-13)
    v_dual = OS.dual_value_reduced(red["w"], red["z"], red["alpha"], red["beta"], p.C_base, p.eps)
    Tb = OS.unfold_erot(red["w"], red["z"], p.C_base, p.eps)
    v_primal = OS.primal_value_reduced(Tb, p.C_base, p.eps)
    # unit-mass reduced problem on G^eps, no log N inside the fold
    G = OS.fold_softmin(p.C_base, p.eps)
    an, bn = OS.normalise(p.a_base), OS.normalise(p.b_base)
    uni = OS._log_sinkhorn(an, bn, G, p.eps, 1e-13, 100000)
    v_unit = uni["f"] @ an + uni["g"] @ bn - p.eps - p.eps * math.log(N)
    for v in (v_dual, v_primal["value"], v_unit):
        assert v == pytest.approx(v_full, rel=1e-11, abs=1e-13)
    assert v_primal["transport_cost"] == pytest.approx(OR.transport_cost(C, Tf), rel=1e-10)
    # the unfolded plan is the full optimum (Lemma 1 + Theorem 2 reconstruction)
    assert np.abs(OR.assemble_block_circulant(Tb) - Tf).max() < 1e-12


def test_N1_reduces_to_full():
    p = I.sector_problem(9, 1, seed=2, eps_frac=0.05)
    C = p.C_base[0].astype(np.float64)
    full = OS.sinkhorn_full(p.a_base, p.b_base, C, p.eps, tol=1e-13)
    red = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=1e-13)
    assert np.abs(full["f"] - red["w"]).max() < 1e-13
    assert full["iters"] == red["iters"]


def test_lemma1_from_asymmetric_start():
    """Brute force at n = 12: the full optimum reached from a random asymmetric start is block-circulant."""
    p = I.sector_problem(3, 4, seed=5, eps_frac=0.1)
    C, a, b = _full(p)
    rng = np.random.default_rng(0)
    sol = OS.sinkhorn_full(a, b, C, p.eps, tol=1e-14, g0=rng.normal(size=12))
    T = np.exp((sol["f"][:, None] + sol["g"][None, :] - C) / p.eps)
    assert OR.is_block_circulant(T, p.N, atol=1e-13)
    red = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=1e-14)
    Tr = OR.assemble_block_circulant(OS.unfold_erot(red["w"], red["z"], p.C_base, p.eps))
    assert np.abs(T - Tr).max() < 1e-12
    err = OR.marginal_errors(T, a, b)
    assert err["row_l1"] < 1e-13 and err["col_l1"] < 1e-13


def test_symmetriser_properties():
    """App. B: T* = (1/N) sum P^k T P^kT keeps the marginals of periodic a, b and is block-circulant."""
    rng = np.random.default_rng(4)
    m, N = 3, 4
    T = rng.uniform(size=(m * N, m * N))
    Ts = OR.symmetrise(T, N)
    assert OR.is_block_circulant(Ts, N, atol=1e-14)
    P = OR.cyclic_permutation(m, N)
    assert np.allclose(P @ P.T, np.eye(m * N))
    assert np.allclose(np.linalg.matrix_power(P, N), np.eye(m * N))
    # the assembled first block row reproduces the symmetrised matrix
    assert np.allclose(OR.assemble_block_circulant(OR.first_block_row(Ts, N)), Ts)
    # entropic objective does not increase (Jensen, convexity of Eq. problem_ROT's objective)
    C = I.full_cost_from_blocks(rng.uniform(size=(N, m, m)))
    assert OR.erot_primal(C, Ts / Ts.sum(), 0.2) <= OR.erot_primal(C, T / T.sum(), 0.2) + 1e-12


def test_marginals_and_nonnegativity_of_unfold():
    p = I.sector_problem(20, 6, seed=7, eps_frac=0.03)
    red = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=1e-13)
    T = OR.assemble_block_circulant(OS.unfold_erot(red["w"], red["z"], p.C_base, p.eps))
    a, b = I.tile_marginal(p.a_base, p.N), I.tile_marginal(p.b_base, p.N)
    e = OR.marginal_errors(T, a, b)
    assert T.min() >= 0
    assert e["row_l1"] < 1e-12 and e["col_l1"] < 1e-12
    assert red["err"] == pytest.approx(e["row_l1"], abs=1e-14)


def test_large_lambda_limit_is_product():
    p = I.sector_problem(8, 3, seed=1, eps_frac=1e4)
    red = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=1e-14)
    T = OR.assemble_block_circulant(OS.unfold_erot(red["w"], red["z"], p.C_base, p.eps))
    a, b = I.tile_marginal(p.a_base, p.N), I.tile_marginal(p.b_base, p.N)
    assert np.abs(T - np.outer(a, b)).max() < 1e-4 * np.outer(a, b).max()


def test_counter_example_tiling_one_block_is_not_optimal():
    """App. A: solving only the diagonal block and tiling it ignores cross-block transport."""
    p = I.image_grid_problem(side=8, seed=0, eps_frac=0.05)
    C, a, b = _full(p)
    red = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=1e-12)
    v_opt = OS.dual_value_reduced(red["w"], red["z"], red["alpha"], red["beta"], p.C_base, p.eps)
    alpha, beta = red["alpha"], red["beta"]
    naive = OS._log_sinkhorn(alpha, beta, p.C_base[0].astype(float), p.eps, 1e-12, 100000)
    T0 = np.exp((naive["f"][:, None] + naive["g"][None, :] - p.C_base[0]) / p.eps)
    blocks = np.zeros((p.N, p.m, p.m))
    blocks[0] = T0
    Tn = OR.assemble_block_circulant(blocks)      # block-diagonal copies of one block's plan
    e = OR.marginal_errors(Tn, a, b)
    assert e["row_l1"] < 1e-10 and e["col_l1"] < 1e-10   # feasible ...
    assert OR.erot_primal(C, Tn, p.eps) > v_opt + 1e-6    # ... but strictly worse


def test_two_stage_on_exact_and_noisy_inputs():
    p = I.image_grid_problem(side=8, seed=1, eps_frac=0.05)
    C, a, b = _full(p)
    ts = OS.two_stage_sinkhorn(a, b, C, p.N, p.eps, tol=1e-12)
    full = OS.sinkhorn_full(a, b, C, p.eps, tol=1e-12)
    assert np.allclose(ts["f"] - ts["f"].mean(), full["f"] - full["f"].mean(), atol=1e-9)
    rng = np.random.default_rng(2)
    an, bn = I.noisy_full_marginal(rng, a), I.noisy_full_marginal(rng, b)
    ts = OS.two_stage_sinkhorn(an, bn, C, p.N, p.eps, tol=1e-12)
    full = OS.sinkhorn_full(an, bn, C, p.eps, tol=1e-12)
    Tt = np.exp((ts["f"][:, None] + ts["g"][None, :] - C) / p.eps)
    Tf = np.exp((full["f"][:, None] + full["g"][None, :] - C) / p.eps)
    assert OR.erot_primal(C, Tt, p.eps) == pytest.approx(OR.erot_primal(C, Tf, p.eps), rel=1e-10)
    assert ts["stage1_iters"] >= 1
    # block averages carry mass 1/N (Algorithm 3's first loop)
    assert OS.block_average(an, p.N).sum() == pytest.approx(1.0 / p.N, rel=1e-14)


# ------------------------------------------------------------------ LOT

def test_lot_hand_example():
    g = _gold("lot_hand_2x2_N2.json")
    C_base = np.array(g["C_base"], float)
    G, ks = OS.fold_min(C_base)
    r = OL.transport_simplex(np.array(g["alpha"]), np.array(g["beta"]), G)
    assert r["value"] == pytest.approx(g["reduced_value"], abs=1e-15)
    assert np.allclose(r["S"], np.array(g["S_opt"]), atol=1e-15)
    C = I.full_cost_from_blocks(C_base)
    a = np.tile(g["alpha"], 2)
    b = np.tile(g["beta"], 2)
    rf = OL.transport_simplex(a, b, C)
    assert rf["value"] == pytest.approx(g["full_value"], abs=1e-14)
    T = OR.assemble_block_circulant(OS.unfold_lot(r["S"], ks, 2))
    assert OR.transport_cost(C, T) == pytest.approx(g["full_value"], abs=1e-14)


@pytest.mark.parametrize("n", [3, 5, 7])
def test_lot_brute_force_uniform(n):
    rng = np.random.default_rng(n)
    C = rng.uniform(0, 1, size=(n, n))
    u = np.full(n, 1.0 / n)
    r = OL.transport_simplex(u, u, C)
    assert r["value"] == pytest.approx(OL.brute_force_uniform(C), abs=1e-14)
    cert = OL.lp_certificate(r["S"], r["u"], r["v"], u, u, C)
    assert cert["nonneg"] and cert["row_err"] < 1e-14 and cert["col_err"] < 1e-14
    assert cert["dual_viol"] < 1e-13 and cert["gap"] < 1e-13


@pytest.mark.parametrize("m,N", [(2, 4), (3, 3), (2, 5)])
def test_clot_reduction_brute_force(m, N):
    """Theorem 1 at n <= 12 with uniform marginals: full LOT (all permutations) == reduced LOT on G."""
    rng = np.random.default_rng(m * 10 + N)
    C_base = rng.uniform(0, 1, size=(N, m, m))
    C = I.full_cost_from_blocks(C_base)
    n = m * N
    brute = OL.brute_force_uniform(C)
    G, ks = OS.fold_min(C_base)
    al = np.full(m, 1.0 / n)
    r = OL.transport_simplex(al, al, G)
    assert N * r["value"] == pytest.approx(brute, abs=1e-13)
    T = OR.assemble_block_circulant(OS.unfold_lot(r["S"], ks, N))
    assert OR.transport_cost(C, T) == pytest.approx(brute, abs=1e-13)
    e = OR.marginal_errors(T, np.full(n, 1 / n), np.full(n, 1 / n))
    assert e["row_l1"] < 1e-14 and e["col_l1"] < 1e-14


@pytest.mark.parametrize("n", [4, 6])
def test_highs_lp_pinned(n):
    """The oracle's sparse HiGHS wrapper (the reference of the GPU LOT tests) against brute force over
    permutations (uniform marginals), an assignment solver, and the oracle's own simplex on general masses."""
    pytest.importorskip("scipy")
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(100 + n)
    C = rng.uniform(0, 1, size=(n, n))
    u = np.full(n, 1.0 / n)
    h = OL.highs_lp(u, u, C)
    assert h["value"] == pytest.approx(OL.brute_force_uniform(C), abs=1e-12)
    ri, ci = linear_sum_assignment(C)
    assert h["value"] == pytest.approx(C[ri, ci].sum() / n, abs=1e-12)
    # general masses with a zero supply
    a = rng.uniform(0, 1, size=n)
    b = rng.uniform(0, 1, size=n)
    a[0] = 0.0
    a, b = a / a.sum() / 3.0, b / b.sum() / 3.0
    r = OL.transport_simplex(a, b, C)
    h = OL.highs_lp(a, b, C)
    assert h["value"] == pytest.approx(r["value"], rel=1e-9)
    assert np.abs(h["S"].sum(1) - a).max() < 1e-9 and np.abs(h["S"].sum(0) - b).max() < 1e-9


def _highs(a, b, C):
    from scipy.optimize import linprog
    M, N = C.shape
    A = np.zeros((M + N, M * N))
    for i in range(M):
        A[i, i * N:(i + 1) * N] = 1
    for j in range(N):
        A[M + j, j::N] = 1
    res = linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([a, b * a.sum() / b.sum()]),
                  bounds=(0, None), method="highs")
    return res.fun


def test_lot_tiny_config_full_vs_reduced_vs_highs():
    """The tiny workload (n = 240, N = 4): reduced LOT == full LOT == HiGHS, with certificates."""
    pytest.importorskip("scipy")
    p = I.sector_problem(60, 4, seed=0)
    C, a, b = _full(p)
    G, ks = OS.fold_min(p.C_base.astype(np.float64))
    alpha, beta = OS.base_marginals(p.a_base, p.b_base, p.N)
    r = OL.transport_simplex(alpha, beta, G)
    cr = OL.lp_certificate(r["S"], r["u"], r["v"], alpha, beta, G)
    assert cr["gap"] < 1e-13 and cr["dual_viol"] < 1e-13 and cr["nonneg"]
    rf = OL.transport_simplex(a, b, C)
    cf = OL.lp_certificate(rf["S"], rf["u"], rf["v"], a, b, C)
    assert cf["gap"] < 1e-13 and cf["dual_viol"] < 1e-13
    assert p.N * r["value"] == pytest.approx(rf["value"], rel=1e-12)
    assert r["value"] == pytest.approx(_highs(alpha, beta, G), rel=1e-9)
    T = OR.assemble_block_circulant(OS.unfold_lot(r["S"], ks, p.N))
    assert OR.transport_cost(C, T) == pytest.approx(rf["value"], rel=1e-12)


# ------------------------------------------------------------------ gradients

def test_envelope_gradient_vs_finite_differences():
    p = I.sector_problem(7, 3, seed=9, eps_frac=0.1)
    env = OG.envelope_grad(p.a_base, p.b_base, p.C_base, p.eps)
    rng = np.random.default_rng(0)
    a0 = p.a_base.astype(np.float64)
    b0 = p.b_base.astype(np.float64)
    C0 = p.C_base.astype(np.float64)
    for _ in range(4):
        d = rng.normal(size=a0.shape)
        fd = OG.central_difference(lambda v: OG.reduced_value(v, b0, C0, p.eps), a0, d, h=1e-6)
        assert env["d_a"] @ d == pytest.approx(fd, rel=1e-6, abs=1e-9)
        d = rng.normal(size=b0.shape)
        fd = OG.central_difference(lambda v: OG.reduced_value(a0, v, C0, p.eps), b0, d, h=1e-6)
        assert env["d_b"] @ d == pytest.approx(fd, rel=1e-6, abs=1e-9)
        d = rng.normal(size=C0.shape)
        fd = OG.central_difference(lambda v: OG.reduced_value(a0, b0, v, p.eps), C0, d, h=1e-6)
        assert (env["d_C"] * d).sum() == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_point_gradient_reduced_equals_full_problem_gradient():
    p = I.sector_problem(6, 4, seed=11, eps_frac=0.1)
    C_base = OG.cost_from_points(p.x, p.y, p.N)
    env = OG.envelope_grad(p.a_base, p.b_base, C_base, p.eps, x=p.x, y=p.y)
    X = I.full_points(p.x, p.N)
    Y = I.full_points(p.y, p.N)
    full = OG.full_problem_grad(np.tile(p.a_base.astype(float), p.N), np.tile(p.b_base.astype(float), p.N),
                                X, Y, p.eps)
    assert env["value"] == pytest.approx(full["value"], rel=1e-11)
    assert np.allclose(env["d_x"], OG.chain_full_to_base(full["d_X"], p.N), atol=1e-10)
    assert np.allclose(env["d_y"], OG.chain_full_to_base(full["d_Y"], p.N), atol=1e-10)
    # d/da_base through the tiling equals the per-block sum of the full gradient
    da_full = full["d_a"].reshape(p.N, p.m).sum(0)
    assert np.allclose(env["d_a"], da_full, atol=1e-10)
    # FD on the points themselves
    rng = np.random.default_rng(3)
    d = rng.normal(size=p.x.shape)

    def val(xx):
        return OG.reduced_value(p.a_base, p.b_base, OG.cost_from_points(xx, xx, p.N), p.eps)
    fd = OG.central_difference(val, p.x, d, h=1e-6)
    assert ((env["d_x"] + env["d_y"]) * d).sum() == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_unrolled_gradient_matches_fd_of_truncated_value_and_tends_to_envelope():
    p = I.sector_problem(6, 3, seed=13, eps_frac=0.1)
    a0, b0, C0 = (p.a_base.astype(float), p.b_base.astype(float), p.C_base.astype(float))
    T = 5
    un = OG.unrolled_value_and_grad(a0, b0, p.eps, T, C_base=C0)

    def vT(aa, bb, CC):
        r = OS.cyclic_sinkhorn(aa, bb, CC, p.eps, tol=0.0, max_iter=T)
        return p.N * (r["w"] @ r["alpha"] + r["z"] @ r["beta"]) - p.eps
    assert un["value"] == pytest.approx(vT(a0, b0, C0), rel=1e-13)
    rng = np.random.default_rng(5)
    d = rng.normal(size=a0.shape)
    fd = OG.central_difference(lambda v: vT(v, b0, C0), a0, d)
    assert un["d_a"] @ d == pytest.approx(fd, rel=1e-6, abs=1e-9)
    d = rng.normal(size=C0.shape)
    fd = OG.central_difference(lambda v: vT(a0, b0, v), C0, d)
    assert (un["d_C"] * d).sum() == pytest.approx(fd, rel=1e-6, abs=1e-9)
    env = OG.envelope_grad(a0, b0, C0, p.eps)
    long = OG.unrolled_value_and_grad(a0, b0, p.eps, 400, C_base=C0)
    assert np.allclose(long["d_C"], env["d_C"], atol=1e-9)
    assert np.allclose(long["d_a"], env["d_a"], atol=1e-9)
