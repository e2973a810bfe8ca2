"""GPU reduced LOT (Theorem 1's small problem by the network simplex) against the CPU oracle.

Every case is checked two independent ways:
* the LP optimality certificate of the GPU's own outputs, evaluated in FP64 on
  the host: S >= 0 with its marginals, u_i + v_j <= G_ij (dual feasibility),
  and <G, S> = <alpha, u> + <beta, v> (zero gap) -- a proof of optimality that
  does not depend on any solver;
* the optimal value of an oracle solver: the textbook transportation simplex
  (m = 60), HiGHS, linear_sum_assignment for uniform marginals (Birkhoff), or
  the closed form at m = 1.
Tolerances: S is returned in FP32 (flows are FP64 while pivoting), so the
marginals carry FP32 rounding (full-scale L1 <= 1e-6) and values agree to 1e-6
relative; the GPU pivots on integer costs rint(G 2^k) with max|G| 2^k < 2^30, so
dual violations stay below 2^-k, about 1e-9 max|G| (checked at 1e-8 (max|G| + 1)).
"""
import numpy as np
import pytest
import torch

from paper_2311_13147_gb300 import inputs as I
from oracle import lot as OL
from oracle import rot as OR
from oracle import sinkhorn as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cy():
    from paper_2311_13147_gb300 import build
    build.build()
    from paper_2311_13147_gb300 import cyclicot
    return cyclicot


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def certificate(S, u, v, alpha, beta, G):
    """FP64 LP certificate of a GPU solution (independent of any solver)."""
    S, u, v, G = (np.asarray(x, np.float64) for x in (S, u, v, G))
    scale = float(np.abs(G).max()) + 1.0
    primal = float((G * S).sum())
    dual = float(u @ alpha + v @ beta)
    return {
        "min_S": float(S.min()),
        "row_l1": float(np.abs(S.sum(1) - alpha).sum()),
        "col_l1": float(np.abs(S.sum(0) - beta).sum()),
        "dual_viol": float((u[:, None] + v[None, :] - G).max()) / scale,
        "slack": float((S * (G - u[:, None] - v[None, :])).sum()) / scale,
        "gap": abs(primal - dual) / scale,
        "primal": primal,
    }


def check_certificate(c, N, marg=1e-6):
    assert c["min_S"] >= 0.0
    assert N * c["row_l1"] <= marg and N * c["col_l1"] <= marg
    assert c["dual_viol"] <= 1e-8
    assert abs(c["slack"]) <= 1e-7 and c["gap"] <= 1e-7


def solve(cy, p, G=None, **kw):
    """Fold on the GPU (OT_MIN), then the reduced LOT; returns host copies and the record."""
    if G is None:
        G, _ = cy.ot_fold_cost(cy.OT_MIN, p.m, p.N, C_base=dev(p.C_base))
    S, u, v, out = cy.ot_lot_reduced(p.m, p.N, dev(p.a_base), dev(p.b_base), G, **kw)
    r = cy.read_lot_results(out, 1)[0]
    return host(S[0]), host(u[0]), host(v[0]), r, G


def test_tiny_matches_oracle_simplex_and_full_lp(cy):
    """n = 240, N = 4: GPU value == N x the oracle's reduced simplex == HiGHS on the full n x n LP."""
    p = I.sector_problem(60, 4, seed=0)
    S, u, v, r, G = solve(cy, p)
    assert r["status"] == cy.OT_OK and r["variant"] == "lot"
    Go, kso = OS.fold_min(p.C_base.astype(np.float64))
    alpha, beta = OS.base_marginals(p.a_base, p.b_base, p.N)
    ref = OL.transport_simplex(alpha, beta, Go)
    assert r["value"] == pytest.approx(p.N * ref["value"], rel=1e-6)
    # the dual is exact for the integer costs rint(G 2^k): within 2^-(k+1) <= 2^-30 max|G| (full scale, mass 1)
    assert abs(r["dual"] - r["value"]) <= 1e-9 * (np.abs(host(G)).max() + 1.0)
    check_certificate(certificate(S, u, v, alpha, beta, host(G)), p.N)
    # the full plan through the GPU unfold: feasible for the n x n problem, cost = the full LP value
    T = host(cy.ot_unfold_plan(cy.OT_PLAN_LOT, p.m, p.N, dev(S), kstar=cy.ot_fold_cost(
        cy.OT_MIN, p.m, p.N, C_base=dev(p.C_base))[1], dense=True))
    C = I.full_cost_from_blocks(p.C_base.astype(np.float64))
    a, b = OS.normalise(I.tile_marginal(p.a_base, p.N)), OS.normalise(I.tile_marginal(p.b_base, p.N))
    full = OL.highs_lp(a, b, C)
    assert OR.transport_cost(C, T) == pytest.approx(full["value"], rel=1e-6)
    assert np.abs(T.sum(1) - a).sum() <= 1e-6 and np.abs(T.sum(0) - b).sum() <= 1e-6


@pytest.mark.parametrize("m,N,seed", [(100, 50, 0), (200, 25, 1), (300, 10, 2)])
def test_paper_synthetic_vs_highs(cy, m, N, seed):
    """The paper's synthetic setting (Gaussian cost blocks, U[0,1) marginals)."""
    p = I.paper_synthetic_problem(m, N, seed=seed)
    S, u, v, r, G = solve(cy, p)
    assert r["status"] == cy.OT_OK
    Go, _ = OS.fold_min(p.C_base.astype(np.float64))
    alpha, beta = OS.base_marginals(p.a_base, p.b_base, p.N)
    assert r["value"] == pytest.approx(p.N * OL.highs_lp(alpha, beta, Go)["value"], rel=1e-6)
    check_certificate(certificate(S, u, v, alpha, beta, host(G)), p.N)
    assert r["marg_l1"] <= 1e-6 and r["marg_l1_col"] <= 1e-6


def test_batch_of_problems_one_launch(cy):
    """count = 3 problems of one size in one launch, each its own optimum."""
    ps = [I.paper_synthetic_problem(128, 4, seed=s) for s in range(3)]
    Gs = [cy.ot_fold_cost(cy.OT_MIN, 128, 4, C_base=dev(p.C_base))[0] for p in ps]
    G = torch.stack(Gs).contiguous()
    a = dev(np.stack([p.a_base for p in ps]))
    b = dev(np.stack([p.b_base for p in ps]))
    S, u, v, out = cy.ot_lot_reduced(128, 4, a, b, G, count=3)
    rs = cy.read_lot_results(out, 3)
    for k, p in enumerate(ps):
        assert rs[k]["status"] == cy.OT_OK
        alpha, beta = OS.base_marginals(p.a_base, p.b_base, 4)
        Go = host(G[k])
        assert rs[k]["value"] == pytest.approx(4 * OL.highs_lp(alpha, beta, Go)["value"], rel=1e-6)
        check_certificate(certificate(host(S[k]), host(u[k]), host(v[k]), alpha, beta, Go), 4)


@pytest.mark.parametrize("m,N,count", [(1000, 10, 1), (1000, 10, 20), (302, 3, 2), (2500, 2, 1), (1502, 3, 1)])
def test_cluster_pricing_matches_single_cta(cy, m, N, count):
    """Several CTAs per instance (a cluster pricing a wider block) reach the same optimum as one
    CTA per instance, with a valid certificate; m = 302 and 1502 take the scalar pricing path."""
    ps = [I.paper_synthetic_problem(m, N, seed=11 + k) for k in range(count)]
    G = torch.stack([cy.ot_fold_cost(cy.OT_MIN, m, N, C_base=dev(p.C_base))[0] for p in ps]).contiguous()
    a = dev(np.stack([p.a_base for p in ps]))
    b = dev(np.stack([p.b_base for p in ps]))
    Sc, uc, vc, oc = cy.ot_lot_reduced(m, N, a, b, G, count=count)
    Ss, us, vs, os_ = cy.ot_lot_reduced(m, N, a, b, G, count=count, single_cta=True)
    rc, rs = cy.read_lot_results(oc, count), cy.read_lot_results(os_, count)
    for k, p in enumerate(ps):
        assert rc[k]["status"] == cy.OT_OK and rs[k]["status"] == cy.OT_OK
        assert rc[k]["value"] == pytest.approx(rs[k]["value"], rel=1e-9)
        alpha, beta = OS.base_marginals(p.a_base, p.b_base, N)
        check_certificate(certificate(host(Sc[k]), host(uc[k]), host(vc[k]), alpha, beta, host(G[k])), N)


def test_cluster_wait_expires_and_reports_timeout(cy):
    """A CTA of the cluster that never hands in its candidate (fault injection on the host's
    request, no GPU fault): the owner's bounded wait expires, every CTA leaves, the status is
    OT_ERR_TIMEOUT, and the next solve on the same buffers is normal."""
    p = I.paper_synthetic_problem(1000, 10, seed=5)
    G, _ = cy.ot_fold_cost(cy.OT_MIN, p.m, p.N, C_base=dev(p.C_base))
    a, b = dev(p.a_base), dev(p.b_base)
    S, u, v, out = cy.ot_lot_reduced(p.m, p.N, a, b, G, debug_flags=cy.OT_DEBUG_WITHHOLD_ARRIVAL,
                                     timeout_ns=20_000_000)
    r = cy.read_lot_results(out, 1)[0]
    assert r["status"] == cy.OT_ERR_TIMEOUT
    S, u, v, out = cy.ot_lot_reduced(p.m, p.N, a, b, G, S=S, u=u, v=v, out=out)
    r = cy.read_lot_results(out, 1)[0]
    assert r["status"] == cy.OT_OK
    Go, _ = OS.fold_min(p.C_base.astype(np.float64))
    alpha, beta = OS.base_marginals(p.a_base, p.b_base, p.N)
    assert r["value"] == pytest.approx(p.N * OL.highs_lp(alpha, beta, Go)["value"], rel=1e-6)


@pytest.mark.parametrize("m", [64, 1000])
def test_uniform_marginals_is_assignment(cy, m):
    """Uniform marginals: by Birkhoff-von Neumann the LP optimum is an assignment (many degenerate pivots)."""
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(m)
    N = 3
    G = rng.uniform(0.0, 10.0, size=(m, m)).astype(np.float32)
    ones = np.ones(m, np.float32)
    S, u, v, out = cy.ot_lot_reduced(m, N, dev(ones), dev(ones), dev(G))
    r = cy.read_lot_results(out, 1)[0]
    assert r["status"] == cy.OT_OK
    ri, ci = linear_sum_assignment(G.astype(np.float64))
    best = float(G.astype(np.float64)[ri, ci].sum()) / m   # N * (1 / (m N)) * sum
    assert r["value"] == pytest.approx(best, rel=1e-6)
    alpha = np.full(m, 1.0 / (m * N))
    check_certificate(certificate(host(S[0]), host(u[0]), host(v[0]), alpha, alpha, G), N)


def test_zero_marginal_entries(cy):
    """Zero supplies and demands are allowed (no logarithms in the LP)."""
    p = I.paper_synthetic_problem(150, 6, seed=4)
    a = p.a_base.copy()
    b = p.b_base.copy()
    a[::7] = 0.0
    b[3::11] = 0.0
    G, _ = cy.ot_fold_cost(cy.OT_MIN, p.m, p.N, C_base=dev(p.C_base))
    S, u, v, out = cy.ot_lot_reduced(p.m, p.N, dev(a), dev(b), G)
    r = cy.read_lot_results(out, 1)[0]
    assert r["status"] == cy.OT_OK
    alpha, beta = OS.base_marginals(a, b, p.N)
    Go = host(G)
    assert r["value"] == pytest.approx(p.N * OL.highs_lp(alpha, beta, Go)["value"], rel=1e-6)
    Sg = host(S[0])
    assert np.all(Sg[a == 0.0, :] == 0.0) and np.all(Sg[:, b == 0.0] == 0.0)
    check_certificate(certificate(Sg, host(u[0]), host(v[0]), alpha, beta, Go), p.N)


def test_single_point_closed_form(cy):
    """m = 1: S = 1/N and the C-LOT value is min_k c_k (every mass goes through the cheapest block)."""
    c = np.array([[[5.0]], [[2.5]], [[7.0]]], np.float32)
    G, _ = cy.ot_fold_cost(cy.OT_MIN, 1, 3, C_base=dev(c))
    S, u, v, out = cy.ot_lot_reduced(1, 3, dev(np.ones(1)), dev(np.ones(1)), G)
    r = cy.read_lot_results(out, 1)[0]
    assert r["status"] == cy.OT_OK
    assert host(S)[0, 0, 0] == pytest.approx(1.0 / 3.0, rel=1e-7)
    assert r["value"] == pytest.approx(2.5, rel=1e-12)


@pytest.mark.parametrize("m,N", [(1024, 10), (1502, 3), (2500, 2), (5120, 2)])
def test_certificate_at_large_sizes(cy, m, N):
    """Up to the largest supported block (m = 5120; the paper's d = 10000, N = 2 has m = 5000).

    The sizes cover each pricing width (one, two and four passes of 16384 arcs) and, at
    m = 1502 (not a multiple of 4), the scalar pricing path over two passes."""
    p = I.paper_synthetic_problem(m, N, seed=7)
    S, u, v, r, G = solve(cy, p)
    assert r["status"] == cy.OT_OK
    alpha, beta = OS.base_marginals(p.a_base, p.b_base, p.N)
    c = certificate(S, u, v, alpha, beta, host(G))
    check_certificate(c, p.N)
    assert r["value"] == pytest.approx(p.N * c["primal"], rel=1e-6)   # c["primal"] from the FP32 plan
    assert abs(r["dual"] - r["value"]) <= 1e-9 * (np.abs(host(G)).max() + 1.0)
    assert np.count_nonzero(S) <= 2 * m - 1   # a basic solution


def test_argument_errors_and_status(cy):
    p = I.paper_synthetic_problem(40, 3, seed=0)
    G, _ = cy.ot_fold_cost(cy.OT_MIN, p.m, p.N, C_base=dev(p.C_base))
    bad = p.a_base.copy()
    bad[5] = -1.0
    S, u, v, out = cy.ot_lot_reduced(p.m, p.N, dev(bad), dev(p.b_base), G)
    r = cy.read_lot_results(out, 1)[0]
    assert r["status"] == cy.OT_ERR_ARG and np.isnan(host(S)).all()
    with pytest.raises(cy.OTError):
        cy.ot_lot_reduced(5121, 2, dev(np.ones(5121)), dev(np.ones(5121)), torch.zeros(1, device="cuda"))
    with pytest.raises(cy.OTError):
        cy.ot_lot_reduced(p.m, p.N, dev(p.a_base), dev(p.b_base), G, ws=torch.empty(16, dtype=torch.uint8,
                                                                                        device="cuda"))
    # a pivot cap ends the solve early: the last basis's flows, mass still on the artificial start arcs
    S, u, v, out = cy.ot_lot_reduced(p.m, p.N, dev(p.a_base), dev(p.b_base), G, max_pivots=3)
    r = cy.read_lot_results(out, 1)[0]
    assert r["status"] == cy.OT_ERR_NOT_CONVERGED and r["pivots"] == 3
    alpha, _ = OS.base_marginals(p.a_base, p.b_base, p.N)
    Sg = host(S[0])
    assert np.count_nonzero(Sg) <= 3 and Sg.min() >= 0.0
    assert r["marg_l1"] == pytest.approx(p.N * np.abs(Sg.sum(1) - alpha).sum(), rel=1e-6)
