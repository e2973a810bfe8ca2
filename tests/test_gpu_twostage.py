"""Algorithm 3 (two-stage cyclic Sinkhorn) on the GPU against the oracle.

* first block row, block averages and tiling: bit-exact (a copy; an FP64 sum
  over N in block order rounded once to FP32, the same on both sides);
* the L2 row rule of Stage 1 (App. F): same iteration count as the oracle's
  Stage 1 (+-1, a rounding flip at the threshold);
* the full two-stage result on exact and on noisy (approximately symmetric)
  image-grid inputs: Stage-2 iterations within 2 of the oracle's, marginals in
  FP64 (row L1 <= tol + 2e-7, column L1 <= 1e-6) and the objective within
  1e-5 of the oracle's plain full Sinkhorn.
"""

import numpy as np
import pytest
import torch

from paper_2311_13147_gb300 import inputs as I
from oracle import rot as OR
from oracle import sinkhorn as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cy():
    from paper_2311_13147_gb300 import build
    build.build()
    from paper_2311_13147_gb300 import cyclicot
    return cyclicot


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def test_first_block_row_average_tile_exact(cy):
    rng = np.random.default_rng(0)
    m, N = 37, 5
    C = rng.uniform(0, 3, size=(m * N, m * N)).astype(np.float32)
    Cb = cy.ot_first_block_row(m, N, dev(C)).cpu().numpy()
    ref = np.stack([C[0:m, k * m:(k + 1) * m] for k in range(N)])
    assert np.array_equal(Cb, ref)
    v = rng.uniform(0, 1, size=m * N).astype(np.float32)
    av = cy.ot_block_average(m, N, dev(v)).cpu().numpy()
    ref = (v.astype(np.float64).reshape(N, m).sum(axis=0) / N).astype(np.float32)
    s = np.zeros(m)
    for k in range(N):
        s = s + v[k * m:(k + 1) * m].astype(np.float64)
    assert np.array_equal(av, (s / N).astype(np.float32))
    z = rng.standard_normal(m)
    g = cy.ot_tile_potentials(m, N, dev(z)).cpu().numpy()
    assert np.array_equal(g, np.tile(z, N))


def _full(p):
    C = I.full_cost_from_blocks(p.C_base)
    return C, np.tile(p.a_base, p.N) / p.N, np.tile(p.b_base, p.N) / p.N


@pytest.mark.parametrize("noisy", [False, True])
def test_two_stage_matches_oracle(cy, noisy):
    p = I.image_grid_problem(side=24, seed=3, eps_frac=0.02)
    C, a, b = _full(p)
    if noisy:
        rng = np.random.default_rng(5)
        a, b = I.noisy_full_marginal(rng, a), I.noisy_full_marginal(rng, b)
    a32, b32 = a.astype(np.float32), b.astype(np.float32)
    tol = 1e-6
    f, g, r1, r2 = cy.two_stage(p.n, p.N, dev(a32), dev(b32), dev(C), p.eps, stage1_l2=1e-3, tol=tol)
    assert r1["status"] == cy.OT_OK and r2["status"] == cy.OT_OK, (r1, r2)
    assert r1["marg_l1"] <= 1e-3   # the stopping norm (L2 row error at the reduced scale)
    ref = OS.two_stage_sinkhorn(a32.astype(np.float64), b32.astype(np.float64), C.astype(np.float64), p.N, p.eps,
                                stage1_l2=1e-3, tol=tol)
    assert abs(r1["iters"] - ref["stage1_iters"]) <= 1, (r1["iters"], ref["stage1_iters"])
    assert abs(r2["iters"] - ref["iters"]) <= 2, (r2["iters"], ref["iters"])
    fg, gg = f.cpu().numpy(), g.cpu().numpy()
    C64 = C.astype(np.float64)
    T = np.exp((fg[:, None] + gg[None, :] - C64) / p.eps)
    e = OR.marginal_errors(T, OS.normalise(a32), OS.normalise(b32))
    assert e["row_l1"] <= tol + 2e-7 and e["col_l1"] <= 1e-6, e
    full = OS.sinkhorn_full(a32, b32, C64, p.eps, tol=1e-12)
    Tf = np.exp((full["f"][:, None] + full["g"][None, :] - C64) / p.eps)
    assert OR.erot_primal(C64, T, p.eps) == pytest.approx(OR.erot_primal(C64, Tf, p.eps), rel=1e-5)
    if not noisy:
        # exact symmetry: Stage 1 already is the solution's tiling, so Stage 2 only polishes
        assert r2["iters"] <= ref["iters"] + 2


def test_l2_rule_on_reduced_solver(cy):
    p = I.sector_problem(60, 4, seed=0, eps_frac=0.05)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, p.m, p.N, C_base=dev(p.C_base), eps=p.eps)
    for tol in (1e-3, 1e-5):
        opt = cy.options(p.eps, tol=tol, stop_norm=cy.OT_STOP_L2_ROW)
        w, z, out = cy.ot_sinkhorn_reduced(p.m, p.N, dev(p.a_base), dev(p.b_base), G, opt)
        r = cy.read_result(out)
        assert r["status"] == cy.OT_OK and r["marg_l1"] <= tol
        alpha, beta = OS.base_marginals(p.a_base, p.b_base, p.N)
        Gr = OS.fold_softmin(p.C_base.astype(np.float64), p.eps)

        def l2(wv, zv):
            rows = np.exp(wv / p.eps + OS.lse((zv[None, :] - Gr) / p.eps, axis=1))
            return float(np.sqrt(((rows - alpha) ** 2).sum()))

        ref = OS._log_sinkhorn(alpha, beta, Gr, p.eps, tol, 100000, err_fn=l2)
        assert abs(r["iters"] - ref["iters"]) <= 1, (tol, r["iters"], ref["iters"])
        # the returned state's own L2 row error, evaluated in FP64
        assert l2(w.cpu().numpy(), z.cpu().numpy()) <= tol * 1.01 + 1e-7
    bad = cy.options(p.eps, stop_norm=7)
    with pytest.raises(cy.OTError):
        cy.ot_sinkhorn_reduced(p.m, p.N, dev(p.a_base), dev(p.b_base), G, bad)
