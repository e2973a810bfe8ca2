"""GPU parity of the batched solver (uneven m and N, one persistent launch).

Every problem of the batch is checked against the CPU FP64 oracle on the same
seeded base points: the folded cost (computed on the GPU from the points)
against the oracle's soft-min fold of the cost built in FP64 from the same
float32 points, and the potentials through the oracle's FP64 evaluation of
the marginal errors.  Block sizes include ones that are not multiples of 4
(padded rows) and one problem with a zero marginal entry (rejected on its own).

Tolerances:
* folded cost: |dG| <= 1e-6 * max C + 1e-6 * eps (FP32 distances from FP32
  coordinates and rotations, plus the soft-min correction's MUFU error);
* marginals: full-scale row L1 <= tol + 1e-6 and column L1 <= 1e-6, evaluated
  in FP64 on the oracle's cost (includes the FP32 fold error weighted by the
  plan);
* iterations within 3% (+2) of the oracle's on its own FP64 fold.
"""

import numpy as np
import pytest
import torch

from paper_2311_13147_gb300 import inputs as I
from oracle import sinkhorn as OS

pytestmark = pytest.mark.gpu

# (m, N, seed, eps_frac): several m not divisible by 4; 257 (one-warp groups), 701 (two warps)
# and 1103 (four warps) fill three float4 slots per thread and take three rows per chunk
CASES = [(37, 3, 1, 0.05), (60, 4, 0, 0.05), (130, 5, 2, 0.03), (257, 2, 3, 0.02), (11, 6, 4, 0.05),
         (401, 8, 5, 0.01), (1, 4, 6, 0.05), (203, 3, 7, 0.01), (701, 3, 8, 0.03), (1103, 2, 9, 0.03)]


@pytest.fixture(scope="module")
def cy():
    from paper_2311_13147_gb300 import build
    build.build()
    from paper_2311_13147_gb300 import cyclicot
    return cyclicot


def f32_problem(m, N, seed, frac, dirichlet=0.5):
    """A sector problem whose oracle cost is built from the float32-rounded points."""
    p = I.sector_problem(m, N, seed=seed, eps_frac=frac, dirichlet=dirichlet, with_cost=False)
    x32 = np.asarray(p.x, np.float32)
    p.x, p.y = x32, x32.copy()
    C = I.cost_blocks_from_points(x32.astype(np.float64), x32.astype(np.float64), N)
    return p, C


def oracle_marginal_errors(w, z, C, a_base, b_base, eps):
    N = C.shape[0]
    alpha, beta = OS.base_marginals(a_base, b_base, N)
    T = OS.unfold_erot(np.asarray(w, np.float64), np.asarray(z, np.float64), C, eps)
    S = T.sum(0)
    return N * np.abs(S.sum(1) - alpha).sum(), N * np.abs(S.sum(0) - beta).sum()


def test_batch_parity_mixed_sizes(cy):
    from paper_2311_13147_gb300.batch import BatchSolver
    probs, costs = zip(*[f32_problem(*c) for c in CASES])
    tol = 1e-6
    bs = BatchSolver(list(probs), tol=tol, max_iter=20000)
    bs.run()
    torch.cuda.synchronize()
    res = bs.results()
    for idx, (p, C) in enumerate(zip(probs, costs)):
        r = res[idx]
        assert r["status"] == cy.OT_OK, (p.name, r)
        assert r["marg_l1"] <= tol
        G_ref = OS.fold_softmin(C, p.eps)
        G = bs.cost(idx).cpu().numpy().astype(np.float64)
        assert np.abs(G - G_ref).max() <= 1e-6 * C.max() + 1e-6 * p.eps, p.name
        orc = OS.cyclic_sinkhorn(p.a_base, p.b_base, C, p.eps, tol=tol)
        assert abs(r["iters"] - orc["iters"]) <= 0.03 * orc["iters"] + 2, (p.name, r["iters"], orc["iters"])
        w, z = (t.cpu().numpy() for t in bs.potentials(idx))
        rl1, cl1 = oracle_marginal_errors(w, z, C, p.a_base, p.b_base, p.eps)
        assert rl1 <= tol + 1e-6 and cl1 <= 1e-6, (p.name, rl1, cl1)
        # potentials agree with the oracle's up to the dual constant (w + c, z - c)
        d = w - orc["w"]
        assert np.abs(d - d.mean()).max() <= 1e-4 * p.eps + 1e-5 * np.abs(orc["w"]).max(), p.name


def test_batch_rejects_one_problem_only(cy):
    from paper_2311_13147_gb300.batch import BatchSolver
    good, _ = f32_problem(60, 4, 0, 0.05)
    bad, _ = f32_problem(45, 3, 1, 0.05)
    bad.a_base = bad.a_base.copy()
    bad.a_base[7] = 0.0   # a zero marginal entry: log-domain potentials undefined
    bs = BatchSolver([good, bad, good], tol=1e-6)
    bs.run()
    torch.cuda.synchronize()
    res = bs.results()
    assert res[0]["status"] == cy.OT_OK and res[2]["status"] == cy.OT_OK
    assert res[1]["status"] == cy.OT_ERR_ARG
    w1, z1 = bs.potentials(1)
    assert torch.isnan(w1).all() and torch.isnan(z1).all()
    # the two copies of the good problem reach the same state
    assert res[0]["iters"] == res[2]["iters"]
    w0, _ = bs.potentials(0)
    w2, _ = bs.potentials(2)
    assert torch.allclose(w0, w2, rtol=0, atol=1e-5 * good.eps)


def test_batch_graph_replay_matches_eager(cy):
    from paper_2311_13147_gb300.batch import BatchSolver
    probs = [f32_problem(*c)[0] for c in CASES[:5]]
    bs = BatchSolver(probs, tol=1e-6)
    bs.run()
    torch.cuda.synchronize()
    eager = bs.results()
    w_e = bs.w.clone()
    bs.w.zero_()
    bs.z.zero_()
    bs.capture()
    for _ in range(2):
        bs.replay()
    torch.cuda.synchronize()
    rep = bs.results()
    for e, r in zip(eager, rep):
        assert r["status"] == cy.OT_OK
        # column sums are accumulated with unordered FP32 reductions: the state may differ by rounding
        assert abs(e["iters"] - r["iters"]) <= 1
    for idx, p in enumerate(probs):
        d = (bs.w - w_e)[bs.descs[idx].v_off:bs.descs[idx].v_off + p.m].cpu().numpy()
        assert np.abs(d - d.mean()).max() <= 1e-5 * p.eps + 1e-6


def test_batch_argument_errors(cy):
    d = [cy.ot_problem_desc(8, 4, 0.1, 6, 0, 0, 0, 8)]   # ld not a multiple of 4
    ws = torch.empty(cy.ot_batch_workspace_bytes(1, 8), dtype=torch.uint8, device="cuda")
    with pytest.raises(cy.OTError):
        cy.ot_batch_prepare(d, ws)
    d = [cy.ot_problem_desc(8, 4, 0.1, 8, 0, 0, 0, 8)]
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(cy.OTError):
        cy.ot_batch_prepare(d, small)
    assert cy.ot_batch_workspace_bytes(0, 8) == 0
    assert cy.ot_batch_workspace_bytes(2000, 8) == 0


def test_batch_autotune_and_configurations(cy):
    """Every launch configuration solves the batch; the tuner returns a valid, cached code."""
    from paper_2311_13147_gb300.batch import BatchSolver
    probs, costs = zip(*[f32_problem(*c) for c in CASES[:6]])
    tol = 1e-6
    bs = BatchSolver(list(probs), tol=tol)
    iters = {}
    for code in range(1, 7):
        bs.opt.tile_override = code
        bs.w.zero_()
        bs.z.zero_()
        bs.run()
        torch.cuda.synchronize()
        res = bs.results()
        cadence = 1 << ((code - 1) >> 1)
        for idx, r in enumerate(res):
            assert r["status"] == cy.OT_OK, (code, idx, r)
            assert r["marg_l1"] <= tol
            assert r["iters"] % cadence == 0
        iters[code] = [r["iters"] for r in res]
        w, z = (t.cpu().numpy() for t in bs.potentials(3))
        p, C = probs[3], costs[3]
        rl1, cl1 = oracle_marginal_errors(w, z, C, p.a_base, p.b_base, p.eps)
        assert rl1 <= tol + 1e-6 and cl1 <= 1e-6, (code, rl1, cl1)
    # the cadence only delays the stop to the next multiple (up to a rounding flip at the threshold)
    for code in range(1, 7):
        base = iters[1 + ((code - 1) & 1)]
        cadence = 1 << ((code - 1) >> 1)
        for a, b in zip(iters[code], base):
            assert b - 1 <= a <= b + cadence, (code, a, b)
    bs.opt.tile_override = 0
    code = bs.autotune()
    assert 1 <= code <= 6
    res = bs.results()
    assert all(r["status"] == cy.OT_OK for r in res)
    code2, _ = cy.ot_batch_autotune(bs.count, bs.total_m, bs.G, bs.a, bs.b, bs.opt, bs.w, bs.z, bs.res, bs.ws)
    assert code2 == code
    bad = cy.options(1.0, tol=tol)
    bad.tile_override = 7
    with pytest.raises(cy.OTError):
        cy.ot_batch_solve(bs.count, bs.total_m, bs.G, bs.a, bs.b, bad, bs.w, bs.z, bs.res, bs.ws)
