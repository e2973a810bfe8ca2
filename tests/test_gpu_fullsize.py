"""Parity at the benchmark's full sizes, in the launch configurations bench.py times.

Where the FP64 oracle cannot process a whole workload, outputs are sampled
and recomputed one by one, or checked through properties that hold at any
size:
* image grid (m = 1024, N = 4): the graph-replayed step; bit-exact min-fold,
  sampled dense-plan entries, the plan's full marginals, the objective;
* batch (512 problems, 17.7 GB of folded cost): autotuned, graph-replayed;
  every status and L1, sampled folded entries recomputed from the points,
  the smallest problems against the FP64 oracle;
* polar (n = 65536, N = 16): the reduced path and the full on-the-fly solve
  stop after the same number of iterations (tiled iterates), the full
  potentials equal the tiled reduced ones, sampled rows' marginals in FP64;
  the value, transport cost and envelope gradients of the value-and-gradient
  call against the oracle's reduced solve at m = 4096;
* the paper's synthetic setting at d = 10000, N = 2: the same properties on
  the stored-cost paths.
"""
import math

import numpy as np
import pytest
import torch

from paper_2311_13147_gb300 import inputs as I
from oracle import grad as OG
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


def capture(body):
    body()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            body()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    return g


def test_image_grid_step_graph_replay(cy):
    p = I.image_grid_problem(side=64, seed=0, eps_frac=0.01)
    m, N, n, eps = p.m, p.N, p.n, p.eps
    Cb, a, b = dev(p.C_base), dev(p.a_base), dev(p.b_base)
    G = torch.empty((m, m), device="cuda")
    Gmin = torch.empty((m, m), device="cuda")
    ks = torch.empty((m, m), dtype=torch.uint8, device="cuda")
    w = torch.empty(m, dtype=torch.float64, device="cuda")
    z = torch.zeros(m, dtype=torch.float64, device="cuda")
    T = torch.empty((n, n), device="cuda")
    res, vres = cy.new_result("cuda"), cy.new_result("cuda")
    opt = cy.options(eps, tol=1e-6, max_iter=100000)
    ws = cy.workspace(cy.OT_OP_SINKHORN_REDUCED, m, N, torch.device("cuda"), opt)
    vws = cy.workspace(cy.OT_OP_VALUE_AND_GRAD, m, N, torch.device("cuda"))

    def body():
        cy.ot_fold_cost(cy.OT_MIN, m, N, C_base=Cb, G=Gmin, kstar=ks)
        cy.ot_fold_cost(cy.OT_SOFTMIN, m, N, C_base=Cb, eps=eps, G=G)
        cy.ot_sinkhorn_reduced(m, N, a, b, G, opt, w=w, z=z, out=res, ws=ws)
        cy.ot_unfold_plan(cy.OT_PLAN_EROT, m, N, w, z=z, C_base=Cb, eps=eps, dense=True, T=T)
        cy.ot_value_and_grad(m, N, a, b, C_base=Cb, w=w, z=z, eps=eps, out=vres, ws=vws)

    g = capture(body)
    T.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    r, rv = cy.read_result(res), cy.read_result(vres)
    assert r["status"] == cy.OT_OK and r["marg_l1"] <= 1e-6
    Gm_ref, k_ref = OS.fold_min(p.C_base)
    assert np.array_equal(Gmin.cpu().numpy(), Gm_ref) and np.array_equal(ks.cpu().numpy(), k_ref)
    ref = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=1e-12)
    Tb = OS.unfold_erot(ref["w"], ref["z"], p.C_base.astype(np.float64), p.eps)
    v = OS.primal_value_reduced(Tb, p.C_base.astype(np.float64), p.eps)
    assert rv["value"] == pytest.approx(v["value"], rel=1e-5)
    # sampled dense-plan entries, each from the oracle's own formula (block rule of Lemma 1)
    Th = T.cpu().numpy()
    wg, zg = w.cpu().numpy(), z.cpu().numpy()
    rng = np.random.default_rng(0)
    for _ in range(2000):
        R, Cc = int(rng.integers(n)), int(rng.integers(n))
        rb, i, cb, j = R // m, R % m, Cc // m, Cc % m
        k = (cb - rb) % N
        ref_e = math.exp((wg[i] + zg[j] - float(p.C_base[k, i, j])) / eps)
        assert abs(Th[R, Cc] - ref_e) <= 2e-5 * ref_e + 1e-30
    a_full = np.tile(OS.normalise(p.a_base), N) / N
    assert np.abs(Th.astype(np.float64).sum(1) - a_full).sum() <= 2e-6


def _softmin_entry(x, y, N, eps, i, j):
    cs = []
    for k in range(N):
        c, s = math.cos(2 * math.pi * k / N), math.sin(2 * math.pi * k / N)
        yk = (c * y[j, 0] - s * y[j, 1], s * y[j, 0] + c * y[j, 1])
        cs.append((x[i, 0] - yk[0]) ** 2 + (x[i, 1] - yk[1]) ** 2)
    mn = min(cs)
    return mn - eps * math.log(sum(math.exp(-(cc - mn) / eps) for cc in cs)), max(cs)


def test_batch_512_full_size(cy):
    from paper_2311_13147_gb300.batch import BatchSolver
    probs = I.batch_problems(count=512, seed=0)
    tol = 1e-6
    bs = BatchSolver(probs, tol=tol, max_iter=100000)
    bs.fold()
    bs.autotune()
    bs.capture()
    bs.w.zero_()
    bs.z.zero_()
    bs.replay()
    torch.cuda.synchronize()
    res = bs.results()
    assert all(r["status"] == cy.OT_OK for r in res)
    assert max(r["marg_l1"] for r in res) <= tol
    rng = np.random.default_rng(1)
    # sampled folded entries from the points, one by one in FP64
    for _ in range(300):
        q = int(rng.integers(len(probs)))
        p, d = probs[q], bs.descs[q]
        i, j = int(rng.integers(p.m)), int(rng.integers(p.m))
        x32 = np.asarray(p.x, np.float32).astype(np.float64)
        ref, cmax = _softmin_entry(x32, x32, p.N, p.eps, i, j)
        got = float(bs.G[d.g_off + i * d.ld + j])
        assert abs(got - ref) <= 1e-6 * p.max_cost + 1e-6 * p.eps, (q, i, j, got, ref)
    # the three smallest problems against the oracle
    order = np.argsort([p.m for p in probs])[:3]
    for q in order:
        p = probs[q]
        x32 = np.asarray(p.x, np.float32).astype(np.float64)
        C = I.cost_blocks_from_points(x32, x32, p.N)
        orc = OS.cyclic_sinkhorn(p.a_base, p.b_base, C, p.eps, tol=tol)
        assert abs(res[q]["iters"] - orc["iters"]) <= 0.03 * orc["iters"] + 2
        w, z = (t.cpu().numpy() for t in bs.potentials(q))
        alpha, beta = OS.base_marginals(p.a_base, p.b_base, p.N)
        S = OS.unfold_erot(w, z, C, p.eps).sum(0)
        assert p.N * np.abs(S.sum(1) - alpha).sum() <= tol + 1e-6
        assert p.N * np.abs(S.sum(0) - beta).sum() <= 1e-6


def test_polar_full_size(cy):
    p = I.polar_grid_problem(eps_frac=0.005)
    m, N, n, eps = p.m, p.N, p.n, p.eps
    x32 = np.asarray(p.x, np.float32)
    X32 = I.full_points(x32.astype(np.float64), N).astype(np.float32)
    tol = 1e-6
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, m, N, x=dev(x32), y=dev(x32), eps=eps)
    w, z, out = cy.ot_sinkhorn_reduced(m, N, dev(p.a_base), dev(p.b_base), G, cy.options(eps, tol=tol, max_iter=5000))
    r = cy.read_result(out)
    assert r["status"] == cy.OT_OK
    a_full = (np.tile(p.a_base, N) / N).astype(np.float32)
    b_full = (np.tile(p.b_base, N) / N).astype(np.float32)
    f, g, fout = cy.ot_sinkhorn_full(n, dev(a_full), dev(b_full), X=dev(X32), Y=dev(X32),
                                     opt=cy.options(eps, tol=tol, max_iter=2 * r["iters"] + 50))
    rf = cy.read_result(fout)
    assert rf["status"] == cy.OT_OK
    assert abs(rf["iters"] - r["iters"]) <= 2, (rf["iters"], r["iters"])   # tiled iterates
    fg, gg = f.cpu().numpy(), g.cpu().numpy()
    wt = np.tile(w.cpu().numpy() + eps * math.log(N), N)
    d = fg - wt
    assert np.abs(d - d.mean()).max() <= 5e-5 * max(1.0, np.abs(wt).max())
    # sampled full rows: marginal in FP64 from the GPU potentials and the exact cost of the FP32 points
    rng = np.random.default_rng(2)
    X64 = X32.astype(np.float64)
    an = OS.normalise(a_full)
    err = 0.0
    for R in rng.integers(0, n, size=64):
        c = ((X64[R][None, :] - X64) ** 2).sum(1)
        row = np.exp((fg[R] + gg - c) / eps).sum()
        err = max(err, abs(row - an[R]) / an[R])
    assert err <= 1e-3   # per-row relative error of a state with full-scale L1 <= 1e-6 on 65536 rows
    # the value-and-gradient call of the workload, against the oracle's reduced solve at m = 4096
    # (same tolerance, hence the same iteration) and its envelope gradients from the same state
    xd = dev(x32)
    d_a, d_b = torch.empty(m, device="cuda"), torch.empty(m, device="cuda")
    d_x, d_y = torch.empty((m, 2), device="cuda"), torch.empty((m, 2), device="cuda")
    vout = cy.ot_value_and_grad(m, N, dev(p.a_base), dev(p.b_base), x=xd, y=xd, w=w, z=z, eps=eps,
                                d_a=d_a, d_b=d_b, d_x=d_x, d_y=d_y)
    rv = cy.read_result(vout)
    assert rv["status"] == cy.OT_OK
    x64 = x32.astype(np.float64)
    C64 = OG.cost_from_points(x64, x64, N)
    env = OG.envelope_grad(p.a_base, p.b_base, C64, eps, tol=tol, x=x64, y=x64)
    assert abs(env["iters"] - r["iters"]) <= 2, (env["iters"], r["iters"])
    v = OS.primal_value_reduced(OS.unfold_erot(env["w"], env["z"], C64, eps), C64, eps)
    del C64
    assert rv["value"] == pytest.approx(v["value"], rel=1e-5)
    assert rv["transport_cost"] == pytest.approx(v["transport_cost"], rel=1e-5)
    rel = lambda g, ref: np.abs(g - ref).max() / np.abs(ref).max()
    assert rel(d_a.cpu().numpy(), env["d_a"]) < 5e-4
    assert rel(d_b.cpu().numpy(), env["d_b"]) < 5e-4
    assert rel((d_x + d_y).cpu().numpy(), env["d_x"] + env["d_y"]) < 5e-4


def test_paper_setting_d10000_n2(cy):
    p = I.paper_synthetic_problem(5000, 2, seed=0)
    m, N, n, eps = p.m, p.N, p.n, p.eps
    tol = 1e-6
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, m, N, C_base=dev(p.C_base), eps=eps)
    w, z, out = cy.ot_sinkhorn_reduced(m, N, dev(p.a_base), dev(p.b_base), G, cy.options(eps, tol=tol, max_iter=20000))
    r = cy.read_result(out)
    assert r["status"] == cy.OT_OK and r["variant"] == "stream"
    C = I.full_cost_from_blocks(p.C_base)
    a_full = (np.tile(p.a_base, N) / N).astype(np.float32)
    b_full = (np.tile(p.b_base, N) / N).astype(np.float32)
    f, g, fout = cy.ot_sinkhorn_full(n, dev(a_full), dev(b_full), C=dev(C), opt=cy.options(eps, tol=tol, max_iter=20000))
    rf = cy.read_result(fout)
    assert rf["status"] == cy.OT_OK
    assert abs(rf["iters"] - r["iters"]) <= 0.03 * r["iters"] + 2, (rf["iters"], r["iters"])
    # potentials of near-zero-mass rows are barely determined (U[0, 1) marginals); the dual
    # objective is: full N (<w, alpha> + <z, beta>) - eps on the reduced side, <f, a> + <g, b> - eps
    fg, gg = f.cpu().numpy(), g.cpu().numpy()
    alpha, beta = OS.base_marginals(p.a_base, p.b_base, N)
    v_red = N * (float(np.dot(w.cpu().numpy(), alpha)) + float(np.dot(z.cpu().numpy(), beta))) - eps
    v_full = float(np.dot(fg, OS.normalise(a_full))) + float(np.dot(gg, OS.normalise(b_full))) - eps
    assert v_red == pytest.approx(v_full, rel=1e-5)
