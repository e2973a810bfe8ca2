"""Mirror-symmetric images (Example 1, N = 2) on the GPU against the FP64 oracle.

* a symmetric 32 x 32 pair (m = 512): fold + reduced solve, objective within
  1e-5 of the oracle's reduced solve, full-scale marginals in FP64;
* an approximately symmetric pair (5% asymmetry): the two-stage solve against
  the oracle's plain full Sinkhorn (objective within 1e-5, marginals);
* 96 x 96 (d = 9216, the paper's larger size), a symmetric pair: the reduced
  solve (the streaming route at m = 4608) and the full GPU Sinkhorn on the
  stored 9216 x 9216 cost give the same objective (Theorem 2 at full size).
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


def test_mirror_reduced_matches_oracle(cy):
    imgs = I.mirror_images(2, 32, 32, seed=11)
    p = I.mirror_problem(imgs[0], imgs[1], lam=0.5)
    m, N = p.m, 2
    tol = 1e-6
    sol = cy.cyclic_erot(dev(p.a_base), dev(p.b_base), p.eps, C_base=dev(p.C_base), tol=tol, max_iter=100000)
    assert sol.result["status"] == cy.OT_OK, sol.result
    C64 = p.C_base.astype(np.float64)
    ref = OS.cyclic_sinkhorn(p.a_base, p.b_base, C64, p.eps, tol=1e-12)
    v_ref = OS.primal_value_reduced(OS.unfold_erot(ref["w"], ref["z"], C64, p.eps), C64, p.eps)
    w, z = sol.w.cpu().numpy(), sol.z.cpu().numpy()
    Tb = OS.unfold_erot(w, z, C64, p.eps)
    v = OS.primal_value_reduced(Tb, C64, p.eps)
    assert v["value"] == pytest.approx(v_ref["value"], rel=1e-5)
    T = OR.assemble_block_circulant(Tb)
    e = OR.marginal_errors(T, I.tile_marginal(p.a_base, N), I.tile_marginal(p.b_base, N))
    assert e["row_l1"] <= tol + 2e-7 and e["col_l1"] <= 1e-6, e


def test_mirror_two_stage_matches_oracle_full(cy):
    imgs = I.mirror_images(2, 32, 32, seed=12, asym=0.05)
    p = I.mirror_problem(imgs[0], imgs[1], lam=0.5)
    n, N = 2 * p.m, 2
    C = I.full_cost_from_blocks(p.C_base)
    a32, b32 = p.meta["a_full"].astype(np.float32), p.meta["b_full"].astype(np.float32)
    tol = 1e-6
    f, g, r1, r2 = cy.two_stage(n, N, dev(a32), dev(b32), dev(C), p.eps, stage1_l2=1e-3, tol=tol)
    assert r1["status"] == cy.OT_OK and r2["status"] == cy.OT_OK, (r1, r2)
    a64, b64 = OS.normalise(a32.astype(np.float64)), OS.normalise(b32.astype(np.float64))
    C64 = C.astype(np.float64)
    ref = OS.sinkhorn_full(a64, b64, C64, p.eps, tol=1e-12)
    Tr = np.exp((ref["f"][:, None] + ref["g"][None, :] - C64) / p.eps)
    fg, gg = f.cpu().numpy(), g.cpu().numpy()
    T = np.exp((fg[:, None] + gg[None, :] - C64) / p.eps)
    assert OR.erot_primal(C64, T, p.eps) == pytest.approx(OR.erot_primal(C64, Tr, p.eps), rel=1e-5)
    e = OR.marginal_errors(T, a64, b64)
    assert e["row_l1"] <= tol + 2e-7 and e["col_l1"] <= 1e-6, e


def test_mirror_96_reduced_equals_full_on_gpu(cy):
    imgs = I.mirror_images(2, 96, 96, seed=13)
    p = I.mirror_problem(imgs[0], imgs[1], lam=0.5)
    m, N, n = p.m, 2, 2 * p.m
    tol = 1e-6
    Cb = dev(p.C_base)
    a, b = dev(p.a_base), dev(p.b_base)
    sol = cy.cyclic_erot(a, b, p.eps, C_base=Cb, tol=tol, max_iter=100000)
    assert sol.result["status"] == cy.OT_OK and sol.result["variant"] == "stream", sol.result
    vr = cy.read_result(cy.ot_value_and_grad(m, N, a, b, C_base=Cb, w=sol.w, z=sol.z, eps=p.eps))
    af = dev((np.tile(p.a_base, N) / N).astype(np.float32))
    bf = dev((np.tile(p.b_base, N) / N).astype(np.float32))
    C = dev(I.full_cost_from_blocks(p.C_base))
    f, g, rf = cy.ot_sinkhorn_full(n, af, bf, C=C, opt=cy.options(p.eps, tol=tol, max_iter=100000))
    rf = cy.read_result(rf)
    assert rf["status"] == cy.OT_OK, rf
    vf = cy.read_result(cy.ot_value_and_grad(n, 1, af, bf, C_base=C.view(1, n, n), w=f, z=g, eps=p.eps))
    assert vr["value"] == pytest.approx(vf["value"], rel=1e-5)
    assert vr["transport_cost"] == pytest.approx(vf["transport_cost"], rel=1e-5)
    # the tiled-iterates identity: both solves take the same number of sweeps (up to rounding at the stop)
    assert abs(sol.result["iters"] - rf["iters"]) <= 2, (sol.result["iters"], rf["iters"])
