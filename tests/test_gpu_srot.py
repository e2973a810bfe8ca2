"""C-SROT (squared-L2 regulariser, Sec. 5.3) on the GPU against the FP64 oracle.

* image-grid and sector problems: objective and transport cost within 1e-5 of
  the oracle's, the plan's marginals in FP64 (row L1 <= tol + 1e-7, column
  L1 <= 1e-6; the solver's own L1, from FP32 row sums, within 1e-7 of the FP64
  one), potentials equal up to the dual's constant;
* Theorem 2 on the GPU: the reduced solve and the plain full solve (N = 1 on
  the assembled n x n cost) give the same objective in the same number of
  sweeps (the alternating minimisation keeps symmetric iterates tiled);
* argument errors.
"""
import numpy as np
import pytest
import torch

from paper_2311_13147_gb300 import inputs as I
from oracle import srot as SR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cy():
    from paper_2311_13147_gb300 import build
    build.build()
    from paper_2311_13147_gb300 import cyclicot
    return cyclicot


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


CASES = [("grid16", lambda: I.image_grid_problem(side=16, seed=0), 10.0),
         ("sector", lambda: I.sector_problem(50, 3, seed=2), 0.3),
         ("grid24", lambda: I.image_grid_problem(side=24, seed=4), 20.0)]


@pytest.mark.parametrize("name,make,lam", CASES)
def test_srot_matches_oracle(cy, name, make, lam):
    p = make()
    lam = float(np.float32(lam))   # the boundary carries lambda in FP32 (ot_options.eps)
    tol = 1e-6
    w, z, out = cy.ot_srot_reduced(p.m, p.N, dev(p.a_base), dev(p.b_base), dev(p.C_base), lam, tol=tol)
    r = cy.read_result(out)
    assert r["status"] == cy.OT_OK and r["variant"] == "srot", r
    C64 = p.C_base.astype(np.float64)
    ref = SR.srot_reduced(p.a_base, p.b_base, C64, lam, tol=1e-11)
    Tr = SR.srot_plan(ref["w"], ref["z"], C64, lam)
    vr = SR.primal_value(Tr, C64, lam)
    assert r["value"] == pytest.approx(vr["value"], rel=1e-5)
    assert r["transport_cost"] == pytest.approx(vr["transport_cost"], rel=1e-5)
    wg, zg = w.cpu().numpy(), z.cpu().numpy()
    T = SR.srot_plan(wg, zg, C64, lam)
    assert SR.primal_value(T, C64, lam)["value"] == pytest.approx(r["value"], rel=1e-9)
    rows = np.abs(T.sum(axis=(0, 2)) - ref["alpha"]).sum() * p.N
    cols = np.abs(T.sum(axis=(0, 1)) - ref["beta"]).sum() * p.N
    assert rows <= tol + 1e-7 and cols <= 1e-6, (rows, cols)
    # the solver's own L1 sums FP32 row sums (about 1e-7 relative per row)
    assert r["marg_l1"] == pytest.approx(rows, abs=1e-7)
    shift = np.mean(wg - ref["w"])
    assert np.abs((wg - shift) - ref["w"]).max() < 1e-4 * max(1.0, np.abs(ref["w"]).max())


def test_srot_reduced_equals_full_on_gpu(cy):
    p = I.image_grid_problem(side=32, seed=1)
    lam = 40.0
    tol = 1e-6
    w, z, out = cy.ot_srot_reduced(p.m, p.N, dev(p.a_base), dev(p.b_base), dev(p.C_base), lam, tol=tol)
    r = cy.read_result(out)
    n = p.n
    Cf = I.full_cost_from_blocks(p.C_base)
    af, bf = np.tile(p.a_base, p.N), np.tile(p.b_base, p.N)
    wf, zf, outf = cy.ot_srot_reduced(n, 1, dev(af), dev(bf), dev(Cf[None]), lam, tol=tol)
    rf = cy.read_result(outf)
    assert r["status"] == cy.OT_OK and rf["status"] == cy.OT_OK, (r, rf)
    assert r["value"] == pytest.approx(rf["value"], rel=1e-5)
    assert r["transport_cost"] == pytest.approx(rf["transport_cost"], rel=1e-5)
    assert abs(r["iters"] - rf["iters"]) <= 2, (r["iters"], rf["iters"])
    # the full potentials are the tiled reduced ones (up to the dual's constant)
    wt = np.tile(w.cpu().numpy(), p.N)
    d = wf.cpu().numpy() - wt
    assert np.abs(d - d.mean()).max() < 1e-4


def test_srot_argument_errors(cy):
    x = dev(np.ones(8, np.float32))
    C = dev(np.ones((2, 8, 8), np.float32))
    with pytest.raises(cy.OTError):
        cy.ot_srot_reduced(8, 2, x, x, C, 0.0)
    with pytest.raises(cy.OTError):
        cy.srot_workspace(8192, 2, torch.device("cuda"))
    bad = dev(np.array([1, 1, 1, 0, 1, 1, 1, 1], np.float32))
    _, _, out = cy.ot_srot_reduced(8, 2, bad, x, C, 1.0)
    assert cy.read_result(out)["status"] == cy.OT_ERR_ARG


def test_srot_wide_lines_certificate_and_full(cy):
    """N m = 4400 > 4096 terms per line (the kernel keeps 32 terms per thread): the GPU's
    potentials pass the optimality certificate (FP64 marginals and a vanishing primal-dual
    gap), and the full problem (n = 4400, N = 1) gives the same objective in the same sweeps."""
    p = I.sector_problem(1100, 4, seed=7)
    lam = float(np.float32(1000.0))
    tol = 1e-6
    w, z, out = cy.ot_srot_reduced(p.m, p.N, dev(p.a_base), dev(p.b_base), dev(p.C_base), lam, tol=tol)
    r = cy.read_result(out)
    assert r["status"] == cy.OT_OK, r
    C64 = p.C_base.astype(np.float64)
    a64, b64 = np.asarray(p.a_base, np.float64), np.asarray(p.b_base, np.float64)
    alpha, beta = a64 / a64.sum() / p.N, b64 / b64.sum() / p.N
    wg, zg = w.cpu().numpy(), z.cpu().numpy()
    T = SR.srot_plan(wg, zg, C64, lam)
    rows = p.N * np.abs(T.sum(axis=(0, 2)) - alpha).sum()
    cols = p.N * np.abs(T.sum(axis=(0, 1)) - beta).sum()
    assert rows <= tol + 1e-7 and cols <= 1e-6, (rows, cols)
    primal = SR.primal_value(T, C64, lam)["value"]
    dual = SR.dual_value(wg, zg, alpha, beta, C64, lam)
    assert primal == pytest.approx(dual, rel=1e-5)
    assert r["value"] == pytest.approx(primal, rel=1e-9)
    n = p.n
    Cf = I.full_cost_from_blocks(p.C_base)
    wf, zf, outf = cy.ot_srot_reduced(n, 1, dev(np.tile(p.a_base, p.N)), dev(np.tile(p.b_base, p.N)),
                                      dev(Cf[None]), lam, tol=tol)
    rf = cy.read_result(outf)
    assert rf["status"] == cy.OT_OK, rf
    assert r["value"] == pytest.approx(rf["value"], rel=1e-5)
    assert abs(r["iters"] - rf["iters"]) <= 2, (r["iters"], rf["iters"])
