"""GPU parity of the gradients (form 3): envelope and unrolled adjoints against the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_2311_13147_gb300 import inputs as I
from oracle import grad as OG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cy():
    from paper_2311_13147_gb300 import build
    build.build()
    from paper_2311_13147_gb300 import cyclicot
    return cyclicot


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-30)


@pytest.mark.parametrize("T", [1, 5, 60])
def test_unrolled_blocks_vs_oracle_autograd(cy, T):
    p = I.sector_problem(48, 4, seed=2, eps_frac=0.05)
    m, N = p.m, p.N
    Cb = dev(p.C_base)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, m, N, C_base=Cb, eps=p.eps)
    d_a, d_b = torch.empty(m, device="cuda"), torch.empty(m, device="cuda")
    d_C = torch.empty((N, m, m), device="cuda")
    out = cy.ot_value_and_grad(m, N, dev(p.a_base), dev(p.b_base), C_base=Cb, G=G, eps=p.eps,
                               adjoint=cy.OT_ADJ_UNROLLED, unroll_iters=T, d_a=d_a, d_b=d_b, d_C=d_C)
    r = cy.read_result(out)
    assert r["status"] == cy.OT_OK and r["iters"] == T
    ref = OG.unrolled_value_and_grad(p.a_base.astype(float), p.b_base.astype(float), p.eps, T,
                                     C_base=p.C_base.astype(float))
    assert r["value"] == pytest.approx(ref["value"], rel=1e-5)
    assert rel(d_a.cpu().numpy(), ref["d_a"]) < 2e-4
    assert rel(d_b.cpu().numpy(), ref["d_b"]) < 2e-4
    assert rel(d_C.cpu().numpy(), ref["d_C"]) < 2e-4


def test_unrolled_points_vs_oracle_autograd(cy):
    p = I.sector_problem(40, 8, seed=3, eps_frac=0.05)
    m, N = p.m, p.N
    x32 = p.x.astype(np.float32)
    x = dev(x32)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, m, N, x=x, y=x, eps=p.eps)
    d_x, d_y = torch.empty((m, 2), device="cuda"), torch.empty((m, 2), device="cuda")
    out = cy.ot_value_and_grad(m, N, dev(p.a_base), dev(p.b_base), x=x, y=x, G=G, eps=p.eps,
                               adjoint=cy.OT_ADJ_UNROLLED, unroll_iters=20, d_x=d_x, d_y=d_y)
    assert cy.read_result(out)["status"] == cy.OT_OK
    x64 = x32.astype(np.float64)
    ref = OG.unrolled_value_and_grad_points(p.a_base.astype(float), p.b_base.astype(float), x64, x64, N, p.eps, 20)
    g_gpu = (d_x + d_y).cpu().numpy()
    assert rel(g_gpu, ref["d_x"] + ref["d_y"]) < 5e-4


def test_unrolled_tends_to_envelope(cy):
    p = I.sector_problem(64, 4, seed=5, eps_frac=0.05)
    m, N = p.m, p.N
    Cb = dev(p.C_base)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, m, N, C_base=Cb, eps=p.eps)
    a, b = dev(p.a_base), dev(p.b_base)
    w, z, o = cy.ot_sinkhorn_reduced(m, N, a, b, G, cy.options(p.eps, tol=1e-7))
    ea, eC = torch.empty(m, device="cuda"), torch.empty((N, m, m), device="cuda")
    cy.ot_value_and_grad(m, N, a, b, C_base=Cb, w=w, z=z, eps=p.eps, d_a=ea, d_C=eC)
    ua, uC = torch.empty(m, device="cuda"), torch.empty((N, m, m), device="cuda")
    cy.ot_value_and_grad(m, N, a, b, C_base=Cb, G=G, eps=p.eps, adjoint=cy.OT_ADJ_UNROLLED, unroll_iters=300,
                         d_a=ua, d_C=uC)
    assert rel(ua.cpu().numpy(), ea.cpu().numpy()) < 1e-3
    assert rel(uC.cpu().numpy(), eC.cpu().numpy()) < 1e-3


def test_autograd_function_blocks(cy):
    from paper_2311_13147_gb300.autograd import cyclic_erot_value
    p = I.sector_problem(30, 3, seed=7, eps_frac=0.05)
    a = dev(p.a_base).requires_grad_(True)
    b = dev(p.b_base).requires_grad_(True)
    C = dev(p.C_base).requires_grad_(True)
    v = cyclic_erot_value(a, b, p.eps, C_base=C, tol=1e-7)
    (2.0 * v).backward()
    env = OG.envelope_grad(p.a_base, p.b_base, p.C_base, p.eps)
    assert float(v.detach()) == pytest.approx(env["value"], rel=1e-5)
    assert rel(a.grad.cpu().numpy(), 2 * env["d_a"]) < 1e-4
    assert rel(b.grad.cpu().numpy(), 2 * env["d_b"]) < 1e-4
    assert rel(C.grad.cpu().numpy(), 2 * env["d_C"]) < 1e-4


def test_differentiation_workload_envelope_points(cy):
    """Differentiation workload: ring points m = 1024, N = 8, cost from points on the fly.

    GPU envelope gradient vs the oracle's FP64 envelope gradient, and vs FP64
    central differences (h = 1e-6) of the oracle's value on random directions.
    """
    from paper_2311_13147_gb300.autograd import cyclic_erot_value
    p = I.sector_problem(1024, 8, seed=0, eps_frac=0.05, with_cost=False)
    x32 = p.x.astype(np.float32)
    x = dev(x32).requires_grad_(True)
    a = dev(p.a_base).requires_grad_(True)
    b = dev(p.b_base).requires_grad_(True)
    v = cyclic_erot_value(a, b, p.eps, x=x, y=x, N=8, tol=1e-7)
    v.backward()
    x64 = x32.astype(np.float64)
    C64 = OG.cost_from_points(x64, x64, 8)
    env = OG.envelope_grad(p.a_base, p.b_base, C64, p.eps, x=x64, y=x64, tol=1e-12)
    assert float(v.detach()) == pytest.approx(env["value"], rel=1e-5)
    assert rel(x.grad.cpu().numpy(), env["d_x"] + env["d_y"]) < 5e-4
    assert rel(a.grad.cpu().numpy(), env["d_a"]) < 5e-4
    rng = np.random.default_rng(0)
    for _ in range(4):
        d = rng.normal(size=x64.shape)
        fd = OG.central_difference(lambda xx: OG.reduced_value(p.a_base, p.b_base, OG.cost_from_points(xx, xx, 8),
                                                               p.eps, tol=1e-12), x64, d, h=1e-6)
        assert float((x.grad.cpu().numpy() * d).sum()) == pytest.approx(fd, rel=2e-3, abs=1e-7)


# ------------------------------------------------------------------ the differentiation workload as specified
#
# n = 8192 ring points, N = 8 (m = 1024), cost = squared Euclidean distance from the
# base points on the fly, eps = 0.05 max C (and 0.01 max C for the unrolled adjoint,
# where 200 iterations stop short of convergence).

def _diff_problem(m=1024, eps_frac=0.05):
    p = I.sector_problem(m, 8, seed=0, eps_frac=eps_frac, with_cost=False)
    x32 = p.x.astype(np.float32)
    return p, x32, x32.astype(np.float64)


def _gpu_value_grad(cy, p, x32, adjoint, unroll_iters=0, tol=1e-7):
    """Value and gradients w.r.t. (a_base, b_base, shared points) through the C ABI."""
    m, N = p.m, p.N
    x = dev(x32)
    a, b = dev(p.a_base), dev(p.b_base)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, m, N, x=x, y=x, eps=p.eps)
    d_a, d_b = torch.empty(m, device="cuda"), torch.empty(m, device="cuda")
    d_x, d_y = torch.empty((m, 2), device="cuda"), torch.empty((m, 2), device="cuda")
    if adjoint == cy.OT_ADJ_UNROLLED:
        out = cy.ot_value_and_grad(m, N, a, b, x=x, y=x, G=G, eps=p.eps, adjoint=adjoint, unroll_iters=unroll_iters,
                                   d_a=d_a, d_b=d_b, d_x=d_x, d_y=d_y)
    else:
        w, z, so = cy.ot_sinkhorn_reduced(m, N, a, b, G, cy.options(p.eps, tol=tol, max_iter=100000))
        assert cy.read_result(so)["status"] == cy.OT_OK
        out = cy.ot_value_and_grad(m, N, a, b, x=x, y=x, w=w, z=z, eps=p.eps, d_a=d_a, d_b=d_b, d_x=d_x, d_y=d_y)
    r = cy.read_result(out)
    assert r["status"] == cy.OT_OK, r
    return r, d_a.cpu().numpy(), d_b.cpu().numpy(), (d_x + d_y).cpu().numpy()


def _directions(rng, a_base, b_base, x):
    """A random direction in (a_base, b_base, x): zero-sum marginal parts scaled by the entries
    (tangent to the simplex, and a + h da stays positive), Gaussian point part."""
    a = np.asarray(a_base, np.float64)
    b = np.asarray(b_base, np.float64)
    ra, rb = rng.normal(size=a.shape), rng.normal(size=b.shape)
    da = a * (ra - (a @ ra) / a.sum())
    db = b * (rb - (b @ rb) / b.sum())
    dx = rng.normal(size=x.shape)
    return da, db, dx


@pytest.mark.parametrize("eps_frac", [0.05, 0.01])
def test_unrolled_200_differentiation_workload(cy, eps_frac):
    """Unrolled adjoint, T = 200 checkpointed iterations at m = 1024, N = 8, points: elementwise
    against the oracle's float64 autograd through the same 200 iterations (1e-3 relative)."""
    p, x32, x64 = _diff_problem(eps_frac=eps_frac)
    r, ga, gb, gx = _gpu_value_grad(cy, p, x32, cy.OT_ADJ_UNROLLED, unroll_iters=200)
    assert r["iters"] == 200
    ref = OG.unrolled_value_and_grad_points(p.a_base.astype(float), p.b_base.astype(float), x64, x64, 8, p.eps, 200)
    assert r["value"] == pytest.approx(ref["value"], rel=1e-5)
    assert rel(ga, ref["d_a"]) < 1e-3
    assert rel(gb, ref["d_b"]) < 1e-3
    assert rel(gx, ref["d_x"] + ref["d_y"]) < 1e-3


def test_envelope_fd_32_directions_differentiation_workload(cy):
    """Envelope gradient at m = 1024, N = 8 against FP64 central differences (h = 1e-6) of the
    oracle's converged value on 32 seeded directions in (a_base, b_base, x).

    Bound: the GPU gradient is within 5e-4 max|g| of the oracle's elementwise (the envelope
    tolerance), so |g_gpu . d - FD| <= 5e-4 sum_parts max|g_part| ||d_part||_1 plus the FD
    error (value to ~1e-13 at marginal L1 1e-12, divided by 2h)."""
    p, x32, x64 = _diff_problem()
    r, ga, gb, gx = _gpu_value_grad(cy, p, x32, cy.OT_ADJ_ENVELOPE)
    a64, b64 = p.a_base.astype(np.float64), p.b_base.astype(np.float64)

    def value(a, b, x):
        return OG.reduced_value(a, b, OG.cost_from_points(x, x, 8), p.eps, tol=1e-12)

    env = OG.envelope_grad(a64, b64, OG.cost_from_points(x64, x64, 8), p.eps, x=x64, y=x64, tol=1e-12)
    sa, sb, sx = np.abs(env["d_a"]).max(), np.abs(env["d_b"]).max(), np.abs(env["d_x"] + env["d_y"]).max()
    rng = np.random.default_rng(2024)
    h = 1e-6
    for _ in range(32):
        da, db, dx = _directions(rng, a64, b64, x64)
        fd = (value(a64 + h * da, b64 + h * db, x64 + h * dx) - value(a64 - h * da, b64 - h * db, x64 - h * dx)) / (2 * h)
        got = float(ga @ da + gb @ db + (gx * dx).sum())
        bound = 5e-4 * (sa * np.abs(da).sum() + sb * np.abs(db).sum() + sx * np.abs(dx).sum()) + 1e-6
        assert abs(got - fd) <= bound, (got, fd, bound)


def test_unrolled_fd_32_directions(cy):
    """Unrolled adjoint (T = 200) at m = 256, N = 8 against FP64 central differences (h = 1e-6) of
    the oracle's 200-iteration value V_T on 32 seeded directions (bound as above, with the
    unrolled tolerance 1e-3)."""
    p, x32, x64 = _diff_problem(m=256, eps_frac=0.01)
    r, ga, gb, gx = _gpu_value_grad(cy, p, x32, cy.OT_ADJ_UNROLLED, unroll_iters=200)
    a64, b64 = p.a_base.astype(np.float64), p.b_base.astype(np.float64)

    def value(a, b, x):
        return OG.unrolled_value_and_grad_points(a, b, x, x, 8, p.eps, 200)["value"]

    ref = OG.unrolled_value_and_grad_points(a64, b64, x64, x64, 8, p.eps, 200)
    sa, sb, sx = np.abs(ref["d_a"]).max(), np.abs(ref["d_b"]).max(), np.abs(ref["d_x"] + ref["d_y"]).max()
    rng = np.random.default_rng(7)
    h = 1e-6
    for _ in range(32):
        da, db, dx = _directions(rng, a64, b64, x64)
        fd = (value(a64 + h * da, b64 + h * db, x64 + h * dx) - value(a64 - h * da, b64 - h * db, x64 - h * dx)) / (2 * h)
        got = float(ga @ da + gb @ db + (gx * dx).sum())
        bound = 1e-3 * (sa * np.abs(da).sum() + sb * np.abs(db).sum() + sx * np.abs(dx).sum()) + 1e-6
        assert abs(got - fd) <= bound, (got, fd, bound)


def test_envelope_vs_full_problem_gradient_differentiation_workload(cy):
    """Envelope point gradient at m = 1024, N = 8 against the oracle's gradient of the FULL
    n = 8192 problem (plain Sinkhorn, no reduction), chained to the base points."""
    p, x32, x64 = _diff_problem()
    r, ga, gb, gx = _gpu_value_grad(cy, p, x32, cy.OT_ADJ_ENVELOPE)
    X = I.full_points(x64, 8)
    a_full = np.tile(p.a_base.astype(np.float64), 8)
    b_full = np.tile(p.b_base.astype(np.float64), 8)
    full = OG.full_problem_grad(a_full, b_full, X, X, p.eps, tol=1e-12)
    assert r["value"] == pytest.approx(full["value"], rel=1e-5)
    g_full = OG.chain_full_to_base(full["d_X"], 8) + OG.chain_full_to_base(full["d_Y"], 8)
    assert rel(gx, g_full) < 5e-4
