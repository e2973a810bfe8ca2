"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle.

Tolerances, each derived from the arithmetic on both sides:
* LOT min-fold, kstar and the unfold index map: bit-exact.
* EROT objective (regularised value and transport cost): 1e-5 relative.
* Marginals: the oracle evaluates the GPU's potentials in FP64; the full-scale
  row L1 error must be <= the requested tolerance plus 2e-7 and the column L1
  (exact by construction up to rounding) <= 1e-6.
* Folded cost G^eps: |dG| <= 4e-7 * max|G| + 1e-6 * eps (FP32 rounding of the
  min plus MUFU log2/exp2 error times eps).
"""
import math

import numpy as np
import pytest
import torch

from paper_2311_13147_gb300 import inputs as I
from oracle import grad as OG
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


def dev(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def fp64_row_col_errors(w, z, C_base, a_base, b_base, eps):
    """Oracle-side FP64 marginal errors of the plan defined by (w, z) (mass 1/N convention)."""
    N = C_base.shape[0]
    alpha, beta = OS.base_marginals(a_base, b_base, N)
    T = OS.unfold_erot(np.asarray(w, np.float64), np.asarray(z, np.float64), C_base.astype(np.float64), eps)
    S = T.sum(0)
    return N * np.abs(S.sum(1) - alpha).sum(), N * np.abs(S.sum(0) - beta).sum()


SIZES = [(60, 4, 0), (37, 3, 1), (130, 5, 2), (257, 2, 3)]


# ------------------------------------------------------------------ folds

@pytest.mark.parametrize("m,N,seed", SIZES + [(1, 7, 4), (1024, 4, 5)])
def test_fold_min_bit_exact(cy, m, N, seed):
    p = I.sector_problem(m, N, seed=seed)
    G, ks = cy.ot_fold_cost(cy.OT_MIN, m, N, C_base=dev(p.C_base))
    Go, kso = OS.fold_min(p.C_base)
    assert np.array_equal(host(G), Go.astype(np.float32))
    assert np.array_equal(host(ks), kso)


def test_fold_min_ties_and_grid_ties(cy):
    # the image grid has exact ties between rotated blocks; kstar must take the smallest index
    p = I.image_grid_problem(side=16, seed=0)
    G, ks = cy.ot_fold_cost(cy.OT_MIN, p.m, p.N, C_base=dev(p.C_base))
    Go, kso = OS.fold_min(p.C_base)
    assert np.array_equal(host(G), Go.astype(np.float32))
    assert np.array_equal(host(ks), kso)
    # scalar (unaligned) path: m*m not a multiple of 4
    p = I.sector_problem(7, 5, seed=1)
    G, ks = cy.ot_fold_cost(cy.OT_MIN, 7, 5, C_base=dev(p.C_base))
    Go, kso = OS.fold_min(p.C_base)
    assert np.array_equal(host(G), Go.astype(np.float32)) and np.array_equal(host(ks), kso)


@pytest.mark.parametrize("m,N,seed", SIZES + [(1024, 4, 5)])
def test_fold_softmin_stored(cy, m, N, seed):
    p = I.sector_problem(m, N, seed=seed, eps_frac=0.01)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, m, N, C_base=dev(p.C_base), eps=p.eps)
    Go = OS.fold_softmin(p.C_base.astype(np.float64), p.eps)
    err = np.abs(host(G) - Go).max()
    assert err <= 4e-7 * np.abs(Go).max() + 1e-6 * p.eps, err


@pytest.mark.parametrize("m,N,seed", [(60, 4, 0), (33, 8, 1), (1024, 8, 2), (100, 3, 3), (300, 16, 4), (150, 11, 5)])
def test_fold_from_points(cy, m, N, seed):
    """Column-strip folds for N <= 16 (4, 8 or 16 blocks per pass; N = 3 and 11 pad the last pair)."""
    p = I.sector_problem(m, N, seed=seed, eps_frac=0.05)
    x = dev(p.x.astype(np.float32))
    for mode in (cy.OT_SOFTMIN, cy.OT_MIN):
        G, ks = cy.ot_fold_cost(mode, m, N, x=x, y=x, eps=p.eps)
        Cb = OG.cost_from_points(p.x.astype(np.float32).astype(np.float64), p.x.astype(np.float32).astype(np.float64), N)
        Go = OS.fold_softmin(Cb, p.eps) if mode == cy.OT_SOFTMIN else Cb.min(0)
        # FP32 rotation and distance: a few ulp of max C
        assert np.abs(host(G) - Go).max() <= 2e-6 * p.max_cost


# ------------------------------------------------------------------ reduced / full Sinkhorn

def _solve_reduced(cy, p, tol, max_iter=20000):
    Cb = dev(p.C_base)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, p.m, p.N, C_base=Cb, eps=p.eps)
    opt = cy.options(p.eps, tol=tol, max_iter=max_iter)
    w, z, out = cy.ot_sinkhorn_reduced(p.m, p.N, dev(p.a_base), dev(p.b_base), G, opt)
    return Cb, G, w, z, cy.read_result(out)


@pytest.mark.parametrize("m,N,seed,frac", [(60, 4, 0, 0.05), (37, 3, 1, 0.02), (130, 5, 2, 0.01), (257, 2, 3, 0.01)])
def test_reduced_sinkhorn_parity(cy, m, N, seed, frac):
    p = I.sector_problem(m, N, seed=seed, eps_frac=frac)
    tol = 1e-6
    Cb, G, w, z, res = _solve_reduced(cy, p, tol)
    assert res["status"] == cy.OT_OK, res
    assert res["marg_l1"] <= tol
    orc = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=tol)
    # same iteration (identical stopping rule), up to a rounding flip at the threshold
    assert abs(res["iters"] - orc["iters"]) <= 1, (res["iters"], orc["iters"])
    wg, zg = host(w), host(z)
    rl1, cl1 = fp64_row_col_errors(wg, zg, p.C_base, p.a_base, p.b_base, p.eps)
    assert rl1 <= tol + 2e-7 and cl1 <= 1e-6, (rl1, cl1)
    # objective through the value kernel vs the oracle's value at its own converged state
    out = cy.ot_value_and_grad(m, N, dev(p.a_base), dev(p.b_base), C_base=Cb, w=w, z=z, eps=p.eps)
    r = cy.read_result(out)
    ref = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=1e-13)
    Tb = OS.unfold_erot(ref["w"], ref["z"], p.C_base.astype(np.float64), p.eps)
    v = OS.primal_value_reduced(Tb, p.C_base.astype(np.float64), p.eps)
    assert r["value"] == pytest.approx(v["value"], rel=1e-5)
    assert r["transport_cost"] == pytest.approx(v["transport_cost"], rel=1e-5)
    # potentials agree up to the dual constant
    d = (wg - ref["w"])
    assert np.abs(d - d.mean()).max() <= 1e-5 * max(1.0, np.abs(ref["w"]).max()) + 10 * p.eps * 1e-6


def test_reduced_image_grid_parity(cy):
    """The image-grid workload (64x64, N = 4, m = 1024) at eps = 0.01 max C to 1e-6."""
    p = I.image_grid_problem(side=64, seed=0, eps_frac=0.01)
    tol = 1e-6
    Cb, G, w, z, res = _solve_reduced(cy, p, tol)
    assert res["status"] == cy.OT_OK, res
    orc = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=tol)
    assert abs(res["iters"] - orc["iters"]) <= 2, (res["iters"], orc["iters"])
    rl1, cl1 = fp64_row_col_errors(host(w), host(z), p.C_base, p.a_base, p.b_base, p.eps)
    assert rl1 <= tol + 3e-7 and cl1 <= 1e-6, (rl1, cl1)
    out = cy.ot_value_and_grad(p.m, p.N, dev(p.a_base), dev(p.b_base), C_base=Cb, w=w, z=z, eps=p.eps)
    r = cy.read_result(out)
    Tb = OS.unfold_erot(orc["w"], orc["z"], p.C_base.astype(np.float64), p.eps)
    v = OS.primal_value_reduced(Tb, p.C_base.astype(np.float64), p.eps)
    assert r["value"] == pytest.approx(v["value"], rel=1e-5)
    assert r["transport_cost"] == pytest.approx(v["transport_cost"], rel=1e-5)


@pytest.mark.parametrize("m,N,seed", [(60, 4, 0), (11, 5, 1), (300, 3, 2)])
def test_full_sinkhorn_stored_parity_and_tiling(cy, m, N, seed):
    p = I.sector_problem(m, N, seed=seed, eps_frac=0.02)
    C = I.full_cost_from_blocks(p.C_base)
    a = np.tile(p.a_base, N)
    b = np.tile(p.b_base, N)
    tol = 1e-6
    opt = cy.options(p.eps, tol=tol)
    f, g, out = cy.ot_sinkhorn_full(p.n, dev(a), dev(b), C=dev(C), opt=opt)
    res = cy.read_result(out)
    assert res["status"] == cy.OT_OK
    ref = OS.sinkhorn_full(a, b, C.astype(np.float64), p.eps, tol=tol)
    assert abs(res["iters"] - ref["iters"]) <= 1
    # the same iterations as the reduced solve (tiled-iterates identity)
    _, _, w, z, rr = _solve_reduced(cy, p, tol)
    assert abs(rr["iters"] - res["iters"]) <= 1
    fg, gg = host(f), host(g)
    wt = np.tile(host(w) + p.eps * math.log(N), N)   # unit-mass row potential
    d = fg - wt
    assert np.abs(d - d.mean()).max() <= 2e-5 * max(1.0, np.abs(wt).max())
    T = np.exp((fg[:, None] + gg[None, :] - C.astype(np.float64)) / p.eps)
    e = OR.marginal_errors(T, OS.normalise(a), OS.normalise(b))
    assert e["row_l1"] <= tol + 2e-7 and e["col_l1"] <= 1e-6


@pytest.mark.parametrize("n,seed", [(64, 0), (300, 1), (5000, 2)])
def test_full_sinkhorn_points_on_the_fly(cy, n, seed):
    """Two-pass kernel, cost computed from coordinates (never stored)."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, size=(n, 2)).astype(np.float32)
    Y = rng.uniform(0, 1, size=(n, 2)).astype(np.float32)
    a = rng.dirichlet(np.ones(n)).astype(np.float32) + 1e-6
    b = rng.dirichlet(np.ones(n)).astype(np.float32) + 1e-6
    eps = 0.02 * 2.0
    tol = 1e-6
    f, g, out = cy.ot_sinkhorn_full(n, dev(a), dev(b), X=dev(X), Y=dev(Y), opt=cy.options(eps, tol=tol))
    res = cy.read_result(out)
    assert res["status"] == cy.OT_OK, res
    if n <= 600:
        C = ((X[:, None, :].astype(np.float64) - Y[None, :, :]) ** 2).sum(-1)
        ref = OS.sinkhorn_full(a, b, C, eps, tol=tol)
        assert abs(res["iters"] - ref["iters"]) <= 1
        T = np.exp((host(f)[:, None] + host(g)[None, :] - C) / eps)
        e = OR.marginal_errors(T, OS.normalise(a), OS.normalise(b))
        assert e["row_l1"] <= tol + 2e-7 and e["col_l1"] <= 1e-6
    else:
        # sampled rows: FP64 row marginals of the GPU potentials on 64 rows
        fg, gg = host(f), host(g)
        rows = rng.choice(n, 64, replace=False)
        C = ((X[rows, None, :].astype(np.float64) - Y[None, :, :]) ** 2).sum(-1)
        r = np.exp((fg[rows, None] + gg[None, :] - C) / eps).sum(1)
        an = OS.normalise(a)[rows]
        assert np.abs(r - an).sum() <= 64 / n * 10 * tol + 1e-7


# ------------------------------------------------------------------ unfold

def test_unfold_lot_bit_exact(cy):
    p = I.sector_problem(60, 4, seed=0)
    G, ks = cy.ot_fold_cost(cy.OT_MIN, 60, 4, C_base=dev(p.C_base))
    Go, kso = OS.fold_min(p.C_base.astype(np.float64))
    alpha, beta = OS.base_marginals(p.a_base, p.b_base, 4)
    S = OL.transport_simplex(alpha, beta, Go)["S"].astype(np.float32)
    Sd = dev(S)
    Tc = cy.ot_unfold_plan(cy.OT_PLAN_LOT, 60, 4, Sd, kstar=ks)
    To = OS.unfold_lot(S.astype(np.float64), kso, 4).astype(np.float32)
    assert np.array_equal(host(Tc), To)
    Td = cy.ot_unfold_plan(cy.OT_PLAN_LOT, 60, 4, Sd, kstar=ks, dense=True)
    assert np.array_equal(host(Td), OR.assemble_block_circulant(To.astype(np.float64)).astype(np.float32))


@pytest.mark.parametrize("m,N,seed", [(60, 4, 0), (37, 3, 1), (300, 5, 2), (1024, 4, 3)])
def test_unfold_erot(cy, m, N, seed):
    """Compact, dense and from-points unfolds; m = 1024 gives each item a run of many sub-tiles."""
    p = I.sector_problem(m, N, seed=seed, eps_frac=0.02)
    Cb, G, w, z, res = _solve_reduced(cy, p, 1e-6)
    wg, zg = host(w), host(z)
    To = OS.unfold_erot(wg, zg, p.C_base.astype(np.float64), p.eps)
    Tc = host(cy.ot_unfold_plan(cy.OT_PLAN_EROT, m, N, w, z=z, C_base=Cb, eps=p.eps))
    assert np.abs(Tc - To).max() <= 2e-5 * To.max()
    Td = host(cy.ot_unfold_plan(cy.OT_PLAN_EROT, m, N, w, z=z, C_base=Cb, eps=p.eps, dense=True))
    # dense layout is the exact circulant assembly of the compact blocks
    assert np.array_equal(Td, OR.assemble_block_circulant(Tc.astype(np.float64)).astype(np.float32))
    # from points
    x = dev(p.x.astype(np.float32))
    Tp = host(cy.ot_unfold_plan(cy.OT_PLAN_EROT, m, N, w, z=z, x=x, y=x, eps=p.eps))
    assert np.abs(Tp - To).max() <= 1e-4 * To.max()


# ------------------------------------------------------------------ gradients (envelope)

def test_envelope_gradients_blocks(cy):
    p = I.sector_problem(40, 4, seed=3, eps_frac=0.05)
    Cb, G, w, z, res = _solve_reduced(cy, p, 1e-7)
    m, N = p.m, p.N
    d_a = torch.empty(m, device="cuda")
    d_b = torch.empty(m, device="cuda")
    d_C = torch.empty((N, m, m), device="cuda")
    out = cy.ot_value_and_grad(m, N, dev(p.a_base), dev(p.b_base), C_base=Cb, w=w, z=z, eps=p.eps,
                               d_a=d_a, d_b=d_b, d_C=d_C)
    env = OG.envelope_grad(p.a_base, p.b_base, p.C_base, p.eps)
    r = cy.read_result(out)
    assert r["value"] == pytest.approx(env["value"], rel=1e-5)
    sc = np.abs(env["d_a"]).max()
    assert np.abs(host(d_a) - env["d_a"]).max() <= 1e-4 * sc
    assert np.abs(host(d_b) - env["d_b"]).max() <= 1e-4 * np.abs(env["d_b"]).max()
    assert np.abs(host(d_C) - env["d_C"]).max() <= 1e-4 * env["d_C"].max()


def test_envelope_gradients_points(cy):
    p = I.sector_problem(64, 8, seed=4, eps_frac=0.05)
    m, N = p.m, p.N
    x32 = p.x.astype(np.float32)
    x = dev(x32)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, m, N, x=x, y=x, eps=p.eps)
    w, z, out = cy.ot_sinkhorn_reduced(m, N, dev(p.a_base), dev(p.b_base), G, cy.options(p.eps, tol=1e-7))
    assert cy.read_result(out)["status"] == cy.OT_OK
    d_x = torch.empty((m, 2), device="cuda")
    d_y = torch.empty((m, 2), device="cuda")
    out = cy.ot_value_and_grad(m, N, dev(p.a_base), dev(p.b_base), x=x, y=x, w=w, z=z, eps=p.eps,
                               d_x=d_x, d_y=d_y)
    x64 = x32.astype(np.float64)
    env = OG.envelope_grad(p.a_base, p.b_base, OG.cost_from_points(x64, x64, N), p.eps, x=x64, y=x64)
    r = cy.read_result(out)
    assert r["value"] == pytest.approx(env["value"], rel=1e-5)
    g_gpu = host(d_x) + host(d_y)
    g_ref = env["d_x"] + env["d_y"]
    assert np.abs(g_gpu - g_ref).max() <= 2e-4 * np.abs(g_ref).max()


# ------------------------------------------------------------------ faults (host-detected and device-reported)

def test_argument_errors(cy):
    p = I.sector_problem(8, 2, seed=0)
    Cb = dev(p.C_base)
    with pytest.raises(cy.OTError) as e:
        cy.ot_fold_cost(cy.OT_SOFTMIN, 8, 2, C_base=Cb, eps=0.0)
    assert e.value.code == cy.OT_ERR_ARG
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, 8, 2, C_base=Cb, eps=p.eps)
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(cy.OTError) as e:
        cy.ot_sinkhorn_reduced(8, 2, dev(p.a_base), dev(p.b_base), G, cy.options(p.eps), ws=small)
    assert e.value.code == cy.OT_ERR_WORKSPACE


def test_device_reported_statuses(cy):
    p = I.sector_problem(50, 3, seed=0, eps_frac=0.01)
    Cb = dev(p.C_base)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, 50, 3, C_base=Cb, eps=p.eps)
    a, b = dev(p.a_base), dev(p.b_base)
    # max_iter too small -> NOT_CONVERGED with the last iterate
    _, _, out = cy.ot_sinkhorn_reduced(50, 3, a, b, G, cy.options(p.eps, tol=1e-12, max_iter=3))
    r = cy.read_result(out)
    assert r["status"] == cy.OT_ERR_NOT_CONVERGED and r["iters"] == 3
    # a zero marginal entry -> OT_ERR_ARG from the device
    a0 = a.clone()
    a0[5] = 0.0
    _, _, out = cy.ot_sinkhorn_reduced(50, 3, a0, b, G, cy.options(p.eps))
    assert cy.read_result(out)["status"] == cy.OT_ERR_ARG
    # NaN in the cost -> OT_ERR_NONFINITE
    Gn = G.clone()
    Gn[3, 4] = float("nan")
    _, _, out = cy.ot_sinkhorn_reduced(50, 3, a, b, Gn, cy.options(p.eps))
    assert cy.read_result(out)["status"] == cy.OT_ERR_NONFINITE
    # the context is still usable afterwards
    _, _, out = cy.ot_sinkhorn_reduced(50, 3, a, b, G, cy.options(p.eps))
    assert cy.read_result(out)["status"] == cy.OT_OK


def test_bounded_barrier_wait_expires(cy):
    """Block 0 withholds its barrier arrival; the others' 2 ms waits run out -> OT_ERR_TIMEOUT."""
    p = I.sector_problem(200, 4, seed=0, eps_frac=0.02)
    Cb = dev(p.C_base)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, 200, 4, C_base=Cb, eps=p.eps)
    opt = cy.options(p.eps, timeout_ns=2_000_000, debug_flags=cy.OT_DEBUG_WITHHOLD_ARRIVAL)
    _, _, out = cy.ot_sinkhorn_reduced(200, 4, dev(p.a_base), dev(p.b_base), G, opt)
    assert cy.read_result(out)["status"] == cy.OT_ERR_TIMEOUT
    _, _, out = cy.ot_sinkhorn_reduced(200, 4, dev(p.a_base), dev(p.b_base), G, cy.options(p.eps))
    assert cy.read_result(out)["status"] == cy.OT_OK


def test_warm_start_resume(cy):
    """Resuming from a checkpointed z finishes in fewer iterations at the same fixed point."""
    p = I.sector_problem(120, 4, seed=6, eps_frac=0.01)
    Cb = dev(p.C_base)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, p.m, p.N, C_base=Cb, eps=p.eps)
    a, b = dev(p.a_base), dev(p.b_base)
    _, z1, out1 = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G, cy.options(p.eps, tol=1e-3))
    r1 = cy.read_result(out1)
    w2, z2, out2 = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G, cy.options(p.eps, tol=1e-6, warm_start=True), z=z1)
    r2 = cy.read_result(out2)
    w3, z3, out3 = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G, cy.options(p.eps, tol=1e-6))
    r3 = cy.read_result(out3)
    assert r2["status"] == r3["status"] == cy.OT_OK
    assert r2["iters"] < r3["iters"]
    assert abs(r1["iters"] + r2["iters"] - r3["iters"]) <= 2
    d = host(w2) - host(w3)
    assert np.abs(d - d.mean()).max() < 1e-4 * p.max_cost


def test_solver_variants_agree(cy):
    """Ring (FP32 sweep), bulk-reduce (FP64 partials, one barrier per sweep), fused (two barriers) and
    two-pass solvers give the same iterate."""
    p = I.image_grid_problem(side=32, seed=2, eps_frac=0.01)
    Cb = dev(p.C_base)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, p.m, p.N, C_base=Cb, eps=p.eps)
    a, b = dev(p.a_base), dev(p.b_base)
    w1, z1, o1 = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G, cy.options(p.eps, tol=1e-6))
    r1 = cy.read_result(o1)
    w2, z2, o2 = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G,
                                        cy.options(p.eps, tol=1e-6, debug_flags=cy.OT_DEBUG_NO_CLUSTER))
    r2 = cy.read_result(o2)
    assert r1["variant"] == "ring" and r2["variant"] == "fused"
    assert abs(r1["iters"] - r2["iters"]) <= 1 and r1["status"] == r2["status"] == cy.OT_OK
    d = host(w1) - host(w2)
    assert np.abs(d - d.mean()).max() <= 1e-6 * p.max_cost
    w4, z4, o4 = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G, cy.options(p.eps, tol=1e-6, debug_flags=cy.OT_DEBUG_NO_RING))
    r4 = cy.read_result(o4)
    assert r4["variant"] == "bulk" and abs(r4["iters"] - r1["iters"]) <= 1 and r4["status"] == cy.OT_OK
    d = host(w1) - host(w4)
    assert np.abs(d - d.mean()).max() <= 1e-6 * p.max_cost
    # odd size -> two-pass kernel on the same problem family
    q = I.sector_problem(97, 3, seed=1, eps_frac=0.02)
    Gq, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, q.m, q.N, C_base=dev(q.C_base), eps=q.eps)
    _, _, o3 = cy.ot_sinkhorn_reduced(q.m, q.N, dev(q.a_base), dev(q.b_base), Gq, cy.options(q.eps, tol=1e-6))
    assert cy.read_result(o3)["variant"] == "twopass"


@pytest.mark.parametrize("m,N,seed", [(4100, 2, 0), (6000, 2, 1)])
def test_reduced_streaming_route_parity(cy, m, N, seed):
    """Rows wider than the resident kernels take (4097..8192 columns) stream through the batch kernel."""
    p = I.sector_problem(m, N, seed=seed, eps_frac=0.05)
    tol = 1e-6
    Cb, G, w, z, res = _solve_reduced(cy, p, tol)
    assert res["status"] == cy.OT_OK, res
    assert res["variant"] == "stream"
    assert res["marg_l1"] <= tol
    wg, zg = host(w), host(z)
    rl1, cl1 = fp64_row_col_errors(wg, zg, p.C_base, p.a_base, p.b_base, p.eps)
    assert rl1 <= tol + 1e-6 and cl1 <= 1e-6, (rl1, cl1)
    orc = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=tol)
    assert abs(res["iters"] - orc["iters"]) <= 0.03 * orc["iters"] + 2, (res["iters"], orc["iters"])
    d = wg - orc["w"]
    assert np.abs(d - d.mean()).max() <= 1e-4 * p.eps + 1e-5 * np.abs(orc["w"]).max()


def test_full_streaming_route_warm_start(cy):
    """A full problem of n = 4400 (stored cost) through the streaming route, cold and warm."""
    p = I.sector_problem(1100, 4, seed=4, eps_frac=0.05)
    C = I.full_cost_from_blocks(p.C_base)
    a = np.tile(p.a_base, p.N)
    b = np.tile(p.b_base, p.N)
    tol = 1e-6
    f, g, out = cy.ot_sinkhorn_full(p.n, dev(a), dev(b), C=dev(C), opt=cy.options(p.eps, tol=tol))
    res = cy.read_result(out)
    assert res["status"] == cy.OT_OK and res["variant"] == "stream"
    fg, gg = host(f), host(g)
    T = np.exp((fg[:, None] + gg[None, :] - C.astype(np.float64)) / p.eps)
    e = OR.marginal_errors(T, OS.normalise(a), OS.normalise(b))
    assert e["row_l1"] <= tol + 1e-6 and e["col_l1"] <= 1e-6, e
    # warm start from the converged g: stops after the first measured sweep
    f2, g2, out2 = cy.ot_sinkhorn_full(p.n, dev(a), dev(b), C=dev(C), opt=cy.options(p.eps, tol=tol, warm_start=True),
                                       g=g.clone())
    r2 = cy.read_result(out2)
    assert r2["status"] == cy.OT_OK and r2["iters"] <= 2


# ------------------------------------------------------------------ reported marginal norms and objective

def _full_plan_norms(w, z, p):
    """The paper's marginal errors from their definition on the assembled n x n plan (Lemma 1):
    row L1 sum |T 1 - a|, column L1 and column L2 ||T^T 1 - b||_2 (Sec. 7.1), unit-mass a, b."""
    Tb = OS.unfold_erot(np.asarray(w, np.float64), np.asarray(z, np.float64), p.C_base.astype(np.float64), p.eps)
    T = OR.assemble_block_circulant(Tb)
    a = np.tile(OS.normalise(p.a_base), p.N) / p.N
    b = np.tile(OS.normalise(p.b_base), p.N) / p.N
    e = OR.marginal_errors(T, a, b)
    v = OS.primal_value_reduced(Tb, p.C_base.astype(np.float64), p.eps)
    return e, v


NORM_CASES = [("sector", 130, 5, 0.01), ("grid", 32, 4, 0.01), ("grid", 64, 4, 0.01), ("paper", 200, 20, 0.0)]


def _norm_problem(kind, s, N, frac):
    if kind == "sector":
        return I.sector_problem(s, N, seed=3, eps_frac=frac)
    if kind == "grid":
        return I.image_grid_problem(side=s, seed=1, eps_frac=frac)
    return I.paper_synthetic_problem(s, N, seed=1)


@pytest.mark.parametrize("kind,s,N,frac", NORM_CASES)
def test_reported_norms_and_value_vs_full_plan(cy, kind, s, N, frac):
    """marg_l1, marg_l1_col and marg_l2_col of ot_value_and_grad against the oracle's FP64 norms
    of the same potentials, evaluated on the assembled n x n plan.

    The GPU forms every plan entry with ex2.approx (relative error <= 2^-22 ~ 2.4e-7) from FP32
    arguments and sums them in FP32 before the FP64 accumulation (a few roundings of 6e-8), so
    each row or column sum carries a relative error of at most ~4e-7 of its mass; summed over a
    unit-mass plan that bounds every reported L1 norm (and the L2 norm, which is below the L1)
    by 5e-7 absolute.
    (1) The converged state (norms ~1e-7, i.e. at that floor): within 5e-7 + 1% relative.
    (2) The converged potentials with a seeded perturbation of 0.02 eps (norms ~1e-2): within
        5e-7 + 1e-4 relative, where any formula slip (scale N, sqrt, row/column swap) is visible;
        value and transport cost of that plan within 1e-5 relative.
    """
    p = _norm_problem(kind, s, N, frac)
    Cb, G, w, z, res = _solve_reduced(cy, p, 1e-6, max_iter=100000)
    assert res["status"] == cy.OT_OK
    a, b = dev(p.a_base), dev(p.b_base)
    rng = np.random.default_rng(11)
    wz = [(host(w), host(z))]
    wz.append((wz[0][0] + 0.02 * p.eps * rng.standard_normal(p.m), wz[0][1] + 0.02 * p.eps * rng.standard_normal(p.m)))
    for case, (wh, zh) in enumerate(wz):
        out = cy.ot_value_and_grad(p.m, p.N, a, b, C_base=Cb, w=dev(wh), z=dev(zh), eps=p.eps)
        r = cy.read_result(out)
        assert r["status"] == cy.OT_OK
        e, v = _full_plan_norms(wh, zh, p)
        rt = 1e-2 if case == 0 else 1e-4
        assert abs(r["marg_l1"] - e["row_l1"]) <= 5e-7 + rt * e["row_l1"], (case, r["marg_l1"], e["row_l1"])
        assert abs(r["marg_l1_col"] - e["col_l1"]) <= 5e-7 + rt * e["col_l1"], (case, r["marg_l1_col"], e["col_l1"])
        assert abs(r["marg_l2_col"] - e["col_l2"]) <= 5e-7 + rt * e["col_l2"], (case, r["marg_l2_col"], e["col_l2"])
        assert r["value"] == pytest.approx(v["value"], rel=1e-5)
        assert r["transport_cost"] == pytest.approx(v["transport_cost"], rel=1e-5)
    # the solver's own stopping measure is the same row L1 of the returned state
    assert abs(res["marg_l1"] - _full_plan_norms(*wz[0], p)[0]["row_l1"]) <= 5e-7 + 1e-2 * res["marg_l1"]


# ------------------------------------------------------------------ the paper's synthetic setting (Sec. 7.1, App. D)

@pytest.mark.parametrize("m,N", [(1000, 10), (200, 50), (4100, 10)])
def test_paper_synthetic_erot_vs_oracle(cy, m, N):
    """Cyclic Sinkhorn on the paper's synthetic inputs: cost blocks ~ N(3, 5^2) shifted to be
    non-negative, marginal blocks ~ U[0, 1) (near-zero entries included), lambda = 0.5.  m = 4100
    (d = 41000) takes the streaming route with ragged rows (4100 columns: not a multiple of the
    row chunk).  Against the oracle at the same tolerance: iterations, FP64 marginals of the GPU
    potentials, value and transport cost (1e-5 relative)."""
    p = I.paper_synthetic_problem(m, N, seed=0)
    tol = 1e-6
    Cb, G, w, z, res = _solve_reduced(cy, p, tol, max_iter=100000)
    assert res["status"] == cy.OT_OK, res
    assert res["marg_l1"] <= tol
    if m > 4096:
        assert res["variant"] == "stream"
    orc = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=tol)
    assert abs(res["iters"] - orc["iters"]) <= 0.03 * orc["iters"] + 2, (res["iters"], orc["iters"])
    wg, zg = host(w), host(z)
    rl1, cl1 = fp64_row_col_errors(wg, zg, p.C_base, p.a_base, p.b_base, p.eps)
    assert rl1 <= tol + (1e-6 if m > 4096 else 2e-7) and cl1 <= 1e-6, (rl1, cl1)
    out = cy.ot_value_and_grad(m, N, dev(p.a_base), dev(p.b_base), C_base=Cb, w=w, z=z, eps=p.eps)
    r = cy.read_result(out)
    v = OS.primal_value_reduced(OS.unfold_erot(orc["w"], orc["z"], p.C_base.astype(np.float64), p.eps),
                                p.C_base.astype(np.float64), p.eps)
    assert r["value"] == pytest.approx(v["value"], rel=1e-5)
    assert r["transport_cost"] == pytest.approx(v["transport_cost"], rel=1e-5)


# ------------------------------------------------------------------ ring solver (per-thread copy ring, FP32 sweep)

RING_CASES = [
    (2100, 2, 0.05, 0, 0),      # two warp groups x 16 columns per thread, every band resident
    (3000, 3, 0.02, 1, 0),      # 3000 columns: the copy ring streams the bands (ragged last chunk)
    (4096, 2, 0.01, 2, 0),      # the widest route, streaming
    (1024, 4, 0.01, 3, 0),      # single-group ring kernel (256 threads), resident
    (1500, 2, 0.02, 4, 0),      # two warp groups x 8 columns per thread, resident
    (252, 3, 0.02, 5, 0),       # single-group, ragged (252 columns: most threads idle on the tail)
]


@pytest.mark.parametrize("m,N,frac,seed,flags", RING_CASES)
def test_ring_solver_parity(cy, m, N, frac, seed, flags):
    """The ring solver against the oracle: the same iteration count (identical stopping rule),
    FP64 marginals of the returned potentials, potentials up to the dual constant."""
    p = I.sector_problem(m, N, seed=seed, eps_frac=frac)
    tol = 1e-6
    Cb = dev(p.C_base)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, m, N, C_base=Cb, eps=p.eps)
    w, z, out = cy.ot_sinkhorn_reduced(m, N, dev(p.a_base), dev(p.b_base), G,
                                       cy.options(p.eps, tol=tol, max_iter=100000, debug_flags=flags))
    res = cy.read_result(out)
    assert res["status"] == cy.OT_OK, res
    assert res["variant"] == "ring"
    assert res["marg_l1"] <= tol
    orc = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base, p.eps, tol=tol)
    assert abs(res["iters"] - orc["iters"]) <= 1, (res["iters"], orc["iters"])
    wg, zg = host(w), host(z)
    rl1, cl1 = fp64_row_col_errors(wg, zg, p.C_base, p.a_base, p.b_base, p.eps)
    assert rl1 <= tol + 2e-7 and cl1 <= 1e-6, (rl1, cl1)
    d = wg - orc["w"]
    assert np.abs(d - d.mean()).max() <= 1e-5 * max(1.0, np.abs(orc["w"]).max()) + 10 * p.eps * 1e-6


def test_ring_solver_warm_start_and_statuses(cy):
    """Warm start, NOT_CONVERGED, a device-detected bad marginal and the bounded barrier on the
    ring route (m = 2100 > 2048 columns)."""
    p = I.sector_problem(2100, 2, seed=5, eps_frac=0.02)
    G, _ = cy.ot_fold_cost(cy.OT_SOFTMIN, p.m, p.N, C_base=dev(p.C_base), eps=p.eps)
    a, b = dev(p.a_base), dev(p.b_base)
    _, z1, o1 = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G, cy.options(p.eps, tol=1e-3))
    r1 = cy.read_result(o1)
    w2, z2, o2 = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G, cy.options(p.eps, tol=1e-6, warm_start=True), z=z1)
    w3, z3, o3 = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G, cy.options(p.eps, tol=1e-6))
    r2, r3 = cy.read_result(o2), cy.read_result(o3)
    assert r1["variant"] == r2["variant"] == r3["variant"] == "ring"
    assert r2["status"] == r3["status"] == cy.OT_OK and r2["iters"] < r3["iters"]
    assert abs(r1["iters"] + r2["iters"] - r3["iters"]) <= 2
    d = host(w2) - host(w3)
    assert np.abs(d - d.mean()).max() < 1e-4 * p.max_cost
    _, _, o = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G, cy.options(p.eps, tol=1e-12, max_iter=3))
    r = cy.read_result(o)
    assert r["status"] == cy.OT_ERR_NOT_CONVERGED and r["iters"] == 3
    a0 = a.clone()
    a0[7] = 0.0
    _, _, o = cy.ot_sinkhorn_reduced(p.m, p.N, a0, b, G, cy.options(p.eps))
    assert cy.read_result(o)["status"] == cy.OT_ERR_ARG
    opt = cy.options(p.eps, timeout_ns=2_000_000, debug_flags=cy.OT_DEBUG_WITHHOLD_ARRIVAL)
    _, _, o = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G, opt)
    assert cy.read_result(o)["status"] == cy.OT_ERR_TIMEOUT
    _, _, o = cy.ot_sinkhorn_reduced(p.m, p.N, a, b, G, cy.options(p.eps))
    assert cy.read_result(o)["status"] == cy.OT_OK
