"""Mirror symmetry (Example 1, N = 2): the pixel ordering, Assumption 1, and the
reduced = full identity of Theorem 2 on mirror images (CPU, FP64 oracle).

The pins are independent of the generator's arithmetic: a brute-force check
that the order is a permutation whose second half mirrors the first, a
distance matrix recomputed with scipy from the ordered pixel positions, and
the oracle's full Sinkhorn against its reduced solve.
"""

import numpy as np
import pytest
from scipy.spatial.distance import cdist

from paper_2311_13147_gb300 import inputs as I
from oracle import rot as OR
from oracle import sinkhorn as OS


@pytest.mark.parametrize("h,w", [(1, 2), (4, 6), (6, 8), (64, 64), (96, 96)])
def test_mirror_order_permutes_pixels_and_mirrors_the_second_half(h, w):
    rows, cols = I.mirror_order(h, w)
    assert sorted(zip(rows.tolist(), cols.tolist())) == [(r, c) for r in range(h) for c in range(w)]
    m = h * w // 2
    assert (cols[:m] < w // 2).all()                       # the first half is the left half
    assert (rows[m:] == rows[:m]).all() and (cols[m:] == w - 1 - cols[:m]).all()


def test_mirror_order_small_case_by_hand():
    # h = 2, w = 4: left half column by column, then the mirrored columns 3, 2
    rows, cols = I.mirror_order(2, 4)
    assert list(zip(rows.tolist(), cols.tolist())) == [(0, 0), (1, 0), (0, 1), (1, 1),
                                                        (0, 3), (1, 3), (0, 2), (1, 2)]


def test_symmetric_image_gives_tiled_marginal_and_circulant_cost():
    imgs = I.mirror_images(2, 12, 10, seed=3)
    assert np.array_equal(imgs[0], imgs[0][:, ::-1])
    p = I.mirror_problem(imgs[0], imgs[1], lam=0.5)
    m = p.m
    a_full = p.meta["a_full"]
    assert np.array_equal(a_full[:m], a_full[m:])          # a = (alpha; alpha), Assumption 1
    rows, cols = I.mirror_order(12, 10)
    pos = np.stack([rows, cols], 1).astype(np.float64)
    C_direct = cdist(pos, pos).astype(np.float32)          # Euclidean pixel distances, in the mirror order
    assert np.array_equal(I.full_cost_from_blocks(p.C_base), C_direct)


def test_asymmetric_image_block_average():
    imgs = I.mirror_images(2, 8, 8, seed=4, asym=0.2)
    p = I.mirror_problem(imgs[0], imgs[1], lam=0.5)
    a_full = p.meta["a_full"]
    # the base marginal is Algorithm 3's block average, renormalised to unit mass
    alpha = OS.block_average(a_full, 2)
    assert np.allclose(p.a_base, alpha / alpha.sum(), rtol=1e-6)


def test_mirror_reduced_equals_full_oracle():
    """Theorem 2 on a symmetric 8 x 8 pair: the full optimum is the unfolded reduced one."""
    imgs = I.mirror_images(2, 8, 8, seed=5)
    p = I.mirror_problem(imgs[0], imgs[1], lam=0.5)
    C = I.full_cost_from_blocks(p.C_base).astype(np.float64)
    # the full marginals from the (float32) base blocks, so both sides solve the same inputs;
    # they equal the image's own vectorised marginals to float32 rounding
    a, b = I.tile_marginal(p.a_base, 2), I.tile_marginal(p.b_base, 2)
    assert np.allclose(a, p.meta["a_full"], rtol=1e-6) and np.allclose(b, p.meta["b_full"], rtol=1e-6)
    full = OS.sinkhorn_full(a, b, C, p.eps, tol=1e-13)
    Tf = np.exp((full["f"][:, None] + full["g"][None, :] - C) / p.eps)
    red = OS.cyclic_sinkhorn(p.a_base, p.b_base, p.C_base.astype(np.float64), p.eps, tol=1e-13)
    Tb = OS.unfold_erot(red["w"], red["z"], p.C_base.astype(np.float64), p.eps)
    assert np.abs(OR.assemble_block_circulant(Tb) - Tf).max() < 1e-12
    v = OS.primal_value_reduced(Tb, p.C_base.astype(np.float64), p.eps)
    assert v["value"] == pytest.approx(OR.erot_primal(C, Tf, p.eps), rel=1e-11)
    assert v["transport_cost"] == pytest.approx(OR.transport_cost(C, Tf), rel=1e-10)
