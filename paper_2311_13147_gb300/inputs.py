"""Seeded synthetic inputs with n-order cyclic symmetry.

This module is shared by the CUDA path, the tests and the CPU oracle.  It
only *constructs inputs* -- point clouds, marginals and cost blocks that
satisfy Assumption 1 (Sec. 4: a = (alpha; ...; alpha), b = (beta; ...; beta),
C block-circulant, Eq. assumption_for_input_vectors and Eq. blkstr_cost).  It
holds none of the method's arithmetic (no fold, no Sinkhorn, no unfold).

Notation.  The paper writes d for the full size, n for the cyclic order and
m = d/n for the block size; this library writes n for the full size, N for
the cyclic order and keeps m = n/N.  The first block row of the cost,
C_k = C[0:m, k*m:(k+1)*m], is stored as ``C_base[k]`` (shape [N, m, m]).

Every generator builds its values in float64 and rounds them once to float32;
``C_base`` is computed from the float64 geometry, and the full cost is
assembled from ``C_base`` by the circulant rule (block (r, c) = C_{(c-r) mod N})
so that the full float32 matrix is exactly block-circulant.

Marginals: ``a_base`` / ``b_base`` are the base blocks normalised to unit mass
(the full vectors are tile(a_base)/N).  Entries are clamped to at least
1e-12 * max before normalisation so that log-domain solvers never see log 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "CyclicProblem",
    "sector_points",
    "rotation",
    "cost_blocks_from_points",
    "full_cost_from_blocks",
    "full_points",
    "max_cost_points",
    "tile_marginal",
    "sector_problem",
    "image_grid_problem",
    "mirror_order",
    "mirror_images",
    "mirror_problem",
    "polar_grid_problem",
    "paper_synthetic_problem",
    "batch_problems",
    "noisy_full_marginal",
    "bench_sizes",
]


@dataclass
class CyclicProblem:
    """One cyclic-symmetric OT instance (Assumption 1).

    Attributes
    ----------
    m, N : block size and cyclic order (full size n = N*m).
    a_base, b_base : float32 [m], unit mass.
    eps : entropic regulariser (the paper's lambda, Eq. reg_for_entropy_ROT).
    C_base : float32 [N, m, m] first block row, or None when only points exist.
    x, y : float64 [m, 2] base source / target points when the cost is the
        squared Euclidean distance C_k[i, j] = |x_i - R^k y_j|^2, else None.
    angle : rotation angle between consecutive blocks (2*pi/N for point
        clouds; the image grid uses a 90-degree pixel permutation instead).
    """

    name: str
    m: int
    N: int
    a_base: np.ndarray
    b_base: np.ndarray
    eps: float
    C_base: Optional[np.ndarray] = None
    x: Optional[np.ndarray] = None
    y: Optional[np.ndarray] = None
    max_cost: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.N * self.m


def _normalise(v: np.ndarray) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    v = np.maximum(v, 1e-12 * v.max())
    return v / v.sum()


def rotation(theta: float) -> np.ndarray:
    """2x2 rotation matrix by angle theta (float64)."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, -s], [s, c]], dtype=np.float64)


def sector_points(rng: np.random.Generator, m: int, N: int,
                  r_lo: float = 0.5, r_hi: float = 1.0) -> np.ndarray:
    """m base points with angle ~ U[0, 2*pi/N) and radius ~ U[r_lo, r_hi]."""
    theta = rng.uniform(0.0, 2.0 * np.pi / N, size=m)
    r = rng.uniform(r_lo, r_hi, size=m)
    return np.stack([r * np.cos(theta), r * np.sin(theta)], axis=1)


def max_cost_points(p: np.ndarray, N: int) -> float:
    """Largest squared distance between any two points of the full cloud.

    Every pair (R^r x_i, R^c x_j) of the full cloud appears as some C_k[i, j],
    so max C is the squared diameter of the full cloud; it is attained by two
    vertices of its convex hull.
    """
    from scipy.spatial import ConvexHull

    P = full_points(p, N)
    try:
        v = P[ConvexHull(P).vertices]
    except Exception:  # degenerate clouds (collinear or tiny): brute force
        v = P
    d = v[:, None, :] - v[None, :, :]
    return float((d * d).sum(axis=2).max())


def full_points(p: np.ndarray, N: int) -> np.ndarray:
    """Stack R^k p for k = 0..N-1 (float64 [N*m, 2]); block k is rotated by 2*pi*k/N."""
    return np.concatenate([p @ rotation(2.0 * np.pi * k / N).T for k in range(N)], axis=0)


def cost_blocks_from_points(x: np.ndarray, y: np.ndarray, N: int) -> np.ndarray:
    """C_base[k, i, j] = |x_i - R^k y_j|^2 in float64 (input construction)."""
    out = np.empty((N, x.shape[0], y.shape[0]), dtype=np.float64)
    for k in range(N):
        yk = y @ rotation(2.0 * np.pi * k / N).T
        d = x[:, None, :] - yk[None, :, :]
        out[k] = (d * d).sum(axis=2)
    return out


def full_cost_from_blocks(C_base: np.ndarray) -> np.ndarray:
    """Assemble the n x n cost from its first block row by Eq. blkstr_cost.

    Block (r, c) of the result is C_base[(c - r) mod N]; the dtype is kept, so
    a float32 C_base gives an exactly block-circulant float32 matrix.
    """
    N, m, _ = C_base.shape
    C = np.empty((N * m, N * m), dtype=C_base.dtype)
    for r in range(N):
        for c in range(N):
            C[r * m:(r + 1) * m, c * m:(c + 1) * m] = C_base[(c - r) % N]
    return C


def tile_marginal(v_base: np.ndarray, N: int) -> np.ndarray:
    """Full marginal (v; v; ...; v)/N in float64 (Eq. assumption_for_input_vectors)."""
    v = np.asarray(v_base, dtype=np.float64)
    return np.tile(v / v.sum(), N) / N


def noisy_full_marginal(rng: np.random.Generator, v_full: np.ndarray,
                        sigma: float = 0.01) -> np.ndarray:
    """Approximate symmetry: v * (1 + sigma * N(0,1)), clipped at 0, renormalised."""
    v = np.asarray(v_full, dtype=np.float64) * (1.0 + sigma * rng.standard_normal(v_full.shape))
    return _normalise(np.maximum(v, 0.0))


def _finish(name, m, N, a, b, eps_frac, C64=None, x=None, y=None, eps_abs=None, meta=None):
    a32 = _normalise(a).astype(np.float32)
    b32 = _normalise(b).astype(np.float32)
    C32 = None if C64 is None else np.ascontiguousarray(C64.astype(np.float32))
    if C64 is not None:
        maxc = float(C32.max())
    else:
        maxc = float(meta.get("max_cost"))
    eps = float(eps_abs) if eps_abs is not None else float(eps_frac * maxc)
    return CyclicProblem(name=name, m=m, N=N, a_base=a32, b_base=b32, eps=eps,
                         C_base=C32, x=x, y=y, max_cost=maxc, meta=dict(meta or {}))


def sector_problem(m: int, N: int, seed: int = 0, eps_frac: float = 0.05,
                   dirichlet: float = 1.0, with_cost: bool = True) -> CyclicProblem:
    """Ring/sector point cloud (the tiny and differentiation workloads).

    m base points, angle ~ U[0, 2*pi/N), radius ~ U[0.5, 1], rotated by
    2*pi*k/N; source and target point sets coincide (x == y); a_base, b_base ~
    Dirichlet(dirichlet * 1_m); C = squared Euclidean distance; eps = eps_frac *
    max C.
    """
    rng = np.random.default_rng(seed)
    p = sector_points(rng, m, N)
    a = rng.dirichlet(dirichlet * np.ones(m))
    b = rng.dirichlet(dirichlet * np.ones(m))
    C64 = cost_blocks_from_points(p, p, N) if with_cost else None
    meta = {"kind": "sector", "seed": seed}
    if C64 is None:
        meta["max_cost"] = max_cost_points(p, N)
    return _finish(f"sector_m{m}_N{N}_s{seed}", m, N, a, b, eps_frac, C64, p, p.copy(), meta=meta)


def _grid_rotate(r: np.ndarray, c: np.ndarray, side: int):
    """90-degree rotation of pixel indices about the grid centre: (r, c) -> (c, side-1-r)."""
    return c, side - 1 - r


def image_grid_problem(side: int = 64, seed: int = 0, eps_frac: float = 0.01,
                       blobs: int = 3) -> CyclicProblem:
    """Image grid with 4-fold rotational symmetry (N = 4, m = (side/2)^2).

    The base block is the top-left quadrant in row-major order; block k holds
    the base pixels rotated k times by 90 degrees about the grid centre (the
    90-degree counterpart of Example 1's pixel ordering).  Pixel centres are
    ((r+.5)/side, (c+.5)/side); C is the squared Euclidean distance between
    centres.  Squared integer offsets divided by side^2 are exact in float32.
    a_base, b_base: sums of ``blobs`` Gaussian blobs in the base quadrant
    (centre uniform in the quadrant, sigma ~ U[2, 6] px, amplitude ~ U[.5, 1.5]).
    """
    assert side % 2 == 0
    h = side // 2
    m, N = h * h, 4
    rng = np.random.default_rng(seed)
    rr, cc = np.meshgrid(np.arange(h), np.arange(h), indexing="ij")
    r0, c0 = rr.ravel(), cc.ravel()
    blocks = [(r0, c0)]
    for _ in range(1, N):
        blocks.append(_grid_rotate(*blocks[-1], side))
    C64 = np.empty((N, m, m), dtype=np.float64)
    for k in range(N):
        rk, ck = blocks[k]
        dr = r0[:, None].astype(np.int64) - rk[None, :].astype(np.int64)
        dc = c0[:, None].astype(np.int64) - ck[None, :].astype(np.int64)
        C64[k] = (dr * dr + dc * dc) / float(side * side)

    def blob_field():
        v = np.zeros(m)
        for _ in range(blobs):
            cr, ccn = rng.uniform(0, h), rng.uniform(0, h)
            sig = rng.uniform(2.0, 6.0)
            amp = rng.uniform(0.5, 1.5)
            v += amp * np.exp(-((r0 + 0.5 - cr) ** 2 + (c0 + 0.5 - ccn) ** 2) / (2 * sig * sig))
        return v

    a = blob_field()
    b = blob_field()
    coords = np.stack([(r0 + 0.5) / side, (c0 + 0.5) / side], axis=1)
    meta = {"kind": "image_grid", "side": side, "seed": seed,
            "pixel_blocks": [np.stack(bk, 1) for bk in blocks]}
    return _finish(f"grid{side}_N4_s{seed}", m, N, a, b, eps_frac, C64, coords, coords.copy(), meta=meta)


def mirror_order(h: int, w: int):
    """Pixel order pi of the mirror vectorisation (Example 1, Eq. vectorization_mirror).

    Returns (rows, cols), int64 [h*w].  Entries k < h*w/2 run over the left half
    of the image column by column; entry k + h*w/2 is the pixel in the same row
    and the mirrored column w-1-c.  An image that is symmetric about the
    vertical axis therefore becomes a = (alpha; alpha), and any distance between
    pixel positions becomes a 2-block circulant cost (the mirror is an isometry).
    """
    assert h > 0 and w > 0 and w % 2 == 0
    k = np.arange(h * w, dtype=np.int64)
    q = k // h
    cols = np.where(k < h * w // 2, q, 3 * w // 2 - q - 1)
    return k % h, cols


def mirror_images(count: int, h: int = 64, w: int = 64, seed: int = 0, blobs: int = 4,
                  asym: float = 0.0) -> np.ndarray:
    """Gray-scale images symmetric about the vertical axis, float64 [count][h][w], each summing to 1.

    Each image is a background of 2% of its peak plus ``blobs`` Gaussian blobs
    with centres uniform in the left half (sigma ~ U[2, 8] px, amplitude ~
    U[0.5, 1.5]); the right half is the exact mirror of the left.  ``asym`` > 0
    then multiplies every pixel by (1 + asym * N(0, 1)) (clipped at 0), so the
    symmetry is only approximate, as for photographs.
    """
    assert w % 2 == 0
    rng = np.random.default_rng(seed)
    rr, cc = np.meshgrid(np.arange(h) + 0.5, np.arange(w // 2) + 0.5, indexing="ij")
    out = np.empty((count, h, w))
    for i in range(count):
        left = np.zeros((h, w // 2))
        for _ in range(blobs):
            cr, ccn = rng.uniform(0, h), rng.uniform(0, w / 2)
            sig = rng.uniform(2.0, 8.0)
            left += rng.uniform(0.5, 1.5) * np.exp(-((rr - cr) ** 2 + (cc - ccn) ** 2) / (2 * sig * sig))
        left += 0.02 * left.max()
        img = np.concatenate([left, left[:, ::-1]], axis=1)
        if asym > 0.0:
            img = np.maximum(img * (1.0 + asym * rng.standard_normal(img.shape)), 0.0)
        out[i] = img / img.sum()
    return out


def mirror_problem(A: np.ndarray, B: np.ndarray, lam: float = 0.5) -> CyclicProblem:
    """C-EROT between two h x w images under the mirror order (N = 2, m = h*w/2).

    a and b are the images vectorised by ``mirror_order``; the cost is the
    Euclidean distance between pixel positions, in pixels (the distance used
    with the paper's real images), C_base[k][i][j] = |p_i - p_(k m + j)|.  The
    base marginals are the block sums a_i + a_(m+i) (Alg. 3's block average up
    to the factor 1/N; exact for symmetric images).  ``meta`` keeps the full
    vectorised marginals (float64, unit mass) for the full and two-stage solves.
    ``lam`` is the absolute regulariser (0.5 in the paper's experiments).
    """
    h, w = A.shape
    rows, cols = mirror_order(h, w)
    m = h * w // 2
    a_full = _normalise(np.asarray(A, np.float64)[rows, cols])
    b_full = _normalise(np.asarray(B, np.float64)[rows, cols])
    r0, c0 = rows[:m], cols[:m]
    C64 = np.empty((2, m, m))
    for k in range(2):
        dr = r0[:, None] - rows[k * m:(k + 1) * m][None, :]
        dc = c0[:, None] - cols[k * m:(k + 1) * m][None, :]
        C64[k] = np.sqrt((dr * dr + dc * dc).astype(np.float64))
    meta = {"kind": "mirror", "h": h, "w": w, "a_full": a_full, "b_full": b_full}
    return _finish(f"mirror{h}x{w}", m, 2, a_full[:m] + a_full[m:], b_full[:m] + b_full[m:], 0.0, C64,
                   eps_abs=lam, meta=meta)


def polar_grid_problem(n_radii: int = 256, n_angles: int = 16, N: int = 16, seed: int = 0,
                       eps_frac: float = 0.005, comps: int = 5,
                       with_cost: bool = False) -> CyclicProblem:
    """Polar grid in the unit disk with N sectors (the large workload).

    Base sector points: radius (t+.5)/n_radii, angle (s+.5)*(2*pi/N)/n_angles;
    m = n_radii * n_angles.  Marginals: ``comps`` Gaussian components per base
    sector (centres uniform in the sector, sigma ~ U[0.05, 0.2], weights ~
    U[0.5, 1.5]).  The cost is the squared Euclidean distance (max about 4).
    """
    rng = np.random.default_rng(seed)
    t = (np.arange(n_radii) + 0.5) / n_radii
    s = (np.arange(n_angles) + 0.5) * (2.0 * np.pi / N) / n_angles
    R, S = np.meshgrid(t, s, indexing="ij")
    p = np.stack([(R * np.cos(S)).ravel(), (R * np.sin(S)).ravel()], axis=1)
    m = p.shape[0]

    def mixture():
        v = np.zeros(m)
        for _ in range(comps):
            th = rng.uniform(0, 2 * np.pi / N)
            rad = rng.uniform(0.05, 1.0)
            cen = np.array([rad * np.cos(th), rad * np.sin(th)])
            sig = rng.uniform(0.05, 0.2)
            w = rng.uniform(0.5, 1.5)
            v += w * np.exp(-((p - cen) ** 2).sum(1) / (2 * sig * sig))
        return v

    a = mixture()
    b = mixture()
    meta = {"kind": "polar_grid", "seed": seed, "max_cost": max_cost_points(p, N)}
    C64 = cost_blocks_from_points(p, p, N) if with_cost else None
    return _finish(f"polar{m}_N{N}_s{seed}", m, N, a, b, eps_frac, C64, p, p.copy(), meta=meta)


def paper_synthetic_problem(m: int, N: int, seed: int = 0, lam: float = 0.5) -> CyclicProblem:
    """Non-geometric blocks shaped like the paper's synthetic data (App. D).

    alpha, beta ~ U[0, 1) (then normalised); C_k entries ~ N(3, 5^2), shifted
    by |min| over all blocks so that C >= 0; lambda = 0.5 (Sec. 7.1).
    """
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 1.0, size=m)
    b = rng.uniform(0.0, 1.0, size=m)
    C64 = rng.normal(3.0, 5.0, size=(N, m, m))
    C64 += abs(C64.min())
    return _finish(f"paper_m{m}_N{N}_s{seed}", m, N, a, b, 0.0, C64, eps_abs=lam,
                   meta={"kind": "paper_synthetic", "seed": seed})


def paper_synthetic_device(count: int, m: int, N: int, seed: int, device):
    """`count` instances of the paper's synthetic setting (App. D) drawn on the device.

    Cost blocks C_k ~ N(3, 5^2) shifted by |min| over each instance's blocks,
    marginal blocks ~ U[0, 1) (normalised by the solvers), from torch's seeded
    device generator: shapes and distributions of ``paper_synthetic_problem``
    for sizes whose host generation would take minutes (d = 10000 rows).
    Returns (C_base [count][N][m][m], a_base [count][m], b_base [count][m]), FP32.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    C = torch.randn((count, N, m, m), generator=g, device=device, dtype=torch.float32).mul_(5.0).add_(3.0)
    C.add_(C.view(count, -1).amin(dim=1).abs().view(count, 1, 1, 1))
    a = torch.rand((count, m), generator=g, device=device, dtype=torch.float32)
    b = torch.rand((count, m), generator=g, device=device, dtype=torch.float32)
    return C, a, b


def batch_problems(count: int = 512, seed: int = 0, n_lo: int = 1024, n_hi: int = 16384,
                   orders=(2, 3, 4, 6, 8), eps_frac: float = 0.01, dirichlet: float = 0.5,
                   with_cost: bool = False):
    """Uneven batch: N ~ U(orders), m ~ U-int[ceil(n_lo/N), floor(n_hi/N)].

    Each problem is a ring/sector cloud with Dirichlet(dirichlet) marginals and
    eps = eps_frac * max C.  Returns a list of CyclicProblem (costs optional).
    """
    rng = np.random.default_rng(seed)
    out = []
    for p_idx in range(count):
        N = int(rng.choice(orders))
        m = int(rng.integers(-(-n_lo // N), n_hi // N + 1))
        pts = sector_points(rng, m, N)
        a = rng.dirichlet(dirichlet * np.ones(m))
        b = rng.dirichlet(dirichlet * np.ones(m))
        C64 = cost_blocks_from_points(pts, pts, N) if with_cost else None
        meta = {"kind": "batch", "seed": seed, "index": p_idx, "max_cost": max_cost_points(pts, N)}
        out.append(_finish(f"batch{p_idx}_m{m}_N{N}", m, N, a, b, eps_frac, C64, pts, pts.copy(),
                           meta=meta))
    return out


def histogram_pairs(m: int, count: int = 64, seed: int = 0, dirichlet: float = 0.5):
    """`count` (a_base, b_base) pairs ~ Dirichlet(dirichlet * 1_m), clamped and normalised, float32 [count][m].

    The "64 shared-cost histograms per cost" of the precision workload: every
    pair is a separate transport problem on the same folded cost.
    """
    rng = np.random.default_rng(seed)
    a = np.stack([_normalise(rng.dirichlet(dirichlet * np.ones(m))) for _ in range(count)])
    b = np.stack([_normalise(rng.dirichlet(dirichlet * np.ones(m))) for _ in range(count)])
    return a.astype(np.float32), b.astype(np.float32)


def bench_sizes():
    """Named workload sizes (block size m, order N) used by the benchmark."""
    return {
        "tiny": (60, 4),
        "image_grid": (1024, 4),
        "differentiation": (1024, 8),
        "large_polar": (4096, 16),
    }
