"""Batches of independent cyclic problems: packing, fold, solve and CUDA-graph replay.

Packs a list of problems (block size m, order N, eps, base points and
marginals) into the flat device buffers the C ABI expects -- descriptors,
one float2 point buffer, one cost buffer with 4-aligned rows, one vector
buffer per marginal / potential -- and runs ot_batch_fold (one launch) and
ot_batch_solve (two persistent launches: problems with two and with three
rows per thread group and chunk).  ``BatchSolver.autotune()`` picks the solver's
launch configuration for the batch; ``BatchSolver.capture()`` records the fold
and the solve in a CUDA graph that ``replay()`` launches again.
"""
from __future__ import annotations

import numpy as np
import torch

from . import cyclicot as cy


class BatchSolver:
    def __init__(self, problems, tol=1e-6, max_iter=20000, device="cuda"):
        self.count = len(problems)
        self.device = torch.device(device)
        descs, pts, a, b = [], [], [], []
        g_off = v_off = x_off = 0
        for p in problems:
            m = p.m
            ld = (m + 3) // 4 * 4   # rows padded to 16 bytes for float4 loads
            descs.append(cy.ot_problem_desc(m, p.N, float(p.eps), ld, g_off, v_off, x_off, x_off + m))
            pts.append(np.asarray(p.x, np.float32))
            pts.append(np.asarray(p.y, np.float32))
            a.append(np.asarray(p.a_base, np.float32))
            b.append(np.asarray(p.b_base, np.float32))
            g_off += m * ld
            v_off += m
            x_off += 2 * m
        self.descs = descs
        self.total_m = v_off
        self.total_g = g_off
        dev = self.device
        self.points = torch.from_numpy(np.concatenate(pts)).to(dev)
        self.a = torch.from_numpy(np.concatenate(a)).to(dev)
        self.b = torch.from_numpy(np.concatenate(b)).to(dev)
        self.G = torch.empty(self.total_g, dtype=torch.float32, device=dev)
        self.w = torch.zeros(self.total_m, dtype=torch.float64, device=dev)
        self.z = torch.zeros(self.total_m, dtype=torch.float64, device=dev)
        self.res = torch.zeros(64 * self.count, dtype=torch.uint8, device=dev)
        self.ws = torch.empty(cy.ot_batch_workspace_bytes(self.count, self.total_m), dtype=torch.uint8, device=dev)
        self.opt = cy.options(1.0, tol=tol, max_iter=max_iter)
        cy.ot_batch_prepare(descs, self.ws)
        self.graph = None

    def fold(self):
        cy.ot_batch_fold(self.count, self.points, self.G, self.ws)

    def solve(self):
        cy.ot_batch_solve(self.count, self.total_m, self.G, self.a, self.b, self.opt, self.w, self.z, self.res,
                          self.ws)

    def run(self):
        self.fold()
        self.solve()

    def autotune(self):
        """Pick the launch configuration for this batch (cached per device and problem table)."""
        self.opt.tile_override = 0
        code, ms = cy.ot_batch_autotune(self.count, self.total_m, self.G, self.a, self.b, self.opt, self.w, self.z,
                                        self.res, self.ws)
        self.opt.tile_override = code
        self.tuning_ms = ms
        return code

    def capture(self):
        """Record fold + solve in a CUDA graph (after one eager run, outside capture)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.fold()
                self.solve()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def results(self):
        return cy.read_results(self.res, self.count)

    def potentials(self, p):
        d = self.descs[p]
        return (self.w[d.v_off:d.v_off + d.m], self.z[d.v_off:d.v_off + d.m])

    def cost(self, p):
        d = self.descs[p]
        return self.G[d.g_off:d.g_off + d.m * d.ld].view(d.m, d.ld)[:, :d.m]


class SharedCostBatch:
    """Up to 64 histogram pairs on one cyclic cost: BF16 kernel-domain iterations on the
    tensor cores, then the FP32 log-domain batch solver warm-started from their potentials.

    points: base source / target coordinates [m][2] (cost |x_i - R^k y_j|^2);
    a_hist, b_hist: [P][m] marginals (P <= 64).
    """

    def __init__(self, x, y, N, eps, a_hist, b_hist, tol=1e-6, max_iter=20000, device="cuda"):
        dev = torch.device(device)
        x = np.asarray(x, np.float32)
        y = np.asarray(y, np.float32)
        self.m = m = x.shape[0]
        self.N, self.eps = int(N), float(eps)
        self.P = P = a_hist.shape[0]
        self.ld = ld = (m + 3) // 4 * 4
        self.descs = [cy.ot_problem_desc(m, self.N, self.eps, ld, 0, p * m, 0, m) for p in range(P)]
        self.points = torch.from_numpy(np.concatenate([x, y])).to(dev)
        self.a = torch.from_numpy(np.ascontiguousarray(a_hist, np.float32)).to(dev)
        self.b = torch.from_numpy(np.ascontiguousarray(b_hist, np.float32)).to(dev)
        self.G = torch.empty(m * ld, dtype=torch.float32, device=dev)
        self.w = torch.zeros(P * m, dtype=torch.float64, device=dev)
        self.z = torch.zeros(P * m, dtype=torch.float64, device=dev)
        self.res = torch.zeros(64 * P, dtype=torch.uint8, device=dev)
        self.ws = torch.empty(cy.ot_batch_workspace_bytes(P, P * m), dtype=torch.uint8, device=dev)
        self.kws = torch.empty(cy.ot_kdomain_workspace_bytes(m), dtype=torch.uint8, device=dev)
        self.opt = cy.options(1.0, tol=tol, max_iter=max_iter)
        cy.ot_batch_prepare(self.descs, self.ws)

    def fold(self):
        cy.ot_batch_fold(1, self.points, self.G, self.ws)   # one shared cost

    def kernel_domain(self, iters, row_err=None):
        """BF16 tensor-core iterations; leaves z = eps ln V in self.z."""
        cy.ot_kdomain_solve(self.m, self.G, self.ld, self.eps, self.a, self.b, iters,
                            z_out=self.z.view(self.P, self.m), row_err=row_err, workspace_t=self.kws)

    def polish(self, warm=True):
        self.opt.warm_start = 1 if warm else 0
        cy.ot_batch_solve(self.P, self.P * self.m, self.G, self.a.view(-1), self.b.view(-1), self.opt,
                          self.w, self.z, self.res, self.ws)

    def results(self):
        return cy.read_results(self.res, self.P)

    def potentials(self, p):
        m = self.m
        return self.w[p * m:(p + 1) * m], self.z[p * m:(p + 1) * m]

    def cost(self):
        return self.G.view(self.m, self.ld)[:, :self.m]
