"""CPU FP64 oracle for cyclic-symmetry optimal transport (arXiv 2311.13147).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA library (no kernels, headers, helpers or
constant tables); the only common module is the seeded input generator
``paper_2311_13147_gb300.inputs``, which holds none of the method's
arithmetic.

Everything is plain numpy in float64, written for a reader to check against
the paper line by line, with no blocking, fusion or reordering beyond what the
cited equations state:

* ``rot``       -- problem definitions: Eq. problem_ROT with the regularisers
                   Eq. reg_for_original_OT (LOT) and Eq. reg_for_entropy_ROT
                   (EROT); Lemma 1's block-circulant assembly and the
                   symmetriser of App. B (Eq. lemma_definition_P).
* ``sinkhorn``  -- the folds (Eq. definition_G, Eq. def_Kij), the cyclic
                   Sinkhorn algorithm (Algorithm 2, written in the log form of
                   Eq. optimal_f_sinkhorn_logdomain), the plain Sinkhorn
                   algorithm on the full problem (Algorithm 3 Stage 2), the
                   two-stage algorithm (Algorithm 3), the unfolds (Eq.
                   optimal_solution_problem_CLOT, Eq. optimality_condition)
                   and the dual value of Theorem 2.
* ``lot``       -- a textbook transportation simplex for LOT at tiny sizes
                   (Eq. small_problem_CLOT) and brute force over permutations.
* ``grad``      -- gradients of the EROT value: envelope formulas from
                   Theorem 2's dual, the unrolled-iteration gradient (torch
                   float64 autograd on CPU) and central finite differences.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force, LP certificates, an independent library
solver (scipy HiGHS) or identities the paper fixes; none is "parity unpinned".
"""
from . import rot, sinkhorn, lot, grad  # noqa: F401
