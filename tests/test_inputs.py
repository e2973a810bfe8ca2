"""Seeded input generators: shapes and the distributions they state (no method arithmetic)."""
import numpy as np
import pytest

from paper_2311_13147_gb300 import inputs as I


def test_paper_synthetic_problem_recipe():
    p = I.paper_synthetic_problem(50, 4, seed=3)
    assert p.C_base.shape == (4, 50, 50) and p.a_base.shape == (50,)
    assert p.C_base.min() == pytest.approx(0.0, abs=1e-6)   # shifted by |min| over all blocks
    assert np.all(p.a_base >= 0) and np.all(p.b_base >= 0)


def test_paper_synthetic_device_recipe():
    torch = pytest.importorskip("torch")
    C, a, b = I.paper_synthetic_device(3, 40, 5, seed=1, device="cpu")
    assert C.shape == (3, 5, 40, 40) and a.shape == (3, 40) and b.shape == (3, 40)
    assert C.dtype == torch.float32
    mins = C.view(3, -1).amin(dim=1)
    assert torch.all(mins.abs() <= 1e-5)                      # each instance shifted by its own |min|
    # N(3, 5^2) before the shift: the standard deviation survives it
    assert abs(float(C.std()) - 5.0) < 0.2
    assert float(a.min()) >= 0.0 and float(a.max()) < 1.0 and float(b.max()) < 1.0
    C2, a2, _ = I.paper_synthetic_device(3, 40, 5, seed=1, device="cpu")
    assert torch.equal(C, C2) and torch.equal(a, a2)          # seeded
