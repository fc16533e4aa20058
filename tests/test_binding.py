"""Argument checks of the Python binding's device- and host-pointer solves: a mismatched
output (dtype, shape, layout, device) must be refused before the C ABI is called, since the
kernels write n x k doubles through the raw pointer.  Runs on the CPU (no call reaches the
library)."""
import numpy as np
import pytest

import paper_2202_09288_gb300 as P


def test_host_output_must_match_input():
    B = np.asfortranarray(np.ones((50, 3)))
    with pytest.raises(ValueError):
        P.chol_solve(0, 0, B, np.zeros((50, 3), dtype=np.float32, order="F"))
    with pytest.raises(ValueError):
        P.chol_solve(0, 0, B, np.zeros((50, 2), order="F"))
    with pytest.raises(ValueError):
        P.chol_solve(0, 0, B, np.zeros((50, 3), order="C"))  # row-major: wrong stride
    with pytest.raises(ValueError):
        P.chol_solve(0, 0, B, np.zeros(150))


def test_device_arguments_are_checked():
    torch = pytest.importorskip("torch")
    B = torch.ones(3, 50, dtype=torch.float64)
    # CPU tensors are refused for every device-pointer entry point
    for fn in (lambda: P.chol_solve(0, 0, B, torch.empty_like(B)),
               lambda: P.chol_solve_noalloc(0, 0, B, torch.empty_like(B)),
               lambda: P.chol_refine(0, 0, B, torch.empty_like(B))):
        with pytest.raises(ValueError):
            fn()
    with pytest.raises(ValueError):
        P._check_device_pair(0, B, B, "test")


def test_new_entry_points_are_bound():
    L = P.lib()
    for name in ("chol_factor_panels", "chol_profile_only", "chol_solve_noalloc"):
        assert name in P.EXPORTS and getattr(L, name) is not None
