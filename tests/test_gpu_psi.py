"""dlr_get_psi on DLR handles: psi = X S W^T formed on the device (Section 4,
the low-rank form of the angular flux) equals the product of the factors
that dlr_get_factors returns, on DG0 cells and on bilinear elements (plain
Legendre coefficients), in FP64 (1e-12: rounding of the canonical rotation
and of the product) and mixed precision (1e-6: the rotation of the FP32 X)."""
import numpy as np
import pytest

import workloads
from gpu_util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dlr():
    import paper_2601_18705_gb300 as m
    return m


@pytest.mark.parametrize("element", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_dlr_psi_is_the_factor_product(dlr, element, prec):
    case = workloads.small_case(13, 11, 5, 2, 8, seed=3, T0=0.4)
    with dlr.Solver(dlr.problem_from_case(case, precision=prec, element=element)) as s:
        for _ in range(2):
            s.step(1)
            psi = s.psi()
            X, S, W = s.factors()
            assert psi.shape == ((4 if element else 1) * 13 * 11, 2 * 8)
            assert rel_l2(psi, X @ S @ W.T) < (1e-12 if prec == 0 else 1e-6)
