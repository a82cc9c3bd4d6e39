"""Temperature-dependent opacity and heat capacity on the GPU, taken at each
step's T0 (Eq. T backward Euler; power laws of reading R16): parity with the
oracle through the C ABI for the DLR step and the full-rank SN step
(relative L2 on T and psi: 1e-10 FP64, 2e-5 mixed)."""
import numpy as np
import pytest

import workloads
from gpu_util import rel_l2, run_pair

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 2e-5}


@pytest.fixture(scope="module")
def dlr():
    import paper_2601_18705_gb300 as m
    return m


def _case(nx, ny, r, seed, n_s, n_c):
    c = workloads.small_case(nx, ny, r, 4, 8, seed=seed, T0=0.35)
    T0 = 0.2 + 0.5 * np.random.default_rng(seed).random((ny, nx))  # non-uniform T0
    c.update(T0=T0, sigma_texp=n_s, cv_texp=n_c, T_ref=0.5)
    return c


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_s,n_c", [(3.0, 0.0), (1.5, 1.0)])
def test_dlr_with_temperature_dependent_materials(orc, dlr, prec, n_s, n_c):
    case = _case(29, 23, 6, 3, n_s, n_c)
    out, _ = run_pair(case, prec, 3, orc=orc, dlr=dlr)
    for k, (eT, ep, oi, gi) in enumerate(out):
        assert eT < TOL[prec] and ep < TOL[prec], (k, eT, ep)


def test_zero_exponents_are_the_constant_materials(dlr):
    case = workloads.small_case(20, 17, 4, 4, 8, seed=5, T0=0.4)
    out = []
    for extra in ({}, {"sigma_texp": 0.0, "cv_texp": 0.0, "T_ref": 0.3}):
        c = dict(case, **extra)
        with dlr.Solver(dlr.problem_from_case(c, precision=1)) as s:
            s.step(3)
            out.append(s.T())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec", [0, 1])
def test_sn_with_temperature_dependent_materials(orc, dlr, prec):
    from conftest import oracle_problem
    case = _case(13, 11, 1, 7, 3.0, 1.0)
    p = oracle_problem(case)
    K = case["n_polar"] * case["n_azim"]
    T = case["T0"].reshape(-1).copy()
    psi = np.repeat((case["a_rad"] * case["c"] * T ** 4 / (4 * np.pi))[:, None], K, axis=1)
    spec = dlr.problem_from_case(case, precision=prec, method=dlr.DLR_METHOD_SN,
                                 si_tol=1e-13 if prec == 0 else 0.0)
    with dlr.Solver(spec) as s:
        for _ in range(3):
            psi, T, *_ = orc.sn_step(p, psi, T, si_tol=1e-13)
            s.step(1)
            assert rel_l2(s.T(), T) < TOL[prec]
            assert rel_l2(s.psi(), psi) < TOL[prec]
