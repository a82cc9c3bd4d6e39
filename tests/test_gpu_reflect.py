"""Reflective edges on the GPU (full-rank SN, reading R18): a direction
entering a reflective edge takes its mirror direction's boundary values from
the previous source iteration, injected as a boundary source of the sweep.
Parity with the oracle through the C ABI: relative L2 on T and psi within
1e-10 (FP64) and 2e-5 (mixed); an all-reflective uniform medium follows the
0-D recurrence; DLR instances and odd azimuth counts are refused."""
import numpy as np
import pytest

import workloads
from gpu_util import rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 2e-5}


@pytest.fixture(scope="module")
def dlr():
    import paper_2601_18705_gb300 as m
    return m


def _planck_psi(case, K):
    T0 = case["T0"].reshape(-1)
    return np.repeat((case["a_rad"] * case["c"] * T0 ** 4 / (4 * np.pi))[:, None], K, axis=1)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,reflect", [((12, 10, 4, 8), (1, 0, 0, 0)),
                                           ((37, 29, 2, 8), (0, 1, 1, 0)),
                                           ((5, 64, 2, 4), (1, 1, 1, 1)),
                                           ((70, 33, 2, 6), (0, 0, 0, 1))])
def test_sn_reflective_matches_oracle(orc, dlr, prec, shape, reflect):
    from conftest import oracle_problem
    nx, ny, npol, naz = shape
    case = workloads.small_case(nx, ny, 1, npol, naz, seed=nx + ny, T0=0.4)
    T0 = case["T0"].copy()
    T0.reshape(-1)[: nx * 2] = 0.9  # a hot strip along the bottom rows
    case["T0"] = T0
    case["T_edge"] = (0.6, -1.0, 0.3, -1.0)
    p = oracle_problem(case)
    p.reflect = reflect
    K = npol * naz
    T = case["T0"].reshape(-1).copy()
    psi = _planck_psi(case, K)
    spec = dlr.problem_from_case(case, precision=prec, method=dlr.DLR_METHOD_SN,
                                 si_tol=1e-13 if prec == 0 else 0.0, reflect=reflect)
    with dlr.Solver(spec) as s:
        for _ in range(3):
            psi, T, phi, it, *_ = orc.sn_step(p, psi, T, si_tol=1e-13, si_max_iter=20000)
            assert it > 0
            s.step(1)
            assert rel_l2(s.T(), T) < TOL[prec]
            assert rel_l2(s.psi(), psi) < TOL[prec]
            if prec == 0:
                assert abs(s.stats()["si_iters_last"] - it) <= 1


def test_sn_all_reflective_uniform_medium(dlr):
    nx, ny, sig, rho, T0, dt = 40, 36, 10.0, 0.5, 0.5, 0.02
    case = workloads.small_case(nx, ny, 1, 2, 8, T0=T0)
    case["sigma"] = np.full((ny, nx), sig)
    case["rho_cv"] = np.full((ny, nx), rho)
    case["dt"] = dt
    a, c = case["a_rad"], case["c"]
    Tz, phiz = T0, a * c * T0 ** 4
    spec = dlr.problem_from_case(case, precision=0, method=dlr.DLR_METHOD_SN, si_tol=1e-14,
                                 reflect=(1, 1, 1, 1))
    with dlr.Solver(spec) as s:
        for _ in range(10):
            B0 = a * c * Tz ** 4 / (4 * np.pi)
            dB = a * c * Tz ** 3 / np.pi
            D = rho + 4 * np.pi * dt * sig * dB
            ss = sig * 4 * np.pi * dt * sig * dB / D
            q = sig * B0 * rho / D
            phiz = (4 * np.pi * q + phiz / (c * dt)) / (sig - ss + 1 / (c * dt))
            Tz = Tz + dt * sig * (phiz - 4 * np.pi * B0) / D
            s.step(1)
            np.testing.assert_allclose(s.T(), Tz, rtol=1e-12)


def test_sn_reflective_batch_equals_alone(dlr):
    import torch
    a = workloads.small_case(33, 300, 1, 2, 8, seed=3, T0=0.6)
    b = workloads.small_case(19, 23, 1, 4, 8, seed=4, T0=0.5)
    refl = [(1, 0, 1, 0), (0, 0, 0, 0)]
    alone = []
    for c, r in zip((a, b), refl):
        with dlr.Solver(dlr.problem_from_case(c, precision=1, method=dlr.DLR_METHOD_SN, reflect=r)) as s:
            s.step(2)
            alone.append((s.T(), s.psi()))
    st = torch.cuda.Stream()
    ss = [dlr.Solver(dlr.problem_from_case(c, precision=1, method=dlr.DLR_METHOD_SN, reflect=r), stream=st)
          for c, r in zip((a, b), refl)]
    try:
        dlr.step_batch(ss, 2)
        got = [(s.T(), s.psi()) for s in ss]
    finally:
        for s in ss:
            s.close()
    for (Ta, pa), (Tg, pg) in zip(alone, got):
        assert np.array_equal(Ta, Tg) and np.array_equal(pa, pg)


def test_reflective_refusals(dlr):
    case = workloads.small_case(8, 8, 2, 2, 6)
    with pytest.raises(dlr.DlrError):   # DLR method
        dlr.Solver(dlr.problem_from_case(case, precision=0, reflect=(1, 0, 0, 0)))
    case = workloads.small_case(8, 8, 1, 2, 5)
    with pytest.raises(dlr.DlrError):   # x mirror needs an even azimuth count
        dlr.Solver(dlr.problem_from_case(case, precision=0, method=dlr.DLR_METHOD_SN,
                                         reflect=(0, 1, 0, 0)))
    with dlr.Solver(dlr.problem_from_case(case, precision=0, method=dlr.DLR_METHOD_SN,
                                          reflect=(0, 0, 1, 1))) as s:  # y mirror: any count
        s.step(1)


@pytest.mark.parametrize("prec", [0, 1])
def test_sn_reflective_with_dsa_matches_oracle(orc, dlr, prec):
    from conftest import oracle_problem
    case = workloads.small_case(23, 19, 1, 2, 8, seed=8, T0=1.0)
    case["sigma"] = case["sigma"] * 10.0
    reflect = (1, 0, 1, 0)
    p = oracle_problem(case)
    p.reflect = reflect
    p.dsa, p.dsa_tol, p.dsa_max_iter = 1, 0.1, 3
    T = case["T0"].reshape(-1).copy()
    psi = _planck_psi(case, 16)
    spec = dlr.problem_from_case(case, precision=prec, method=dlr.DLR_METHOD_SN,
                                 si_tol=1e-13 if prec == 0 else 0.0, reflect=reflect, dsa=1)
    with dlr.Solver(spec) as s:
        for _ in range(2):
            psi, T, phi, it, *_ = orc.sn_step(p, psi, T, si_tol=1e-13, si_max_iter=20000)
            s.step(1)
            assert rel_l2(s.T(), T) < TOL[prec]
            assert rel_l2(s.psi(), psi) < TOL[prec]
        assert s.stats()["dsa_iters_total"] > 0
