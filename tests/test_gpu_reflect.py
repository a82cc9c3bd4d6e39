"""Reflective edges on the GPU.  Full-rank SN (reading R18): a direction
entering a reflective edge takes its mirror direction's boundary values from
the previous source iteration, injected as a boundary source of the sweep.
DLR (reading R19): the collocation sweeps take the mirror angle's value
interpolated through the chosen angles, and the L-step solves its reflected
inflow by a fixed point on the boundary values.  Parity with the oracle
through the C ABI: relative L2 on T and psi within 1e-10 (FP64) and 2e-5
(mixed); at full rank the DLR step equals the SN step; an all-reflective
uniform medium follows the 0-D recurrence; odd azimuth counts (x mirror) and
the augmented step are refused."""
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
    with pytest.raises(dlr.DlrError):   # the augmented step
        dlr.Solver(dlr.problem_from_case(case, precision=0, reflect=(1, 0, 0, 0), augment=1))
    case = workloads.small_case(8, 8, 1, 2, 5)
    with pytest.raises(dlr.DlrError):   # x mirror needs an even azimuth count
        dlr.Solver(dlr.problem_from_case(case, precision=0, method=dlr.DLR_METHOD_SN,
                                         reflect=(0, 1, 0, 0)))
    with pytest.raises(dlr.DlrError):
        dlr.Solver(dlr.problem_from_case(case, precision=0, reflect=(1, 0, 0, 0)))
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


# ---------------------------------------------------------------------------
# DLR with reflective edges (reading R19)
# ---------------------------------------------------------------------------

def _hot_case(nx, ny, r, npol, naz):
    case = workloads.small_case(nx, ny, r, npol, naz, seed=nx + ny + r, T0=0.4)
    T0 = case["T0"].copy()
    T0.reshape(-1)[: nx * 2] = 0.9  # a hot strip along the bottom rows
    case["T0"] = T0
    case["T_edge"] = (0.6, -1.0, 0.3, -1.0)
    return case


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,r,reflect", [((12, 10, 2, 8), 4, (1, 0, 0, 0)),
                                             ((37, 29, 2, 8), 6, (0, 1, 1, 0)),
                                             ((21, 40, 4, 8), 8, (1, 1, 1, 1)),
                                             ((70, 33, 2, 6), 5, (0, 0, 0, 1))])
def test_dlr_reflective_matches_oracle(orc, dlr, prec, shape, r, reflect):
    nx, ny, npol, naz = shape
    case = _hot_case(nx, ny, r, npol, naz)
    out, stats = run_pair(case, prec, 3, orc=orc, dlr=dlr, reflect=reflect,
                          si_tol=1e-13 if prec == 0 else None)
    for eT, ep, *_ in out:
        assert eT < TOL[prec] and ep < TOL[prec], out
    assert stats["refl_passes_last"] > 1
    assert stats["status"] == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_dlr_reflective_rank32_matches_oracle(orc, dlr, prec):
    # rank class 32 and more than 1024 angles (the unfused step 8)
    case = _hot_case(24, 20, 32, 16, 72)
    out, stats = run_pair(case, prec, 2, orc=orc, dlr=dlr, reflect=(1, 0, 1, 1),
                          si_tol=1e-13 if prec == 0 else None)
    for eT, ep, *_ in out:
        assert eT < TOL[prec] and ep < TOL[prec], out


@pytest.mark.parametrize("reflect", [(1, 0, 0, 0), (0, 1, 1, 0), (1, 1, 1, 1)])
def test_dlr_full_rank_reflective_equals_sn(dlr, reflect):
    # at full rank (r = number of cells) the DLR step is the SN step, also
    # behind reflective edges: both GPU paths, from the same isotropic state
    n = 3
    case = workloads.small_case(n, n, n * n, 2, 8, seed=n + 7, T0=0.5)
    T0 = case["T0"].copy()
    T0.reshape(-1)[0] = 0.9
    case["T0"] = T0
    case["T_edge"] = (0.6, 0.4, 0.3, -1.0)
    d = dlr.problem_from_case(case, precision=0, si_tol=1e-14, reflect=reflect)
    s = dlr.problem_from_case(case, precision=0, method=dlr.DLR_METHOD_SN, si_tol=1e-14,
                              reflect=reflect)
    with dlr.Solver(d) as a, dlr.Solver(s) as b:
        for _ in range(3):
            a.step(1)
            b.step(1)
            assert rel_l2(a.T(), b.T()) < 1e-10
            assert rel_l2(a.psi(), b.psi()) < 1e-10


@pytest.mark.parametrize("r", [1, 3])
def test_dlr_all_reflective_uniform_medium(dlr, r):
    nx, ny, sig, rho, T0, dt = 40, 36, 10.0, 0.5, 0.5, 0.02
    case = workloads.small_case(nx, ny, r, 4, 8, T0=T0)
    case["sigma"] = np.full((ny, nx), sig)
    case["rho_cv"] = np.full((ny, nx), rho)
    case["dt"] = dt
    a, c = case["a_rad"], case["c"]
    Tz, phiz = T0, a * c * T0 ** 4
    spec = dlr.problem_from_case(case, precision=0, si_tol=1e-14, reflect=(1, 1, 1, 1))
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
        # the collocation fluxes of an isotropic state are equal up to
        # rounding: step 5 completes the basis instead of keeping copies
        X, S, W = s.factors()
        h2 = 1.0 / (nx * ny)
        np.testing.assert_allclose(h2 * X.T @ X, np.eye(r), atol=1e-12)
        assert s.stats()["refl_passes_last"] <= 3


def test_dlr_reflective_batch_equals_alone(dlr):
    import torch
    a = _hot_case(33, 70, 6, 2, 8)
    b = _hot_case(19, 23, 4, 4, 8)
    refl = [(1, 0, 1, 0), (0, 0, 0, 0)]
    alone = []
    for c, rf in zip((a, b), refl):
        with dlr.Solver(dlr.problem_from_case(c, precision=1, reflect=rf)) as s:
            s.step(2)
            alone.append((s.T(), s.stats()["refl_passes_last"]))
    st = torch.cuda.Stream()
    ss = [dlr.Solver(dlr.problem_from_case(c, precision=1, reflect=rf), stream=st)
          for c, rf in zip((a, b), refl)]
    try:
        dlr.step_batch(ss, 2)
        got = [(s.T(), s.stats()["refl_passes_last"]) for s in ss]
    finally:
        for s in ss:
            s.close()
    for (Ta, pa), (Tg, pg) in zip(alone, got):
        assert np.array_equal(Ta, Tg) and pa == pg
    assert alone[0][1] > 1 and alone[1][1] == 0


def test_dlr_reflective_with_dsa_matches_oracle(orc, dlr):
    case = _hot_case(23, 19, 6, 2, 8)
    case["sigma"] = case["sigma"] * 10.0
    out, stats = run_pair(case, 0, 2, orc=orc, dlr=dlr, reflect=(1, 0, 1, 0), dsa=1, dsa_tol=0.1,
                          dsa_max_iter=3, si_tol=1e-13)
    for eT, ep, *_ in out:
        assert eT < TOL[0] and ep < TOL[0], out
    assert stats["dsa_iters_total"] > 0
