"""GPU parity of the whole SN-like DLR step (Algorithm 1) against the oracle,
through the C ABI.  Tolerances: relative L2 on T and on psi = X S W^T of
1e-10 (FP64 path) and 2e-5 (mixed FP32/FP64 path)."""
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


def test_lattice32_fp64_ten_steps(orc, dlr):
    out, stats = run_pair(workloads.lattice32(), 0, 10, orc=orc, dlr=dlr)
    for k, (eT, ep, oi, gi) in enumerate(out):
        assert eT < 1e-10 and ep < 1e-10, (k, eT, ep)
    assert stats["steps"] == 10 and stats["si_iters_total"] > 10


def test_lattice32_mixed(orc, dlr):
    out, _ = run_pair(workloads.lattice32(), 1, 10, orc=orc, dlr=dlr)
    for k, (eT, ep, oi, gi) in enumerate(out):
        assert eT < 2e-5 and ep < 2e-5, (k, eT, ep)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(40, 36, 8, 4, 8), (67, 33, 5, 4, 8), (33, 70, 12, 8, 16),
                                   (5, 7, 3, 2, 8), (1, 40, 2, 2, 8), (90, 3, 6, 4, 8)])
def test_ragged_meshes(orc, dlr, prec, shape):
    nx, ny, r, npol, naz = shape
    case = workloads.small_case(nx, ny, r, npol, naz, seed=nx + 3 * ny, T0=0.35)
    out, _ = run_pair(case, prec, 3, orc=orc, dlr=dlr)
    for k, (eT, ep, oi, gi) in enumerate(out):
        assert eT < TOL[prec] and ep < TOL[prec], (k, eT, ep)


def test_deim_selection(orc, dlr):
    case = workloads.small_case(24, 20, 6, 4, 8, seed=11, T0=0.3)
    out, _ = run_pair(case, 0, 3, orc=orc, dlr=dlr, selection=1)
    for eT, ep, oi, gi in out:
        assert eT < 1e-10 and ep < 1e-10


def test_fixed_iterations(orc, dlr):
    case = workloads.small_case(30, 26, 6, 4, 8, seed=12, T0=0.8)
    out, stats = run_pair(case, 0, 2, orc=orc, dlr=dlr, si_fixed_iters=3)
    for eT, ep, oi, gi in out:
        assert eT < 1e-10 and ep < 1e-10
    assert stats["si_iters_total"] == 6


@pytest.mark.parametrize("n,npol,naz", [(3, 2, 8), (4, 4, 8)])
def test_full_rank_equals_sn(orc, dlr, n, npol, naz):
    from conftest import oracle_problem
    case = workloads.small_case(n, n, n * n, npol, naz, seed=n, T0=0.5)
    p = oracle_problem(case)
    T = case["T0"].reshape(-1).copy()
    X, S, W = orc.initial_factors(p, T, n * n)
    psi = X @ S @ W.T
    spec = dlr.problem_from_case(case, precision=0)
    with dlr.Solver(spec) as s:
        s.set_factors(X, S, W)
        for _ in range(3):
            psi, T, *_ = orc.sn_step(p, psi, T, si_tol=1e-15)
            s.step(1)
            assert rel_l2(s.T(), T) < 1e-10
            assert rel_l2(s.psi(), psi) < 1e-10


def test_infinite_medium_recurrence(dlr):
    nx, ny, sig, rho, T0, dt = 20, 17, 10.0, 0.5, 0.5, 0.02
    a, c = workloads.A_RAD, workloads.C_LIGHT
    spec = dlr.ProblemSpec(nx=nx, ny=ny, n_polar=4, n_azim=8, rank=3, sigma=np.full(nx * ny, sig),
                           rho_cv=np.full(nx * ny, rho), T0=np.full(nx * ny, T0), dt=dt,
                           precision=0)
    Tz, phiz = T0, a * c * T0 ** 4
    with dlr.Solver(spec) as s:
        for _ in range(20):
            B0 = a * c * Tz ** 4 / (4 * np.pi)
            dB = a * c * Tz ** 3 / np.pi
            D = rho + 4 * np.pi * dt * sig * dB
            ss = sig * 4 * np.pi * dt * sig * dB / D
            q = sig * B0 * rho / D
            phiz = (4 * np.pi * q + phiz / (c * dt)) / (sig - ss + 1 / (c * dt))
            Tz = Tz + dt * sig * (phiz - 4 * np.pi * B0) / D
            for e in range(4):
                s.set_edge_inflow(e, phiz / (4 * np.pi))
            s.step(1)
            np.testing.assert_allclose(s.T(), Tz, rtol=1e-12)


def test_equilibrium_preserved(dlr):
    case = workloads.small_case(30, 20, 5, 4, 8, seed=2, T0=0.7)
    spec = dlr.problem_from_case(case, precision=0)
    spec.T_edge = (0.7, 0.7, 0.7, 0.7)
    with dlr.Solver(spec) as s:
        s.step(3)
        np.testing.assert_allclose(s.T(), 0.7, rtol=1e-12)


def test_batch_equals_alone(dlr):
    cases = [workloads.small_case(24 + 7 * i, 20 + 5 * i, 4 + 2 * i, 4, 8, seed=20 + i, T0=0.3)
             for i in range(4)]
    for prec in (0, 1):
        alone = []
        for cs in cases:
            with dlr.Solver(dlr.problem_from_case(cs, precision=prec)) as s:
                s.step(3)
                alone.append(s.T())
        import torch
        st = torch.cuda.Stream()
        solvers = [dlr.Solver(dlr.problem_from_case(cs, precision=prec), stream=st) for cs in cases]
        dlr.step_batch(solvers, 3)
        for s, Ta in zip(solvers, alone):
            assert np.array_equal(s.T(), Ta)
            s.close()


def test_not_converged_status(dlr):
    case = workloads.small_case(20, 20, 4, 4, 8, seed=5, T0=0.9)
    spec = dlr.problem_from_case(case, precision=0)
    spec.si_tol, spec.si_max_iter = 1e-300, 2
    with dlr.Solver(spec) as s:
        s.step(1)
        with pytest.raises(dlr.DlrError) as e:
            s.T()
        assert "ENOTCONV" in str(e.value)
        with pytest.raises(dlr.DlrError):
            s.step(1)


def test_hbm_budget_rejects(dlr):
    spec = dlr.problem_from_case(workloads.lattice32())
    with pytest.raises(dlr.DlrError) as e:
        dlr.Solver(spec, hbm_budget=1024)
    assert "ENOMEM" in str(e.value)
