"""Diverging source iterations (Algorithm 1 step 4).  A non-finite scalar
flux is reported, not mistaken for convergence (the stopping test of reading
R7): every source-iteration kernel -- per-angle (FP64 and mixed), grouped,
bilinear elements, full-rank SN -- ends the step with DLR_ENOTCONV after that
iteration (a NaN compares false, so a plain max-of-differences test would
read it as a zero change); the non-finite flux is planted through the
temperature (one NaN cell).  A growing iteration is relaxed (reading R22):
on a state with negative effective scattering (T0 < 0 after a loss of
positivity, sigma_s / sigma_t = -1.44) the plain iteration diverges, and the
GPU's relaxed step matches the oracle's."""
import numpy as np
import pytest

import workloads
from conftest import oracle_problem
from gpu_util import rel_l2

pytestmark = pytest.mark.gpu

ENOTCONV = -3


@pytest.fixture(scope="module")
def dlr():
    import paper_2601_18705_gb300 as m
    return m


@pytest.mark.parametrize("kw", [dict(precision=0), dict(precision=1, sweep_mode=1),
                                dict(precision=1, sweep_mode=2), dict(precision=1, element=1),
                                dict(precision=0, element=1), dict(precision=1, method=1)])
def test_non_finite_flux_stops_the_iteration(dlr, kw):
    case = workloads.small_case(40, 36, 4, 2, 8, seed=2, T0=0.5)
    with dlr.Solver(dlr.problem_from_case(case, **kw)) as s:
        T = s.T()
        T[100] = np.nan
        s.set_T(T)
        with pytest.raises(dlr.DlrError):
            s.step(1)
            s.T()
        st = s.stats()
        assert st["status"] == ENOTCONV
        assert st["si_iters_last"] <= 2


def _negative_T_case():
    nx = ny = 6
    c = workloads.small_case(nx, ny, 4, 2, 8, seed=1, T0=0.714)
    c["sigma"] = np.full((ny, nx), 100.0)
    return c


@pytest.mark.parametrize("kw,tol", [(dict(precision=0), 1e-10), (dict(precision=1, sweep_mode=1), 2e-5),
                                    (dict(precision=1, sweep_mode=2), 2e-5)])
def test_relaxed_step_matches_oracle(orc, dlr, kw, tol):
    c = _negative_T_case()
    p = oracle_problem(c)
    X, S, W = orc.initial_factors(p, c["T0"].reshape(-1), 4)
    T = -c["T0"].reshape(-1).copy()
    X1, S1, W1, T1, res = orc.dlr_step(p, X, S, W, T, si_tol=1e-13, si_max_iter=2000)
    assert res.rc == 0
    spec = dlr.problem_from_case(c, allow_nonpositive=1, si_tol=1e-13 if kw["precision"] == 0 else 0.0, **kw)
    with dlr.Solver(spec) as s:
        s.set_factors(X, S, W)
        s.set_T(T)
        s.step(1)
        st = s.stats()
        assert st["status"] == 0 and st["si_iters_last"] < 200
        assert rel_l2(s.T(), T1) < tol
        assert rel_l2(s.psi(), X1 @ S1 @ W1.T) < tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 2e-5)])
def test_relaxed_q1_step_matches_oracle(orc, dlr, prec, tol):
    c = _negative_T_case()
    p = oracle_problem(c)
    X, S, W = orc.initial_factors(p, c["T0"].reshape(-1), 4)
    Xq = np.zeros((4 * p.Nx, 4), order="F")
    Xq[0::4, :] = X
    T = -c["T0"].reshape(-1).copy()
    X1, S1, W1, T1, phi, it, rc = orc.dlr_step_q1(p, Xq, S, W, T, si_tol=1e-13, si_max_iter=2000)
    assert rc == 0
    spec = dlr.problem_from_case(c, precision=prec, element=1, allow_nonpositive=1,
                                 si_tol=1e-13 if prec == 0 else 0.0)
    with dlr.Solver(spec) as s:
        s.set_factors(Xq, S, W)
        s.set_T(T)
        s.step(1)
        assert s.stats()["status"] == 0
        assert rel_l2(s.T(), T1) < tol
        assert rel_l2(s.psi(), X1 @ S1 @ W1.T) < tol
