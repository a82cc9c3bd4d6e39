"""A diverged source iteration (Algorithm 1 step 4; the stopping test of
reading R7) is reported, not mistaken for convergence: once the scalar flux
is no longer finite every source-iteration kernel -- per-angle (FP64 and
mixed), grouped, bilinear elements, full-rank SN -- ends the step with
DLR_ENOTCONV after that iteration (a NaN compares false, so a plain
max-of-differences test would read it as a zero change).  The non-finite
flux is planted through the temperature (one NaN cell)."""
import numpy as np
import pytest

import workloads

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
