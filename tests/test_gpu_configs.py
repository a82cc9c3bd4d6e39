"""Full-size workloads on the GPU (the sizes the benchmark runs): checker256
against the oracle and FP64 against mixed; lognormal1024 FP64 against mixed
plus positivity (the oracle is too slow there, so properties stand in)."""
import numpy as np
import pytest

import workloads
from gpu_util import rel_l2, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dlr():
    import paper_2601_18705_gb300 as m
    return m


def test_checker256_fp64_vs_oracle(orc, dlr):
    out, stats = run_pair(workloads.checker256(), 0, 2, orc=orc, dlr=dlr)
    for eT, ep, oi, gi in out:
        assert eT < 1e-10 and ep < 1e-10, (eT, ep)


def test_checker256_mixed_vs_fp64(dlr):
    case = workloads.checker256()
    res = {}
    for prec in (0, 1):
        with dlr.Solver(dlr.problem_from_case(case, precision=prec)) as s:
            s.step(5)
            res[prec] = (s.T(), s.psi(), s.stats())
    assert rel_l2(res[1][0], res[0][0]) < 2e-5
    assert rel_l2(res[1][1], res[0][1]) < 2e-5
    assert res[1][2]["steps"] == 5


def test_lognormal1024_mixed_vs_fp64(dlr):
    case = workloads.lognormal1024()
    res = {}
    for prec in (0, 1):
        with dlr.Solver(dlr.problem_from_case(case, precision=prec)) as s:
            s.step(2)
            res[prec] = (s.T(), s.stats())
    assert res[1][0].min() > 0 and res[0][0].min() > 0
    assert rel_l2(res[1][0], res[0][0]) < 2e-5
