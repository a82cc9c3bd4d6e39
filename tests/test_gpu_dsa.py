"""Diffusion synthetic acceleration on the GPU (Section 4.5): the DG0
diffusion correction solved by Jacobi-preconditioned CG inside the
source-iteration launch, for the DLR step and the full-rank SN step.
Parity with the oracle through the C ABI: relative L2 on T and psi within
1e-10 (FP64) and 2e-5 (mixed); in FP64 the source-iteration counts match the
oracle's.  The accelerated and the plain iteration reach the same step, and
a batch mixing accelerated and plain instances equals the instances alone."""
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


def _thick(nx, ny, r, npol, naz, seed, scale=10.0, T0=1.0):
    """A lattice case made optically thick and hot: sigma in [10, 1000] per
    4x4 block (the scattering ratio sigma_s / sigma_t close to 1)."""
    c = workloads.small_case(nx, ny, r, npol, naz, seed=seed, T0=T0)
    c["sigma"] = c["sigma"] * scale
    return c


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(37, 29, 6, 4, 8), (5, 64, 4, 2, 8), (2, 3, 4, 2, 4)])
def test_dlr_dsa_matches_oracle(orc, dlr, prec, shape):
    nx, ny, r, npol, naz = shape
    case = _thick(nx, ny, r, npol, naz, seed=nx * ny + 1)
    iters = []
    out, st = run_pair(case, prec, 3, orc=orc, dlr=dlr, si_tol=1e-13 if prec == 0 else None,
                       dsa=1, iters_out=iters)
    for eT, epsi, _, _ in out:
        assert eT < TOL[prec] and epsi < TOL[prec], out
    if prec == 0:
        for it_o, it_g, _ in iters:
            assert abs(it_o - it_g) <= 1, iters
    assert st["dsa_iters_total"] > 0


def test_dsa_cuts_iterations_and_keeps_the_step(dlr):
    case = _thick(40, 33, 6, 4, 8, seed=5)
    res = {}
    for dsa in (0, 1):
        spec = dlr.problem_from_case(case, precision=0, si_tol=1e-12, si_max_iter=20000, dsa=dsa)
        with dlr.Solver(spec) as s:
            s.step(2)
            res[dsa] = (s.T(), s.psi(), s.stats())
    assert rel_l2(res[1][0], res[0][0]) < 1e-9
    assert rel_l2(res[1][1], res[0][1]) < 1e-9
    assert res[1][2]["si_iters_total"] * 4 < res[0][2]["si_iters_total"], (
        res[0][2]["si_iters_total"], res[1][2]["si_iters_total"])
    assert res[0][2]["dsa_iters_total"] == 0 and res[1][2]["dsa_iters_total"] > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_sn_dsa_matches_oracle(orc, dlr, prec):
    from conftest import oracle_problem
    case = _thick(19, 23, 1, 2, 8, seed=13)
    p = oracle_problem(case)
    p.dsa, p.dsa_tol, p.dsa_max_iter = 1, 0.1, 500
    K = 16
    T = case["T0"].reshape(-1).copy()
    psi = np.repeat((case["a_rad"] * case["c"] * T ** 4 / (4 * np.pi))[:, None], K, axis=1)
    spec = dlr.problem_from_case(case, precision=prec, method=dlr.DLR_METHOD_SN,
                                 si_tol=1e-13 if prec == 0 else 0.0, dsa=1)
    with dlr.Solver(spec) as s:
        for _ in range(3):
            psi, T, phi, it, *_ = orc.sn_step(p, psi, T, si_tol=1e-13)
            assert it > 0
            s.step(1)
            assert rel_l2(s.T(), T) < TOL[prec]
            assert rel_l2(s.psi(), psi) < TOL[prec]
            if prec == 0:
                assert abs(s.stats()["si_iters_last"] - it) <= 1


def test_batch_mixing_dsa_and_plain(dlr):
    import torch
    cases = [_thick(24, 20, 6, 4, 8, seed=21), _thick(31, 17, 4, 2, 8, seed=22)]
    flags = [1, 0]
    alone = []
    for c, f in zip(cases, flags):
        with dlr.Solver(dlr.problem_from_case(c, precision=0, si_tol=1e-12, dsa=f)) as s:
            s.step(2)
            alone.append((s.T(), s.psi()))
    stream = torch.cuda.Stream()
    solvers = [dlr.Solver(dlr.problem_from_case(c, precision=0, si_tol=1e-12, dsa=f), stream=stream)
               for c, f in zip(cases, flags)]
    try:
        dlr.step_batch(solvers, 2)
        got = [(s.T(), s.psi()) for s in solvers]
    finally:
        for s in solvers:
            s.close()
    # the plain instance does not see the other's CG: bit for bit
    assert np.array_equal(got[1][0], alone[1][0]) and np.array_equal(got[1][1], alone[1][1])
    # the accelerated one sums its CG partials over a different grid
    assert rel_l2(got[0][0], alone[0][0]) < 1e-11 and rel_l2(got[0][1], alone[0][1]) < 1e-11


def test_dsa_checker256_full_size_same_step(dlr):
    # the 256 x 256 checkerboard (16 x 32 angles, rank 16) in FP64: the
    # accelerated iteration reaches the plain one's step
    case = workloads.checker256(precision="fp64")
    res = {}
    for dsa in (0, 1):
        spec = dlr.problem_from_case(case, precision=0, si_tol=1e-12, dsa=dsa,
                                     allow_nonpositive=1)
        with dlr.Solver(spec) as s:
            s.step(3)
            res[dsa] = (s.T(), s.stats())
    assert rel_l2(res[1][0], res[0][0]) < 1e-8
    assert res[1][1]["si_iters_total"] <= res[0][1]["si_iters_total"]


def test_dsa_bad_arguments(dlr):
    case = workloads.small_case(8, 8, 2, 2, 4)
    for kw in ({"dsa": 2}, {"dsa": 1, "dsa_tol": 1.5}):
        with pytest.raises(dlr.DlrError):
            dlr.Solver(dlr.problem_from_case(case, precision=0, **kw))
