"""Edge cases of the GPU path: the widest mesh the sweep's shared memory
holds (and the error just past it), rank one with a single polar cosine, the
rank equal to the number of angles, and zero steps."""
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


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_widest_mesh_the_sweep_holds(orc, dlr, dtype):
    import torch
    td = getattr(torch, dtype)
    dirs = np.array([[0.6, 0.2], [-0.3, 0.7]])
    edge = [0.5, 0.1, 0.3, 0.2]

    def run(nx, ny):
        rng = np.random.default_rng(nx)
        sig = rng.uniform(0.5, 50.0, nx * ny)
        src = rng.uniform(0.0, 1.0, (2, nx * ny))
        psi = dlr.sweep(nx, ny, dirs, edge, torch.tensor(sig, dtype=td, device="cuda"),
                        torch.tensor(src.reshape(-1), dtype=td, device="cuda"))
        return sig, src, psi.cpu().numpy().reshape(2, nx * ny)

    lo, hi = 1, 16384  # lo fits, hi does not
    with pytest.raises(dlr.DlrError):
        run(hi, 8)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        try:
            run(mid, 8)
            lo = mid
        except dlr.DlrError:
            hi = mid
    assert lo >= 1024  # the mesh sides of the benchmark configurations fit
    nx, ny = lo, 40
    sig, src, psi = run(nx, ny)
    p = orc.Problem(nx, ny, 2, 4, np.ones(nx * ny), np.ones(nx * ny), psi_edge=tuple(edge))
    tol = 1e-13 if dtype == "float64" else 2e-6
    for d, (ox, oy) in enumerate(dirs):
        assert rel_l2(psi[d], orc.sweep(p, ox, oy, sig, src[d])) < tol
    with pytest.raises(dlr.DlrError):
        run(nx + 4, ny)


@pytest.mark.parametrize("prec", [0, 1])
def test_rank_one_single_polar_cosine(orc, dlr, prec):
    case = workloads.small_case(17, 13, 1, 1, 4, seed=13, T0=0.45)
    out, _ = run_pair(case, prec, 4, orc=orc, dlr=dlr)
    for eT, ep, oi, gi in out:
        assert eT < TOL[prec] and ep < TOL[prec], (eT, ep)


@pytest.mark.parametrize("prec", [0, 1])
def test_rank_equal_to_the_number_of_angles(orc, dlr, prec):
    case = workloads.small_case(12, 10, 8, 2, 4, seed=14, T0=0.55)
    out, _ = run_pair(case, prec, 3, orc=orc, dlr=dlr)
    for eT, ep, oi, gi in out:
        assert eT < TOL[prec] and ep < TOL[prec], (eT, ep)


@pytest.mark.parametrize("prec", [0, 1])
def test_full_angular_rank_without_readouts(orc, dlr, prec):
    # r = NOm stepped three times with no factor read-out in between (no
    # rotation to the SVD basis from outside): the step itself keeps the
    # SVD basis at full angular rank, and T follows the oracle
    from conftest import oracle_problem
    case = workloads.small_case(12, 10, 8, 2, 4, seed=14, T0=0.55)
    p = oracle_problem(case)
    T = case["T0"].reshape(-1).copy()
    X, S, W = orc.initial_factors(p, T, case["r"])
    with dlr.Solver(dlr.problem_from_case(case, precision=prec)) as s:
        s.set_factors(X, S, W)
        s.step(3)
        assert s.stats()["status"] == 0
        Tg = s.T()
    for _ in range(3):
        X, S, W, T, *_ = orc.dlr_step(p, X, S, W, T, si_tol=1e-13)
    assert rel_l2(Tg, T) < TOL[prec]


def test_zero_steps_is_a_no_op(dlr):
    case = workloads.small_case(9, 7, 3, 2, 4, seed=15, T0=0.3)
    with dlr.Solver(dlr.problem_from_case(case, precision=1)) as s:
        T0 = s.T()
        s.step(0)
        dlr.step_batch([s], 0)
        assert np.array_equal(s.T(), T0) and s.stats()["steps"] == 0
