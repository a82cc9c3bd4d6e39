"""The augmented step on the GPU (step 5 on [Psi, X0], steps 6-8 at rank 2r,
SVD of the 2r x 2r S truncated back to rank r): parity with the oracle's
augmented step through the C ABI (relative L2 on T and psi = X S W^T: 1e-10
FP64, 2e-5 mixed), and on the full space (2r = nx*ny) the weighted rank-r
truncation of the oracle's SN step."""
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


@pytest.mark.parametrize("prec", [0, 1])
def test_augmented_lattice32(orc, dlr, prec):
    out, stats = run_pair(workloads.lattice32(), prec, 6, orc=orc, dlr=dlr, augment=1)
    for k, (eT, ep, oi, gi) in enumerate(out):
        assert eT < TOL[prec] and ep < TOL[prec], (k, eT, ep)
    assert stats["cell_angle_updates"] == stats["si_iters_total"] * 32 * 32 * 6


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(40, 36, 8, 4, 8), (33, 70, 12, 8, 16), (17, 9, 3, 2, 8)])
def test_augmented_ragged(orc, dlr, prec, shape):
    nx, ny, r, npol, naz = shape
    case = workloads.small_case(nx, ny, r, npol, naz, seed=nx + 7 * ny, T0=0.35)
    out, _ = run_pair(case, prec, 3, orc=orc, dlr=dlr, augment=1)
    for k, (eT, ep, oi, gi) in enumerate(out):
        assert eT < TOL[prec] and ep < TOL[prec], (k, eT, ep)


def test_augmented_full_space_is_truncated_sn(orc, dlr):
    from conftest import oracle_problem
    nx, ny, r, npol, naz = 3, 4, 6, 4, 4
    case = workloads.small_case(nx, ny, r, npol, naz, seed=17, T0=0.5)
    p = oracle_problem(case)
    h2 = (1.0 / nx) * (1.0 / ny)
    _, _, _, w = orc.quadrature(npol, naz)
    sw = np.sqrt(w)[None, :]
    T = case["T0"].reshape(-1).copy()
    X, S, W = orc.initial_factors(p, T, r)
    spec = dlr.problem_from_case(case, precision=0, augment=1, si_tol=1e-15)
    with dlr.Solver(spec) as s:
        s.set_factors(X, S, W)
        psi = X @ S @ W.T
        for _ in range(3):
            psi_sn, T, *_ = orc.sn_step(p, psi, T, si_tol=1e-15)
            U, sv, Vt = np.linalg.svd(np.sqrt(h2) * psi_sn * sw, full_matrices=False)
            assert sv[r - 1] - sv[r] > 1e-6 * sv[0]
            target = (U[:, :r] * sv[:r]) @ Vt[:r] / np.sqrt(h2) / sw
            s.step(1)
            psi = s.psi()
            assert rel_l2(psi, target) < 1e-10
            T = s.T()  # the next SN step starts from the GPU state


def test_augmented_batch_equals_alone(orc, dlr):
    import torch
    from conftest import oracle_problem
    cases = [workloads.small_case(30, 26, 5, 4, 8, seed=41, T0=0.4),
             workloads.small_case(21, 44, 8, 4, 8, seed=42, T0=0.6)]
    starts = []
    for c in cases:
        p = oracle_problem(c)
        starts.append(orc.initial_factors(p, c["T0"].reshape(-1).copy(), c["r"]))
    alone = []
    for c, (X, S, W) in zip(cases, starts):
        with dlr.Solver(dlr.problem_from_case(c, precision=1, augment=1)) as s:
            s.set_factors(X, S, W)
            s.step(3)
            alone.append((s.T(), s.psi()))
    st = torch.cuda.Stream()
    ss = [dlr.Solver(dlr.problem_from_case(c, precision=1, augment=1), stream=st) for c in cases]
    try:
        for s, (X, S, W) in zip(ss, starts):
            s.set_factors(X, S, W)
        dlr.step_batch(ss, 3)
        for s, (Ta, pa) in zip(ss, alone):
            assert np.array_equal(s.T(), Ta) and np.array_equal(s.psi(), pa)
    finally:
        for s in ss:
            s.close()


def test_augmented_rejects_bad_shapes(dlr):
    case = workloads.small_case(10, 10, 20, 4, 8, seed=1, T0=0.3)
    with pytest.raises(dlr.DlrError):
        dlr.Solver(dlr.problem_from_case(case, precision=0, augment=1))  # 2r = 40 > 32
