"""Bilinear (Q1) elements on the GPU (Section 4.4 with the paper's bilinear
elements; the upwind DG system per cell in the Legendre basis 1, xi, eta,
xi eta): the SN-like DLR step against oracle_dlr_step_q1 and the full-rank SN
step against oracle_sn_step_q1, through the C ABI, on ragged meshes and on
the full lattice32 mesh; relative L2 on T and on psi (4 Nx coefficients x
NOm) within 1e-10 (FP64) and 2e-5 (mixed: FP32 sweeps and projections).
Also: at full rank (r = 4 Nx) the GPU DLR step equals the GPU SN step, a
uniform medium follows the 0-D recurrence, batches equal single runs, and
the unsupported combinations are refused."""
import numpy as np
import pytest

import workloads
from conftest import oracle_problem
from gpu_util import rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 2e-5}


@pytest.fixture(scope="module")
def dlr():
    import paper_2601_18705_gb300 as m
    return m


def _q1_start(orc, p, T, r):
    """The oracle's DG0 initial factors as Q1 fields (each cell's constant
    coefficient; orthonormal in the Q1 inner product)."""
    X, S, W = orc.initial_factors(p, T, r)
    Xq = np.zeros((4 * p.Nx, r), order="F")
    Xq[0::4, :] = X
    return Xq, S, W


def _hot(nx, ny, r, npol, naz, edges=(0.6, -1.0, 0.3, -1.0)):
    case = workloads.small_case(nx, ny, r, npol, naz, seed=nx + 2 * ny + r, T0=0.4)
    T0 = case["T0"].copy()
    T0.reshape(-1)[: nx * 2] = 0.9
    case["T0"] = T0
    case["T_edge"] = edges
    return case


def _dlr_pair(orc, dlr, case, steps, prec=0):
    p = oracle_problem(case)
    T = case["T0"].reshape(-1).copy()
    X, S, W = _q1_start(orc, p, T, case["r"])
    spec = dlr.problem_from_case(case, precision=prec, element=1, si_tol=1e-13 if prec == 0 else 0.0)
    out = []
    with dlr.Solver(spec) as s:
        s.set_factors(X, S, W)
        for _ in range(steps):
            X, S, W, T, phi, it, rc = orc.dlr_step_q1(p, X, S, W, T, si_tol=1e-13, si_max_iter=20000)
            assert rc == 0
            s.step(1)
            st = s.stats()
            assert st["status"] == 0
            out.append((rel_l2(s.T(), T), rel_l2(s.psi(), X @ S @ W.T), it, st["si_iters_last"]))
    return out


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,r", [((12, 10, 2, 8), 4), ((37, 29, 2, 8), 6), ((5, 64, 4, 8), 8),
                                     ((70, 33, 2, 6), 5), ((1, 40, 2, 8), 3)])
def test_dlr_q1_matches_oracle(orc, dlr, shape, r, prec):
    nx, ny, npol, naz = shape
    out = _dlr_pair(orc, dlr, _hot(nx, ny, r, npol, naz), 3, prec)
    for eT, ep, it, git in out:
        assert eT < TOL[prec] and ep < TOL[prec], out
        if prec == 0:
            assert abs(it - git) <= 1, out


@pytest.mark.parametrize("prec", [0, 1])
def test_dlr_q1_rank32_many_angles(orc, dlr, prec):
    # rank class 32 and more than 1024 angles (the unfused step 8)
    out = _dlr_pair(orc, dlr, _hot(24, 20, 32, 16, 72), 2, prec)
    for eT, ep, *_ in out:
        assert eT < TOL[prec] and ep < TOL[prec], out


@pytest.mark.parametrize("prec", [0, 1])
def test_dlr_q1_lattice32_full_size(orc, dlr, prec):
    case = workloads.lattice32()
    out = _dlr_pair(orc, dlr, case, 2, prec)
    for eT, ep, *_ in out:
        assert eT < TOL[prec] and ep < TOL[prec], out


def _q1_planck(case, K):
    T = case["T0"].reshape(-1)
    B = case["a_rad"] * case["c"] * T ** 4 / (4 * np.pi)
    psi = np.zeros((K, T.size, 4))
    psi[:, :, 0] = B[None, :]
    return psi


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(12, 10, 2, 8), (37, 29, 2, 4), (5, 64, 2, 8)])
def test_sn_q1_matches_oracle(orc, dlr, shape, prec):
    nx, ny, npol, naz = shape
    case = _hot(nx, ny, 1, npol, naz)
    p = oracle_problem(case)
    K = npol * naz
    T = case["T0"].reshape(-1).copy()
    psi = _q1_planck(case, K)
    spec = dlr.problem_from_case(case, precision=prec, element=1, method=dlr.DLR_METHOD_SN,
                                 si_tol=1e-13 if prec == 0 else 0.0)
    with dlr.Solver(spec) as s:
        np.testing.assert_allclose(s.psi(), psi.reshape(K, -1).T, rtol=1e-14 if prec == 0 else 1e-7)
        for _ in range(3):
            psi, T, phi, it, *_ = orc.sn_step_q1(p, psi, T, si_tol=1e-13, si_max_iter=20000)
            assert it > 0
            s.step(1)
            assert rel_l2(s.T(), T) < TOL[prec]
            assert rel_l2(s.psi(), psi.reshape(K, -1).T) < TOL[prec]
            if prec == 0:
                assert abs(s.stats()["si_iters_last"] - it) <= 1


def test_dlr_q1_full_rank_equals_sn_q1(dlr):
    # r = 4 Nx: the basis spans every Q1 field, so the DLR step is the SN step
    case = _hot(2, 2, 16, 2, 8, edges=(0.6, 0.2, 0.3, -1.0))
    d = dlr.problem_from_case(case, precision=0, element=1, si_tol=1e-14)
    s = dlr.problem_from_case(case, precision=0, element=1, method=dlr.DLR_METHOD_SN, si_tol=1e-14)
    with dlr.Solver(d) as a, dlr.Solver(s) as b:
        for _ in range(3):
            a.step(1)
            b.step(1)
            assert rel_l2(a.T(), b.T()) < 1e-10
            assert rel_l2(a.psi(), b.psi()) < 1e-10


def _zero_d_step(Tz, phiz, sig, rho, dt, c, a):
    B0 = a * c * Tz ** 4 / (4 * np.pi)
    dB = a * c * Tz ** 3 / np.pi
    D = rho + 4 * np.pi * dt * sig * dB
    ss = sig * 4 * np.pi * dt * sig * dB / D
    q = sig * B0 * rho / D
    phiz = (4 * np.pi * q + phiz / (c * dt)) / (sig - ss + 1 / (c * dt))
    Tz = Tz + dt * sig * (phiz - 4 * np.pi * B0) / D
    return Tz, phiz


@pytest.mark.parametrize("method", ["dlr", "sn"])
def test_q1_uniform_medium_recurrence(dlr, method):
    nx, ny, sig, rho, T0, dt = 20, 17, 10.0, 0.5, 0.5, 0.02
    case = workloads.small_case(nx, ny, 3, 2, 8, T0=T0)
    case["sigma"] = np.full((ny, nx), sig)
    case["rho_cv"] = np.full((ny, nx), rho)
    case["dt"] = dt
    a, c = case["a_rad"], case["c"]
    Tz, phiz = T0, a * c * T0 ** 4
    kw = dict(method=dlr.DLR_METHOD_SN) if method == "sn" else {}
    spec = dlr.problem_from_case(case, precision=0, element=1, si_tol=1e-14, **kw)
    with dlr.Solver(spec) as s:
        for _ in range(8):
            Tz, phiz = _zero_d_step(Tz, phiz, sig, rho, dt, c, a)
            for e in range(4):
                s.set_edge_inflow(e, phiz / (4 * np.pi))
            s.step(1)
            np.testing.assert_allclose(s.T(), Tz, rtol=1e-12)


@pytest.mark.parametrize("prec", [0, 1])
def test_q1_batch_equals_alone(dlr, prec):
    import torch
    cases = [_hot(33, 20, 6, 2, 8), _hot(19, 23, 4, 4, 8)]
    alone = []
    for c in cases:
        with dlr.Solver(dlr.problem_from_case(c, precision=prec, element=1)) as s:
            s.step(2)
            alone.append((s.T(), s.psi()))
    st = torch.cuda.Stream()
    ss = [dlr.Solver(dlr.problem_from_case(c, precision=prec, element=1), stream=st) for c in cases]
    try:
        dlr.step_batch(ss, 2)
        got = [(s.T(), s.psi()) for s in ss]
    finally:
        for s in ss:
            s.close()
    for (Ta, pa), (Tg, pg) in zip(alone, got):
        assert np.array_equal(Ta, Tg)
        assert rel_l2(pg, pa) < (1e-12 if prec == 0 else 1e-6)


def test_q1_refusals(dlr):
    case = workloads.small_case(8, 8, 2, 2, 6)
    for kw in (dict(precision=0, dsa=1), dict(precision=0, augment=1),
               dict(precision=0, reflect=(1, 0, 0, 0)), dict(precision=0, selection=1),
               dict(precision=0, element=2)):
        kw.setdefault("element", 1)
        with pytest.raises(dlr.DlrError):
            dlr.Solver(dlr.problem_from_case(case, **kw))
    with pytest.raises(dlr.DlrError):  # DG0 and Q1 handles in one batch
        a = dlr.Solver(dlr.problem_from_case(case, precision=0, element=1))
        b = dlr.Solver(dlr.problem_from_case(case, precision=0), stream=a.stream)
        try:
            dlr.step_batch([a, b], 1)
        finally:
            a.close()
            b.close()
