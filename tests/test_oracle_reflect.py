"""Pins of reflective edges in the oracle (readings R18 for the SN step, R19
for the DLR step): the mirror maps of the quadrature, the lagged source
iteration against a dense solve with the reflection coupled in, a
mirror-doubled domain, the 0-D recurrence of an all-reflective uniform
medium, energy conservation, and the full-rank DLR step equal to the SN
step with reflective edges."""
import numpy as np
import pytest

import workloads
from conftest import oracle_problem
from dense_ref import sn_dense_reflect
from test_oracle_dlr import _zero_d_step


def _mirrors(orc, npol, naz):
    K = npol * naz
    return (np.array([orc.reflect_index(npol, naz, k, 0) for k in range(K)]),
            np.array([orc.reflect_index(npol, naz, k, 1) for k in range(K)]))


@pytest.mark.parametrize("npol,naz", [(2, 8), (4, 12), (3, 6)])
def test_mirror_maps(orc, npol, naz):
    ox, oy, oz, w = orc.quadrature(npol, naz)
    mx, my = _mirrors(orc, npol, naz)
    np.testing.assert_allclose(ox[mx], -ox, atol=1e-15)
    np.testing.assert_allclose(oy[mx], oy, atol=1e-15)
    np.testing.assert_allclose(ox[my], ox, atol=1e-15)
    np.testing.assert_allclose(oy[my], -oy, atol=1e-15)
    np.testing.assert_array_equal(w[mx], w)
    np.testing.assert_array_equal(mx[mx], np.arange(npol * naz))
    np.testing.assert_array_equal(my[my], np.arange(npol * naz))


@pytest.mark.parametrize("reflect", [(1, 0, 0, 0), (0, 1, 1, 0), (1, 1, 1, 1)])
def test_lagged_iteration_equals_dense_solve(orc, reflect):
    c = workloads.small_case(4, 3, 1, 2, 8, seed=5, T0=0.5)
    p = oracle_problem(c)
    p.psi_edge = (0.2, 0.1, 0.05, 0.0)
    p.reflect = reflect
    ox, oy, oz, w = orc.quadrature(2, 8)
    mx, my = _mirrors(orc, 2, 8)
    T0 = c["T0"].reshape(-1)
    psi0 = np.random.default_rng(1).uniform(0.0, 0.5, (p.Nx, p.NOm))
    psi, T, phi, it, out, inn = orc.sn_step(p, psi0, T0, si_tol=1e-15, si_max_iter=20000)
    assert it > 0
    ref = sn_dense_reflect(p, orc.coefficients(p, T0), psi0, ox, oy, w, reflect, mx, my)
    np.testing.assert_allclose(psi, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("axis", [0, 1])
def test_reflective_edge_equals_mirror_doubled_domain(orc, axis):
    # the half domain with a reflective edge is the half of a domain twice as
    # large with the materials and the state mirrored across that edge
    nx, ny, npol, naz = 5, 4, 2, 8
    st = workloads.Stream(9)
    sig = 10.0 ** (2.0 * st.uniform(nx * ny)).reshape(ny, nx)
    T0 = (0.2 + 0.6 * st.uniform(nx * ny)).reshape(ny, nx)
    if axis == 0:
        sigB = np.concatenate([sig[:, ::-1], sig], axis=1)
        TB = np.concatenate([T0[:, ::-1], T0], axis=1)
        edgesA, reflA = (0.0, 0.3, 0.05, 0.0), (1, 0, 0, 0)
        edgesB = (0.3, 0.3, 0.05, 0.0)
        pB = orc.Problem(2 * nx, ny, npol, naz, sigB, np.ones(2 * nx * ny), lx=2.0)
    else:
        sigB = np.concatenate([sig[::-1, :], sig], axis=0)
        TB = np.concatenate([T0[::-1, :], T0], axis=0)
        edgesA, reflA = (0.1, 0.0, 0.0, 0.25), (0, 0, 1, 0)
        edgesB = (0.1, 0.0, 0.25, 0.25)
        pB = orc.Problem(nx, 2 * ny, npol, naz, sigB, np.ones(2 * nx * ny), ly=2.0)
    pA = orc.Problem(nx, ny, npol, naz, sig, np.ones(nx * ny))
    pA.psi_edge, pA.reflect, pB.psi_edge = edgesA, reflA, edgesB
    a, cc = pA.a_rad, pA.c
    TA, TBf = T0.reshape(-1).copy(), TB.reshape(-1).copy()
    psiA = np.repeat((a * cc * TA ** 4 / (4 * np.pi))[:, None], npol * naz, axis=1)
    psiB = np.repeat((a * cc * TBf ** 4 / (4 * np.pi))[:, None], npol * naz, axis=1)
    for _ in range(2):
        psiA, TA, *_ = orc.sn_step(pA, psiA, TA, si_tol=1e-14, si_max_iter=20000)
        psiB, TBf, *_ = orc.sn_step(pB, psiB, TBf, si_tol=1e-14, si_max_iter=20000)
    if axis == 0:
        half = TBf.reshape(ny, 2 * nx)[:, nx:].reshape(-1)
        halfpsi = psiB.reshape(ny, 2 * nx, -1)[:, nx:, :].reshape(nx * ny, -1)
    else:
        half = TBf.reshape(2 * ny, nx)[ny:, :].reshape(-1)
        halfpsi = psiB.reshape(2 * ny, nx, -1)[ny:, :, :].reshape(nx * ny, -1)
    np.testing.assert_allclose(TA, half, rtol=1e-11)
    np.testing.assert_allclose(psiA, halfpsi, rtol=1e-10, atol=1e-12 * np.abs(halfpsi).max())


def test_all_reflective_uniform_medium_is_the_zero_d_recurrence(orc):
    nx, ny, sig, rho, T0, dt = 4, 3, 10.0, 0.5, 0.5, 0.02
    p = orc.Problem(nx, ny, 2, 8, np.full(nx * ny, sig), np.full(nx * ny, rho), dt=dt)
    p.reflect = (1, 1, 1, 1)
    T = np.full(nx * ny, T0)
    psi = np.full((nx * ny, 16), orc.planck(p.a_rad, p.c, T0))
    Tz, phiz = T0, 4 * np.pi * orc.planck(p.a_rad, p.c, T0)
    for _ in range(20):
        Tz, phiz = _zero_d_step(Tz, phiz, sig, rho, dt, p.c, p.a_rad)
        psi, T, phi, it, out, inn = orc.sn_step(p, psi, T, si_tol=1e-15)
        np.testing.assert_allclose(T, Tz, rtol=1e-12)
        np.testing.assert_allclose(phi, phiz, rtol=1e-12)


def test_all_reflective_conserves_energy(orc):
    c = workloads.small_case(6, 5, 1, 2, 8, seed=4, T0=0.6)
    p = oracle_problem(c)
    p.reflect = (1, 1, 1, 1)
    ox, oy, oz, w = orc.quadrature(2, 8)
    T = c["T0"].reshape(-1).copy()
    T[:7] = 1.0
    psi = np.repeat((p.a_rad * p.c * T ** 4 / (4 * np.pi))[:, None], 16, axis=1)
    for _ in range(3):
        E0 = orc.energy(p, T, psi @ w)
        psi, T, phi, it, out, inn = orc.sn_step(p, psi, T, si_tol=1e-15, si_max_iter=20000)
        E1 = orc.energy(p, T, phi)
        assert abs(out - inn) < 1e-10 * out
        assert abs(E1 - E0) < 1e-11 * E1


@pytest.mark.parametrize("n,reflect", [(2, (1, 0, 0, 0)), (3, (0, 1, 1, 0)), (3, (1, 1, 1, 1))])
def test_full_rank_dlr_with_reflective_edges_equals_sn(orc, n, reflect):
    # reading R19: the L-step's reflected inflow is implicit (a fixed point on
    # the boundary values), so at full rank the DLR step is the SN step
    c = workloads.small_case(n, n, n * n, 2, 8, seed=n + 7, T0=0.5)
    p = oracle_problem(c)
    p.psi_edge = (0.2, 0.1, 0.05, 0.0)
    p.reflect = reflect
    r = n * n
    T = c["T0"].reshape(-1).copy()
    T[0] = 0.9
    X, S, W = orc.initial_factors(p, T, r)
    psi = X @ S @ W.T
    Tsn = T.copy()
    for _ in range(2):
        X, S, W, T, res = orc.dlr_step(p, X, S, W, T, si_tol=1e-14, si_max_iter=20000)
        assert res.rc == 0
        psi, Tsn, phi, it, *_ = orc.sn_step(p, psi, Tsn, si_tol=1e-14, si_max_iter=20000)
        np.testing.assert_allclose(T, Tsn, rtol=1e-10)
        np.testing.assert_allclose(X @ S @ W.T, psi, rtol=0, atol=1e-10 * np.abs(psi).max())


@pytest.mark.parametrize("r", [1, 3])
def test_dlr_all_reflective_uniform_medium_is_the_zero_d_recurrence(orc, r):
    nx, ny, sig, rho, T0, dt = 6, 5, 10.0, 0.5, 0.5, 0.02
    p = orc.Problem(nx, ny, 4, 8, np.full(nx * ny, sig), np.full(nx * ny, rho), dt=dt)
    p.reflect = (1, 1, 1, 1)
    X, S, W = orc.initial_factors(p, np.full(nx * ny, T0), r)
    T = np.full(nx * ny, T0)
    Tz, phiz = T0, 4 * np.pi * orc.planck(p.a_rad, p.c, T0)
    for _ in range(15):
        Tz, phiz = _zero_d_step(Tz, phiz, sig, rho, dt, p.c, p.a_rad)
        X, S, W, T, res = orc.dlr_step(p, X, S, W, T, si_tol=1e-14)
        assert res.rc == 0
        np.testing.assert_allclose(T, Tz, rtol=1e-12)
        np.testing.assert_allclose(res.phi, phiz, rtol=1e-12)


def test_dsa_with_reflective_edges_keeps_the_step(orc):
    # DSA (reading R17: vacuum traces in the diffusion operator) only changes
    # how the iteration gets there, also behind reflective edges
    c = workloads.small_case(8, 6, 1, 2, 8, seed=6, T0=1.0)
    c["sigma"] = c["sigma"] * 10.0
    res = []
    for dsa in (0, 1):
        p = oracle_problem(c)
        p.reflect = (1, 0, 1, 0)
        p.dsa, p.dsa_tol, p.dsa_max_iter = dsa, 0.1, 3
        T = c["T0"].reshape(-1).copy()
        psi = np.repeat((p.a_rad * p.c * T ** 4 / (4 * np.pi))[:, None], 16, axis=1)
        psi, T, phi, it, *_ = orc.sn_step(p, psi, T, si_tol=1e-13, si_max_iter=20000)
        res.append((T, psi, it))
    assert np.linalg.norm(res[1][0] - res[0][0]) <= 1e-10 * np.linalg.norm(res[0][0])
    assert np.linalg.norm(res[1][1] - res[0][1]) <= 1e-10 * np.linalg.norm(res[0][1])
    assert res[1][2] < res[0][2]


def test_collocation_at_every_angle_is_the_sn_iteration(orc):
    # steps 1-4 at r = NOm chosen angles: the interpolation through What is
    # exact, so the lagged reflected inflow of the collocation sweeps is the
    # SN one and the collocation fluxes are the SN angular flux
    c = workloads.small_case(4, 4, 16, 2, 8, seed=17, T0=0.5)
    p = oracle_problem(c)
    p.psi_edge = (0.2, 0.0, 0.05, 0.1)
    p.reflect = (1, 0, 0, 1)
    T = c["T0"].reshape(-1).copy()
    T[3] = 0.9
    X, S, W = orc.initial_factors(p, T, 16)
    idx = np.arange(16)[::-1].copy()
    Psi, it, rc = orc.collocation(p, X, S, W, T, idx, si_tol=1e-14, si_max_iter=20000)
    assert rc == 0 and it > 0
    psi, *_ = orc.sn_step(p, X @ S @ W.T, T, si_tol=1e-14, si_max_iter=20000)
    np.testing.assert_allclose(Psi, psi[:, idx], rtol=0, atol=1e-11 * np.abs(psi).max())
