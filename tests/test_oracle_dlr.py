"""Pins of the oracle's SN-like DLR step (Algorithm 1):
  * full rank r = Nx reproduces the full SN step (Galerkin on all of R^Nx);
  * the error against SN falls as the rank grows;
  * the collocation source iteration equals a dense solve of its system;
  * the L-step (C-bar device) equals a dense solve of the coupled system;
  * an infinite homogeneous medium follows the 0-D backward-Euler recurrence
    and relaxes to the quartic equilibrium (reading R9);
  * equilibrium is preserved (pins reading R1); T stays positive;
  * the pivoted-QR angle choice depends only on span W."""
import numpy as np
import pytest

import workloads
from conftest import oracle_problem
from dense_ref import transport_block


def _full_state(X, S, W):
    return X @ S @ W.T


@pytest.mark.parametrize("n,npol,naz", [(2, 2, 4), (3, 2, 8), (4, 4, 8)])
def test_full_rank_dlr_equals_sn(orc, n, npol, naz):
    c = workloads.small_case(n, n, n * n, npol, naz, seed=n, T0=0.5)
    p = oracle_problem(c)
    r = n * n
    T = c["T0"].reshape(-1).copy()
    X, S, W = orc.initial_factors(p, T, r)
    psi = _full_state(X, S, W)
    Tsn = T.copy()
    for step in range(3):
        X, S, W, T, res = orc.dlr_step(p, X, S, W, T)
        assert res.rc == 0
        psi, Tsn, phi, it, out, inn = orc.sn_step(p, psi, Tsn, si_tol=1e-15)
        np.testing.assert_allclose(T, Tsn, rtol=1e-11)
        np.testing.assert_allclose(_full_state(X, S, W), psi, rtol=0,
                                   atol=1e-11 * np.abs(psi).max())
        # the full-rank step conserves energy like SN
        assert abs(res.diag["residual"]) < 1e-10 * res.diag["E_after"]


def test_error_falls_with_rank(orc):
    c = workloads.small_case(8, 8, 1, 4, 8, seed=9, T0=0.3)
    p = oracle_problem(c)
    T0 = c["T0"].reshape(-1)
    X, S, W = orc.initial_factors(p, T0, 1)
    psi = _full_state(X, S, W)
    Tsn = T0.copy()
    for _ in range(2):
        psi, Tsn, *_ = orc.sn_step(p, psi, Tsn, si_tol=1e-15)
    errs = {}
    for r in (2, 4, 8, 16, 32):
        X, S, W = orc.initial_factors(p, T0, r)
        T = T0.copy()
        for _ in range(2):
            X, S, W, T, res = orc.dlr_step(p, X, S, W, T)
            assert res.rc == 0
        errs[r] = np.linalg.norm(_full_state(X, S, W) - psi) / np.linalg.norm(psi)
    assert errs[32] < 1e-11
    assert errs[16] < errs[4] < errs[2]


def test_collocation_equals_dense_solve(orc):
    c = workloads.small_case(5, 4, 3, 2, 8, seed=4, T0=0.6)
    p = oracle_problem(c)
    r = 3
    T0 = c["T0"].reshape(-1)
    X0, S0, W0 = orc.initial_factors(p, T0, r)
    # a non-trivial old state: perturb S0
    S0 = S0 + np.array([[0, 0.01, 0], [0.02, 0.005, 0], [0, 0.003, 0.004]])
    idx = orc.qdeim(W0)
    Psi, it, rc = orc.collocation(p, X0, S0, W0, T0, idx, si_tol=1e-15)
    assert rc == 0
    # dense: for every chosen angle j, T_j psi_j - sigma_s/(4pi) beta^T What^-1 Psi
    #        = q + psi0_j/(c dt) + inflow
    ox, oy, oz, w = orc.quadrature(c["n_polar"], c["n_azim"])
    coef = orc.coefficients(p, T0)
    N = p.Nx
    What = W0[idx, :]
    gamma = np.linalg.solve(What.T, w @ W0)  # beta^T What^{-1} = gamma^T
    Psi0 = X0 @ S0 @ What.T
    A = np.zeros((N * r, N * r))
    b = np.zeros(N * r)
    for j in range(r):
        Tj, g = transport_block(p.nx, p.ny, p.lx / p.nx, p.ly / p.ny, ox[idx[j]], oy[idx[j]],
                                coef["sigma_t"], p.psi_edge)
        A[j * N:(j + 1) * N, j * N:(j + 1) * N] += Tj
        for l in range(r):
            A[j * N:(j + 1) * N, l * N:(l + 1) * N] -= np.diag(coef["sigma_s"] / (4 * np.pi) * gamma[l])
        b[j * N:(j + 1) * N] = coef["q"] + Psi0[:, j] / (p.c * p.dt) + g
    ref = np.linalg.solve(A, b).reshape(r, N).T
    np.testing.assert_allclose(Psi, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_lstep_equals_dense_coupled_solve(orc):
    nx, ny, npol, naz, r = 6, 5, 2, 8, 4
    rng = np.random.default_rng(7)
    sig = rng.uniform(1, 20, nx * ny)
    p = orc.Problem(nx, ny, npol, naz, sig, np.ones(nx * ny), lx=1.2, ly=0.9,
                    psi_edge=(0.4, 0.1, 0.2, 0.05))
    hx, hy = p.lx / nx, p.ly / ny
    h2 = hx * hy
    X, _ = np.linalg.qr(rng.standard_normal((nx * ny, r)))
    X = X / np.sqrt(h2)
    sigma_t = sig + 1 / (p.c * p.dt)
    sigma_s = rng.uniform(0, 0.9, nx * ny) * sig
    q = rng.uniform(0, 1, nx * ny)
    Lt0 = rng.uniform(0, 1, (r, p.NOm))
    L = orc.lstep(p, X, sigma_t, sigma_s, q, Lt0)
    # dense: Galerkin projection of each direction's DG0 transport operator
    ox, oy, oz, w = orc.quadrature(npol, naz)
    K = p.NOm
    A = np.zeros((r * K, r * K))
    b = np.zeros(r * K)
    Ms = h2 * X.T @ (sigma_s[:, None] * X)
    for k in range(K):
        Tk, g = transport_block(nx, ny, hx, hy, ox[k], oy[k], sigma_t, p.psi_edge)
        A[k * r:(k + 1) * r, k * r:(k + 1) * r] += h2 * X.T @ Tk @ X
        for kp in range(K):
            A[k * r:(k + 1) * r, kp * r:(kp + 1) * r] -= Ms * w[kp] / (4 * np.pi)
        b[k * r:(k + 1) * r] = h2 * X.T @ (q + g) + Lt0[:, k] / (p.c * p.dt)
    ref = np.linalg.solve(A, b).reshape(K, r).T
    np.testing.assert_allclose(L, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def _zero_d_step(T, phi, sig, rho, dt, c, a):
    B0 = a * c * T ** 4 / (4 * np.pi)
    dB = a * c * T ** 3 / np.pi
    D = rho + 4 * np.pi * dt * sig * dB
    ss = sig * 4 * np.pi * dt * sig * dB / D
    q = sig * B0 * rho / D
    phin = (4 * np.pi * q + phi / (c * dt)) / (sig - ss + 1 / (c * dt))
    Tn = T + dt * sig * (phin - 4 * np.pi * B0) / D
    return Tn, phin


@pytest.mark.parametrize("r", [1, 3])
def test_infinite_medium_recurrence_and_equilibrium(orc, r):
    nx, ny, sig, rho, T0, dt = 6, 5, 10.0, 0.5, 0.5, 0.02
    p = orc.Problem(nx, ny, 4, 8, np.full(nx * ny, sig), np.full(nx * ny, rho), dt=dt)
    X, S, W = orc.initial_factors(p, np.full(nx * ny, T0), r)
    T = np.full(nx * ny, T0)
    Tz, phiz = T0, 4 * np.pi * orc.planck(p.a_rad, p.c, T0)
    E0 = rho * T0 + phiz / p.c
    for step in range(60):
        Tz, phiz = _zero_d_step(Tz, phiz, sig, rho, dt, p.c, p.a_rad)
        p.psi_edge = (phiz / (4 * np.pi),) * 4  # inflow = the exact new state
        X, S, W, T, res = orc.dlr_step(p, X, S, W, T)
        assert res.rc == 0
        np.testing.assert_allclose(T, Tz, rtol=1e-12)
        np.testing.assert_allclose(res.phi, phiz, rtol=1e-12)
    # relaxes to rho T + a T^4 = E0 (Newton)
    Ts = T0
    for _ in range(50):
        Ts -= (rho * Ts + p.a_rad * Ts ** 4 - E0) / (rho + 4 * p.a_rad * Ts ** 3)
    assert abs(T.mean() - Ts) < 1e-6 * Ts
    # the 0-D recurrence itself conserves E exactly
    assert abs(rho * Tz + phiz / p.c - E0) < 1e-13 * E0


@pytest.mark.parametrize("n_s,n_c", [(3.0, 0.0), (2.0, 1.0)])
def test_infinite_medium_with_temperature_dependent_materials(orc, n_s, n_c):
    """Reading R16: sigma(T) = sigma (T/T_ref)^-n_s and rho c_v(T) = rho_cv
    (T/T_ref)^n_c taken at the step's T0 everywhere (coefficients, sweep
    opacity, temperature update): the uniform medium follows the 0-D
    backward-Euler recurrence with the materials of each step's T0."""
    nx, ny, sig0, rho0, T0, dt, Tr = 5, 4, 10.0, 0.5, 0.5, 0.02, 0.8
    p = orc.Problem(nx, ny, 4, 8, np.full(nx * ny, sig0), np.full(nx * ny, rho0), dt=dt,
                    sigma_texp=n_s, cv_texp=n_c, T_ref=Tr)
    X, S, W = orc.initial_factors(p, np.full(nx * ny, T0), 2)
    T = np.full(nx * ny, T0)
    Tz, phiz = T0, 4 * np.pi * orc.planck(p.a_rad, p.c, T0)
    for step in range(40):
        sig, rho = sig0 * (Tz / Tr) ** -n_s, rho0 * (Tz / Tr) ** n_c
        Tz, phiz = _zero_d_step(Tz, phiz, sig, rho, dt, p.c, p.a_rad)
        p.psi_edge = (phiz / (4 * np.pi),) * 4
        X, S, W, T, res = orc.dlr_step(p, X, S, W, T)
        assert res.rc == 0
        np.testing.assert_allclose(T, Tz, rtol=1e-12)
        np.testing.assert_allclose(res.phi, phiz, rtol=1e-12)
    # the same law with zero exponents is the constant-material step
    q = orc.Problem(nx, ny, 4, 8, np.full(nx * ny, sig0), np.full(nx * ny, rho0), dt=dt,
                    sigma_texp=0.0, cv_texp=0.0, T_ref=Tr)
    r = orc.Problem(nx, ny, 4, 8, np.full(nx * ny, sig0), np.full(nx * ny, rho0), dt=dt)
    q.psi_edge = r.psi_edge = p.psi_edge
    a = orc.dlr_step(q, X, S, W, T)
    b = orc.dlr_step(r, X, S, W, T)
    assert np.array_equal(a[3], b[3])


def test_equilibrium_preserved(orc):
    c = workloads.small_case(8, 6, 4, 4, 8, seed=2, T0=0.7)
    p = oracle_problem(c, psi_edge=[0] * 4)
    p.set_edge_temperatures([0.7] * 4)
    T = c["T0"].reshape(-1).copy()
    X, S, W = orc.initial_factors(p, T, 4)
    B = orc.planck(p.a_rad, p.c, 0.7)
    for _ in range(3):
        X, S, W, T, res = orc.dlr_step(p, X, S, W, T)
        assert res.rc == 0
    np.testing.assert_allclose(T, 0.7, rtol=1e-13)
    np.testing.assert_allclose(_full_state(X, S, W), B, rtol=1e-12)


def test_lattice32_positivity_and_convergence(orc):
    c = workloads.lattice32()
    p = oracle_problem(c)
    T = c["T0"].reshape(-1).copy()
    X, S, W = orc.initial_factors(p, T, c["r"])
    for _ in range(c["steps"]):
        X, S, W, T, res = orc.dlr_step(p, X, S, W, T)
        assert res.rc == 0 and 0 < res.iters < 100
        assert T.min() > 0
        assert abs(res.diag["residual"]) < 1e-2 * res.diag["E_after"]
    assert T.max() > 0.2  # the left inflow heats the slab


def test_selection_depends_only_on_span(orc):
    c = workloads.small_case(10, 9, 5, 4, 8, seed=6, T0=0.3)
    p = oracle_problem(c)
    T = c["T0"].reshape(-1)
    X, S, W = orc.initial_factors(p, T, 5)
    X, S, W, T1, _ = orc.dlr_step(p, X, S, W, T)
    V, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((5, 5)))
    _, _, _, Ta, ra = orc.dlr_step(p, X, S, W, T1)
    _, _, _, Tb, rb = orc.dlr_step(p, X, S @ V, W @ V, T1)
    assert sorted(ra.idx) == sorted(rb.idx)
    np.testing.assert_allclose(Ta, Tb, rtol=1e-12)


def test_forced_indices_and_deim(orc):
    c = workloads.small_case(9, 7, 4, 4, 8, seed=8, T0=0.3)
    p = oracle_problem(c)
    T = c["T0"].reshape(-1)
    X, S, W = orc.initial_factors(p, T, 4)
    _, _, _, Ta, ra = orc.dlr_step(p, X, S, W, T)
    _, _, _, Tb, rb = orc.dlr_step(p, X, S, W, T, forced_idx=ra.idx)
    assert np.array_equal(Ta, Tb)
    _, _, _, Td, rd = orc.dlr_step(p, X, S, W, T, selection=1)
    assert rd.rc == 0 and Td.min() > 0


def test_fixed_iterations_and_cap(orc):
    c = workloads.small_case(9, 7, 4, 4, 8, seed=8, T0=0.9)
    p = oracle_problem(c)
    T = c["T0"].reshape(-1)
    X, S, W = orc.initial_factors(p, T, 4)
    *_, res = orc.dlr_step(p, X, S, W, T, si_fixed_iters=2)
    assert res.rc == 0 and res.iters == 2
    *_, res = orc.dlr_step(p, X, S, W, T, si_tol=1e-30, si_max_iter=3)
    assert res.rc == -2


def _weighted_truncation(psi, h2, w, r):
    """Best rank-r approximation of psi in the norm sum_c sum_k h2 w_k psi^2
    (numpy SVD of the weighted matrix) and the weighted singular values."""
    sw = np.sqrt(w)[None, :]
    U, s, Vt = np.linalg.svd(np.sqrt(h2) * psi * sw, full_matrices=False)
    return (U[:, :r] * s[:r]) @ Vt[:r] / np.sqrt(h2) / sw, s


@pytest.mark.parametrize("nx,ny,r,npol,naz", [(2, 3, 3, 2, 8), (4, 2, 4, 2, 8), (3, 4, 6, 4, 4)])
def test_augmented_step_on_the_full_space_is_the_truncated_sn_step(orc, nx, ny, r, npol, naz):
    """Augmented step (reading R15) with 2r = Nx: orth([Psi, X0]) spans all of
    R^Nx, so its L-step is the full SN step (a Galerkin projection on the
    whole space), and the truncation of the 2r x 2r S keeps the best rank-r
    part of that SN solution in the (h^2, w) norm."""
    c = workloads.small_case(nx, ny, r, npol, naz, seed=nx + 5 * ny, T0=0.5)
    p = oracle_problem(c)
    h2 = (1.0 / nx) * (1.0 / ny)
    _, _, _, w = orc.quadrature(npol, naz)
    T = c["T0"].reshape(-1).copy()
    X, S, W = orc.initial_factors(p, T, r)
    for _ in range(3):
        psi_sn, *_ = orc.sn_step(p, X @ S @ W.T, T, si_tol=1e-15)
        X, S, W, T, res = orc.dlr_step(p, X, S, W, T, augment=1)
        assert res.rc == 0
        target, sv = _weighted_truncation(psi_sn, h2, w, r)
        assert sv[r - 1] - sv[r] > 1e-6 * sv[0]  # a gap: the truncation is unique
        np.testing.assert_allclose(X @ S @ W.T, target, rtol=0, atol=1e-10 * np.abs(target).max())
        np.testing.assert_allclose(h2 * X.T @ X, np.eye(r), atol=1e-12)
        np.testing.assert_allclose(W.T @ (w[:, None] * W), np.eye(r), atol=1e-12)
        # canonical: S is diagonal with the leading singular values
        np.testing.assert_allclose(S, np.diag(sv[:r]), rtol=0, atol=1e-10 * sv[0])


def test_augmented_step_rejects_2r_above_nx(orc):
    c = workloads.small_case(2, 2, 3, 2, 4, seed=1, T0=0.5)
    p = oracle_problem(c)
    T = c["T0"].reshape(-1).copy()
    X, S, W = orc.initial_factors(p, T, 3)
    *_, res = orc.dlr_step(p, X, S, W, T, augment=1)
    assert res.rc == -1


def test_threads_do_not_change_results(orc):
    """The oracle's parallel loops (angles, cells, reflector columns, L-step
    angles) keep every sum in its serial order: one thread and several give
    bitwise the same step.  The mesh is above the size where the loops go
    parallel."""
    c = workloads.small_case(96, 90, 8, 4, 8, seed=21, T0=0.5)
    p = oracle_problem(c)
    out = []
    try:
        for th in (1, 4):
            orc.set_threads(th)
            T = c["T0"].reshape(-1).copy()
            X, S, W = orc.initial_factors(p, T, 8)
            for _ in range(2):
                X, S, W, T, res = orc.dlr_step(p, X, S, W, T)
                assert res.rc == 0
            out.append((X, S, W, T))
    finally:
        orc.set_threads(0)
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_diverged_iteration_is_not_convergence(orc):
    # Algorithm 1 step 4 with the stopping test of reading R7: a scalar flux
    # that is no longer finite (a diverged collocation iteration) must end the
    # step as not converged, never pass the test (NaN compares false)
    c = workloads.small_case(9, 7, 3, 2, 8, seed=3, T0=0.5)
    p = oracle_problem(c)
    T = c["T0"].reshape(-1).copy()
    X, S, W = orc.initial_factors(p, T, 3)
    T[4] = np.nan
    *_, res = orc.dlr_step(p, X, S, W, T, si_tol=1e-13)
    assert res.rc != 0


def test_angle_choice_of_non_finite_factors_fails(orc):
    # Algorithm 1 step 2: with no finite column norm there is no pivot
    W = np.full((16, 3), np.nan)
    for fn in (orc.qdeim, orc.deim):
        with pytest.raises(Exception):
            fn(W)


def _negative_T_case(orc):
    # a uniform thick medium at T0 < 0 (the state Algorithm 1 reaches after a
    # loss of positivity): -rho c_v < 4 pi dt sigma B'(T0) < 0 makes the
    # effective scattering sigma_s = sigma 4 pi dt sigma B' / D negative,
    # sigma_s / sigma_t = -1.44, so the plain source iteration diverges
    nx = ny = 6
    c = workloads.small_case(nx, ny, 4, 2, 8, seed=1, T0=0.5)
    c["sigma"] = np.full((ny, nx), 100.0)
    p = oracle_problem(c)
    T0 = np.full(nx * ny, -0.714)
    X0, S0, W0 = orc.initial_factors(p, -T0, 4)
    return c, p, T0, X0, S0, W0


def test_relaxed_iteration_converges_to_the_dense_solution(orc):
    # reading R22: the collocation iteration is relaxed when it grows; its
    # plain form diverges here (an eigenvalue of the iteration map below -1),
    # the relaxed one reaches the solution of the collocation system
    c, p, T0, X0, S0, W0 = _negative_T_case(orc)
    r = 4
    idx = orc.qdeim(W0)
    ox, oy, oz, w = orc.quadrature(c["n_polar"], c["n_azim"])
    coef = orc.coefficients(p, T0)
    assert (coef["sigma_s"] / coef["sigma_t"]).max() < -1.4
    N = p.Nx
    What = W0[idx, :]
    gamma = np.linalg.solve(What.T, w @ W0)
    Psi0 = X0 @ S0 @ What.T
    M = np.zeros((N, N))
    A = np.zeros((N * r, N * r))
    b = np.zeros(N * r)
    for j in range(r):
        Tj, g = transport_block(p.nx, p.ny, p.lx / p.nx, p.ly / p.ny, ox[idx[j]], oy[idx[j]],
                                coef["sigma_t"], p.psi_edge)
        M += gamma[j] * np.linalg.solve(Tj, np.diag(coef["sigma_s"] / (4 * np.pi)))
        A[j * N:(j + 1) * N, j * N:(j + 1) * N] += Tj
        for l in range(r):
            A[j * N:(j + 1) * N, l * N:(l + 1) * N] -= np.diag(coef["sigma_s"] / (4 * np.pi) * gamma[l])
        b[j * N:(j + 1) * N] = coef["q"] + Psi0[:, j] / (p.c * p.dt) + g
    assert np.linalg.eigvals(M).real.min() < -1.3
    ref = np.linalg.solve(A, b).reshape(r, N).T
    Psi, it, rc = orc.collocation(p, X0, S0, W0, T0, idx, si_tol=1e-15, si_max_iter=2000)
    assert rc == 0 and it < 200
    np.testing.assert_allclose(Psi, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_relaxation_leaves_a_contracting_iteration_alone(orc):
    # the same problem at T0 > 0 contracts: the relaxation never engages, so
    # k iterations of the oracle equal k plain source iterations written out
    # here (sweeps of every chosen angle, phi = Psi gamma)
    c, p, T0, X0, S0, W0 = _negative_T_case(orc)
    T0 = -T0
    idx = orc.qdeim(W0)
    ox, oy, oz, w = orc.quadrature(c["n_polar"], c["n_azim"])
    coef = orc.coefficients(p, T0)
    What = W0[idx, :]
    gamma = np.linalg.solve(What.T, w @ W0)
    Psi0 = X0 @ S0 @ What.T
    phi = Psi0 @ gamma
    for k in range(12):
        Psi = np.column_stack([
            orc.sweep(p, ox[idx[j]], oy[idx[j]], coef["sigma_t"],
                      coef["sigma_s"] * phi / (4 * np.pi) + coef["q"] + Psi0[:, j] / (p.c * p.dt))
            for j in range(len(idx))])
        phi = Psi @ gamma
    got, it, rc = orc.collocation(p, X0, S0, W0, T0, idx, si_fixed_iters=12)
    assert rc == 0
    np.testing.assert_allclose(got, Psi, rtol=1e-12, atol=1e-13 * np.abs(Psi).max())
