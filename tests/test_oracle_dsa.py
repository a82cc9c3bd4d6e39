"""Pins of the oracle's diffusion synthetic acceleration (Section 4.5, reading
R17): the DG0 diffusion operator against closed forms and brute force, the
CG solve against a dense library solve, and the accelerated source iteration
against the unaccelerated one (same fixed point, far fewer iterations in the
thick diffusive regime the method is for)."""
import numpy as np
import pytest

from conftest import oracle_problem
import workloads


def _problem(orc, nx, ny, sigma, n_polar=4, n_azim=8, lx=1.0, ly=1.0):
    return orc.Problem(nx, ny, n_polar, n_azim, np.asarray(sigma, float).reshape(-1),
                       np.ones(nx * ny), lx=lx, ly=ly)


def _dense(orc, p, st, sa):
    N = p.Nx
    A = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, j] = orc.dsa_apply(p, st, sa, e)
    return A


def test_kappa_tends_to_one_quarter(orc):
    # (1/8 pi) int |Om . n| dOm = (1/8 pi) 2 pi = 1/4 for the exact integral
    for axis in (0, 1):
        errs = [abs(orc.dsa_kappa(n, 2 * n, axis) - 0.25) for n in (4, 8, 16, 32)]
        assert errs[-1] < 2e-3
        assert all(b < a for a, b in zip(errs, errs[1:]))
    # azimuths in multiples of 4: the quadrature is symmetric under x <-> y
    assert orc.dsa_kappa(8, 16, 0) == pytest.approx(orc.dsa_kappa(8, 16, 1), rel=1e-13)


def test_constant_field_sees_only_absorption_inside(orc):
    # Fbar and F0 act on jumps: a constant has none away from the boundary
    nx, ny = 9, 8
    st = 10.0 ** workloads.Stream(3).uniform(nx * ny)
    sa = 0.3 * st
    p = _problem(orc, nx, ny, np.ones(nx * ny), lx=1.3, ly=0.7)
    h2 = (1.3 / nx) * (0.7 / ny)
    out = orc.dsa_apply(p, st, sa, np.ones(nx * ny)).reshape(ny, nx)
    inner = out[2:-2, 2:-2]
    np.testing.assert_allclose(inner, h2 * sa.reshape(ny, nx)[2:-2, 2:-2], rtol=1e-13)
    # next to the boundary the vacuum trace adds a positive leak term
    assert np.all(out[0, :] > h2 * sa.reshape(ny, nx)[0, :])


def test_quadratic_matches_the_diffusion_operator(orc):
    # u = x^2, constant sigma_t: the (1/3) Fbar^T M_t^-1 Fbar part is the
    # wide-stencil second difference, -(1/3 sigma_t) u'' h^2 = -(2/3) h^2 / sigma_t
    # exactly, and F0 adds kappa hy (2 u_c - u_{c+1} - u_{c-1}) = -2 kappa hy hx^2
    nx, ny, lx, ly = 12, 10, 1.2, 0.8
    hx, hy = lx / nx, ly / ny
    s_t, s_a = 7.0, 2.5
    p = _problem(orc, nx, ny, np.ones(nx * ny), lx=lx, ly=ly)
    x = (np.arange(nx) + 0.5) * hx
    u = np.tile(x ** 2, ny)
    out = orc.dsa_apply(p, np.full(nx * ny, s_t), np.full(nx * ny, s_a), u).reshape(ny, nx)
    kx = orc.dsa_kappa(p.n_polar, p.n_azim, 0)
    expect = hx * hy * s_a * x ** 2 - (2.0 / 3.0) * hx * hy / s_t - 2.0 * kx * hy * hx ** 2
    np.testing.assert_allclose(out[2:-2, 2:-2], np.tile(expect, (ny, 1))[2:-2, 2:-2], rtol=1e-11)


def test_operator_is_symmetric_positive_definite(orc):
    nx, ny = 7, 5
    st = 10.0 ** (3.0 * workloads.Stream(11).uniform(nx * ny))
    sa = st * workloads.Stream(12).uniform(nx * ny)
    p = _problem(orc, nx, ny, np.ones(nx * ny), lx=0.9, ly=1.4)
    A = _dense(orc, p, st, sa)
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(A).min() > 0
    # the stencil reaches two cells along x or y and nothing else
    for c in range(nx * ny):
        for j in np.nonzero(A[c])[0]:
            dx, dy = abs(c % nx - j % nx), abs(c // nx - j // nx)
            assert (dy == 0 and dx <= 2) or (dx == 0 and dy <= 2)
    # the probed diagonal is the matrix's
    np.testing.assert_allclose(orc.dsa_diag(p, st, sa), np.diag(A), rtol=1e-14)


def test_cg_solves_the_system(orc):
    nx, ny = 11, 9
    st = 10.0 ** (2.0 * workloads.Stream(21).uniform(nx * ny))
    sa = st * (0.01 + 0.5 * workloads.Stream(22).uniform(nx * ny))
    b = workloads.Stream(23).normal(nx * ny)
    p = _problem(orc, nx, ny, np.ones(nx * ny))
    x, it = orc.dsa_solve(p, st, sa, b, tol=1e-13, max_iter=10000)
    xd = np.linalg.solve(_dense(orc, p, st, sa), b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert 1 <= it <= nx * ny
    # a zero right-hand side takes no iteration
    x0, it0 = orc.dsa_solve(p, st, sa, np.zeros(nx * ny))
    assert it0 == 0 and not np.any(x0)


def _thick_case(side, sig, T0=1.0, r=6):
    c = workloads.small_case(side, side, r, 4, 8)
    c["sigma"] = np.full((side, side), sig)
    c["T0"] = np.full((side, side), T0)
    return c


def _dlr(orc, case, dsa, steps=2, tol=1e-12, dsa_tol=0.1):
    p = oracle_problem(case)
    p.dsa, p.dsa_tol, p.dsa_max_iter = dsa, dsa_tol, 1000
    T = case["T0"].reshape(-1).copy()
    X, S, W = orc.initial_factors(p, T, case["r"])
    its, dits = [], []
    for _ in range(steps):
        X, S, W, T, res = orc.dlr_step(p, X, S, W, T, si_tol=tol, si_max_iter=20000)
        assert res.rc == 0
        its.append(res.iters)
        dits.append(res.diag["dsa_iters"])
    return T, X @ S @ W.T, its, dits


def test_dlr_fixed_point_unchanged_and_iterations_cut(orc):
    case = _thick_case(24, 1e3)
    T0, psi0, it0, _ = _dlr(orc, case, 0)
    T1, psi1, it1, d1 = _dlr(orc, case, 1)
    assert np.linalg.norm(T1 - T0) <= 1e-9 * np.linalg.norm(T0)
    assert np.linalg.norm(psi1 - psi0) <= 1e-9 * np.linalg.norm(psi0)
    assert min(it0) > 100 and max(it1) <= 12, (it0, it1)
    assert all(d > 0 for d in d1)


def test_dlr_dsa_on_a_thin_problem_changes_nothing(orc):
    # sigma_s ~ 0: the right-hand side vanishes, no CG iteration runs
    case = _thick_case(16, 1e-3, T0=0.01)
    T0, psi0, it0, _ = _dlr(orc, case, 0, steps=1)
    T1, psi1, it1, d1 = _dlr(orc, case, 1, steps=1)
    assert np.linalg.norm(T1 - T0) <= 1e-12 * np.linalg.norm(T0)
    assert it1[0] <= it0[0]


def test_sn_iterations_bounded_as_the_mean_free_path_shrinks(orc):
    # Section 4.5: DSA keeps the iteration count bounded in the diffusion
    # limit, where plain source iteration needs ever more sweeps
    plain, acc = [], []
    for sig in (1e2, 1e3, 1e4):
        case = _thick_case(16, sig)
        res = []
        for dsa in (0, 1):
            p = oracle_problem(case)
            p.dsa, p.dsa_tol, p.dsa_max_iter = dsa, 0.1, 1000
            T = case["T0"].reshape(-1).copy()
            psi = np.tile(np.array([orc.planck(p.a_rad, p.c, t) for t in T])[:, None], (1, p.NOm))
            psi, T1, phi, it, *_ = orc.sn_step(p, psi, T, si_tol=1e-11, si_max_iter=50000)
            assert it > 0
            res.append((T1, it))
        assert np.linalg.norm(res[1][0] - res[0][0]) <= 1e-8 * np.linalg.norm(res[0][0])
        plain.append(res[0][1])
        acc.append(res[1][1])
    assert plain[0] < plain[1] < plain[2], plain
    assert max(acc) <= 10, acc
