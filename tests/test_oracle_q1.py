"""Pins of the oracle's bilinear (Q1) upwind DG sweep (Section 4.4 with the
paper's bilinear elements): a globally bilinear solution is reproduced
exactly, a smooth one converges at second order in the cell averages (DG0
at first), and the cell equations with the test function 1 add up to the
global balance."""
import numpy as np
import pytest


def _problem(orc, nx, ny, lx=1.0, ly=1.0):
    return orc.Problem(nx, ny, 2, 4, np.ones(nx * ny), np.ones(nx * ny), lx=lx, ly=ly)


def _centres(p):
    hx, hy = p.lx / p.nx, p.ly / p.ny
    xc = (np.arange(p.nx) + 0.5) * hx
    yc = (np.arange(p.ny) + 0.5) * hy
    return np.meshgrid(xc, yc), hx / 2, hy / 2


def _gauss(n=4):
    return np.polynomial.legendre.leggauss(n)


def _project(p, f):
    """Legendre coefficients (1, xi, eta, xi eta) per cell of f(x, y), by
    4 x 4 Gauss quadrature (exact for the polynomial degrees used)."""
    (X, Y), a, b = _centres(p)
    g, w = _gauss()
    out = np.zeros((p.ny, p.nx, 4))
    norm = np.array([4.0, 4.0 / 3.0, 4.0 / 3.0, 4.0 / 9.0])
    for gi, wi in zip(g, w):
        for gj, wj in zip(g, w):
            val = f(X + a * gi, Y + b * gj)
            basis = (1.0, gi, gj, gi * gj)
            for k in range(4):
                out[:, :, k] += wi * wj * val * basis[k]
    return (out / norm).reshape(-1, 4)


def _inflow(p, f, ox, oy):
    """Traces of f on the upwind boundary faces as (constant, slope)."""
    (X, Y), a, b = _centres(p)
    g, w = _gauss()
    xb = 0.0 if ox > 0 else p.lx
    yb = 0.0 if oy > 0 else p.ly
    in_x = np.zeros((p.ny, 2))
    in_y = np.zeros((p.nx, 2))
    for gi, wi in zip(g, w):
        in_x[:, 0] += wi * f(xb, Y[:, 0] + b * gi) / 2
        in_x[:, 1] += wi * f(xb, Y[:, 0] + b * gi) * gi / (2 / 3)
        in_y[:, 0] += wi * f(X[0, :] + a * gi, yb) / 2
        in_y[:, 1] += wi * f(X[0, :] + a * gi, yb) * gi / (2 / 3)
    return in_x, in_y


@pytest.mark.parametrize("ox,oy", [(0.6, 0.3), (-0.5, 0.7), (0.2, -0.9), (-0.8, -0.4)])
def test_bilinear_solution_is_exact(orc, ox, oy):
    p = _problem(orc, 7, 5, lx=1.3, ly=0.7)
    al, be, ga, de, st = 0.7, -0.4, 1.1, 0.9, 2.5
    u = lambda x, y: al + be * x + ga * y + de * x * y
    q = lambda x, y: ox * (be + de * y) + oy * (ga + de * x) + st * u(x, y)
    in_x, in_y = _inflow(p, u, ox, oy)
    psi = orc.sweep_q1(p, ox, oy, np.full(p.Nx, st), _project(p, q), in_x, in_y)
    np.testing.assert_allclose(psi, _project(p, u), rtol=0, atol=1e-12)


def _smooth_error(orc, n, ox, oy, st):
    p = _problem(orc, n, n)
    u = lambda x, y: 2.0 + np.sin(np.pi * x) * np.cos(0.5 * np.pi * y)
    ux = lambda x, y: np.pi * np.cos(np.pi * x) * np.cos(0.5 * np.pi * y)
    uy = lambda x, y: -0.5 * np.pi * np.sin(np.pi * x) * np.sin(0.5 * np.pi * y)
    q = lambda x, y: ox * ux(x, y) + oy * uy(x, y) + st * u(x, y)
    in_x, in_y = _inflow(p, u, ox, oy)
    psi = orc.sweep_q1(p, ox, oy, np.full(p.Nx, st), _project(p, q), in_x, in_y)
    exact = _project(p, u)
    e_q1 = np.sqrt(np.mean((psi[:, 0] - exact[:, 0]) ** 2))
    # DG0 on the same problem: cell-average source, constant inflow
    orc_p = _problem(orc, n, n)
    orc_p.psi_edge = (0.0,) * 4
    in0x, in0y = in_x[:, 0].copy(), in_y[:, 0].copy()
    psi0 = orc.sweep_in(orc_p, ox, oy, np.full(p.Nx, st), _project(p, q)[:, 0], in0x, in0y)
    e_dg0 = np.sqrt(np.mean((psi0 - exact[:, 0]) ** 2))
    return e_q1, e_dg0


def test_second_order_convergence(orc):
    errs = [_smooth_error(orc, n, 0.6, 0.45, 1.5) for n in (8, 16, 32)]
    q1 = [e[0] for e in errs]
    dg0 = [e[1] for e in errs]
    rates_q1 = np.log2(np.array(q1[:-1]) / np.array(q1[1:]))
    rates_dg0 = np.log2(np.array(dg0[:-1]) / np.array(dg0[1:]))
    assert np.all(rates_q1 > 1.8), rates_q1
    assert np.all(rates_dg0 < 1.3), rates_dg0
    assert q1[-1] < 0.05 * dg0[-1]


def test_global_balance(orc):
    # the cell equations with v = 1 summed over the mesh: the interior faces
    # cancel, leaving outflow - inflow + int sigma_t u = int src
    p = _problem(orc, 6, 9, lx=0.8, ly=1.1)
    rng = np.random.default_rng(3)
    ox, oy = -0.55, 0.35
    st = rng.uniform(0.5, 20.0, p.Nx)
    src = rng.uniform(0.0, 2.0, (p.Nx, 4))
    in_x = rng.uniform(0.0, 1.0, (p.ny, 2))
    in_y = rng.uniform(0.0, 1.0, (p.nx, 2))
    psi = orc.sweep_q1(p, ox, oy, st, src, in_x, in_y)
    hx, hy = p.lx / p.nx, p.ly / p.ny
    area = hx * hy
    U = psi.reshape(p.ny, p.nx, 4)
    # outflow through the downwind faces (face means: the constant part of the trace)
    ix_out = 0 if ox < 0 else p.nx - 1
    iy_out = 0 if oy < 0 else p.ny - 1
    sgn_x = 1.0 if ox > 0 else -1.0
    sgn_y = 1.0 if oy > 0 else -1.0
    out = abs(ox) * hy * np.sum(U[:, ix_out, 0] + sgn_x * U[:, ix_out, 1])
    out += abs(oy) * hx * np.sum(U[iy_out, :, 0] + sgn_y * U[iy_out, :, 2])
    inn = abs(ox) * hy * np.sum(in_x[:, 0]) + abs(oy) * hx * np.sum(in_y[:, 0])
    lhs = out - inn + area * np.sum(st * psi[:, 0])
    rhs = area * np.sum(src[:, 0])
    assert abs(lhs - rhs) < 1e-12 * rhs


# ---- the full-rank SN step on Q1 elements ----

from test_oracle_dlr import _zero_d_step  # noqa: E402
import workloads  # noqa: E402
from conftest import oracle_problem  # noqa: E402


def _q1_planck(p, T):
    B = p.a_rad * p.c * np.asarray(T) ** 4 / (4 * np.pi)
    psi = np.zeros((p.NOm, p.Nx, 4))
    psi[:, :, 0] = B[None, :]
    return psi


def test_sn_q1_infinite_medium_recurrence(orc):
    nx, ny, sig, rho, T0, dt = 5, 4, 10.0, 0.5, 0.5, 0.02
    p = orc.Problem(nx, ny, 2, 8, np.full(nx * ny, sig), np.full(nx * ny, rho), dt=dt)
    T = np.full(nx * ny, T0)
    psi = _q1_planck(p, T)
    Tz, phiz = T0, 4 * np.pi * orc.planck(p.a_rad, p.c, T0)
    for _ in range(10):
        Tz, phiz = _zero_d_step(Tz, phiz, sig, rho, dt, p.c, p.a_rad)
        p.psi_edge = (phiz / (4 * np.pi),) * 4
        psi, T, phi, it, *_ = orc.sn_step_q1(p, psi, T, si_tol=1e-15)
        np.testing.assert_allclose(T, Tz, rtol=1e-12)
        np.testing.assert_allclose(phi[:, 0], phiz, rtol=1e-12)
        np.testing.assert_allclose(phi[:, 1:], 0.0, atol=1e-12 * phiz)


@pytest.mark.parametrize("seed", [1, 2])
def test_sn_q1_energy_balance(orc, seed):
    c = workloads.small_case(7, 5, 1, 4, 8, seed=seed, T0=0.6)
    p = oracle_problem(c)
    p.psi_edge = (0.3, 0.0, 0.05, 0.0)
    ox, oy, oz, w = orc.quadrature(4, 8)
    T = c["T0"].reshape(-1).copy()
    T[:6] = 1.0
    psi = _q1_planck(p, T)
    h2 = (p.lx / p.nx) * (p.ly / p.ny)
    rho = np.asarray(p.rho_cv).reshape(-1)
    for _ in range(3):
        phi0 = np.tensordot(w, psi, axes=(0, 0))[:, 0]
        E0 = h2 * np.sum(rho * T + phi0 / p.c)
        psi, T, phi, it, out, inn = orc.sn_step_q1(p, psi, T, si_tol=1e-15, si_max_iter=20000)
        assert it > 0
        E1 = h2 * np.sum(rho * T + phi[:, 0] / p.c)
        assert abs(E1 - E0 + p.dt * (out - inn)) < 1e-12 * E1


def test_sn_q1_equilibrium_preserved(orc):
    c = workloads.small_case(6, 6, 1, 4, 8, T0=0.7)
    p = oracle_problem(c, psi_edge=[0] * 4)
    p.set_edge_temperatures([0.7] * 4)
    T = np.full(p.Nx, 0.7)
    psi = _q1_planck(p, T)
    for _ in range(2):
        psi, T, phi, it, *_ = orc.sn_step_q1(p, psi, T, si_tol=1e-15)
    np.testing.assert_allclose(T, 0.7, rtol=1e-13)
    np.testing.assert_allclose(psi[:, :, 0], psi[0, 0, 0], rtol=1e-12)
    np.testing.assert_allclose(psi[:, :, 1:], 0.0, atol=1e-12 * psi[0, 0, 0])


# ---- the SN-like DLR step on Q1 elements ----

def _q1_weights(p):
    hx, hy = p.lx / p.nx, p.ly / p.ny
    return np.tile(hx * hy * np.array([1.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 9.0]), p.Nx)


def _factors_of(p, w, psi_full, r):
    """X, S, W with X S W^T = psi_full (4 Nx x NOm) at rank r = 4 Nx: X the
    scaled unit basis (orthonormal in the Q1 inner product), S W^T its
    coefficients, factored by a w-weighted QR."""
    wq = _q1_weights(p)
    X = np.diag(1.0 / np.sqrt(wq))[:, :r]
    C = (np.sqrt(wq)[:, None] * psi_full)[:r]
    Q, R = np.linalg.qr(np.sqrt(w)[:, None] * C.T)
    return X, R.T.copy(), Q / np.sqrt(w)[:, None]


def test_full_rank_dlr_q1_equals_sn_q1(orc):
    c = workloads.small_case(2, 2, 16, 2, 8, seed=4, T0=0.5)
    p = oracle_problem(c)
    p.psi_edge = (0.2, 0.0, 0.1, 0.05)
    ox, oy, oz, w = orc.quadrature(2, 8)
    T = c["T0"].reshape(-1).copy()
    T[0] = 0.9
    psi = _q1_planck(p, T)                        # (NOm, Nx, 4)
    X, S, W = _factors_of(p, w, psi.reshape(p.NOm, -1).T, 16)
    np.testing.assert_allclose(X @ S @ W.T, psi.reshape(p.NOm, -1).T, atol=1e-14)
    Td = T.copy()
    for _ in range(2):
        X, S, W, Td, phid, itd, rc = orc.dlr_step_q1(p, X, S, W, Td, si_tol=1e-14)
        assert rc == 0 and itd > 0
        psi, T, phi, it, *_ = orc.sn_step_q1(p, psi, T, si_tol=1e-14)
        np.testing.assert_allclose(Td, T, rtol=1e-11)
        full = psi.reshape(p.NOm, -1).T
        np.testing.assert_allclose(X @ S @ W.T, full, rtol=0, atol=1e-11 * np.abs(full).max())
        np.testing.assert_allclose(phid, phi, rtol=0, atol=1e-11 * np.abs(phi).max())


def test_dlr_q1_infinite_medium_recurrence(orc):
    nx, ny, sig, rho, T0, dt = 4, 3, 10.0, 0.5, 0.5, 0.02
    p = orc.Problem(nx, ny, 2, 8, np.full(nx * ny, sig), np.full(nx * ny, rho), dt=dt)
    X = np.zeros((4 * p.Nx, 1))
    X[0::4, 0] = 1.0                      # the constant, orthonormal on the unit square
    W = np.full((p.NOm, 1), 1.0 / np.sqrt(4 * np.pi))
    S = np.array([[orc.planck(p.a_rad, p.c, T0) * np.sqrt(4 * np.pi)]])
    T = np.full(p.Nx, T0)
    Tz, phiz = T0, 4 * np.pi * orc.planck(p.a_rad, p.c, T0)
    for _ in range(10):
        Tz, phiz = _zero_d_step(Tz, phiz, sig, rho, dt, p.c, p.a_rad)
        p.psi_edge = (phiz / (4 * np.pi),) * 4
        X, S, W, T, phi, it, rc = orc.dlr_step_q1(p, X, S, W, T, si_tol=1e-15)
        assert rc == 0
        np.testing.assert_allclose(T, Tz, rtol=1e-12)
        np.testing.assert_allclose(phi[:, 0], phiz, rtol=1e-12)


# ---- DSA on Q1 elements (reading R20) ----

def _q1_coeffs_of(p, f):
    return _project(p, f)                       # (Nx, 4), exact for bilinear f


def test_q1_derivative_is_exact_on_continuous_bilinear_fields(orc):
    p = _problem(orc, 6, 5, lx=1.2, ly=0.9)
    hx, hy = p.lx / p.nx, p.ly / p.ny
    (X, Y), a, b = _centres(p)
    Dx, Dy = orc.q1_deriv(p, 0), orc.q1_deriv(p, 1)
    inner = np.zeros((p.ny, p.nx), bool)
    inner[1:-1, 1:-1] = True
    inner = inner.reshape(-1)
    for f, dfx, dfy in [(lambda x, y: x, lambda x, y: 1.0 + 0 * x, lambda x, y: 0 * x),
                        (lambda x, y: x * y, lambda x, y: y, lambda x, y: x),
                        (lambda x, y: 2 - y + 0.5 * x * y, lambda x, y: 0.5 * y, lambda x, y: -1 + 0.5 * x)]:
        u = _q1_coeffs_of(p, f).reshape(-1)
        # int_K v d f / dx_j for every basis function v: the Q1 mass times the projection
        wq = np.tile(hx * hy * np.array([1.0, 1 / 3, 1 / 3, 1 / 9]), p.Nx)
        for D, df in ((Dx, dfx), (Dy, dfy)):
            expect = wq * _q1_coeffs_of(p, df).reshape(-1)
            got = D @ u
            np.testing.assert_allclose(got.reshape(-1, 4)[inner], expect.reshape(-1, 4)[inner],
                                       rtol=0, atol=1e-13)


def test_q1_derivative_on_constants_is_the_centred_difference(orc):
    p = _problem(orc, 5, 4, lx=1.1, ly=0.8)
    hy = p.ly / p.ny
    u0 = np.random.default_rng(5).uniform(0.5, 2.0, p.Nx)
    u = np.zeros((p.Nx, 4))
    u[:, 0] = u0
    got = (orc.q1_deriv(p, 0) @ u.reshape(-1)).reshape(-1, 4)[:, 0].reshape(p.ny, p.nx)
    g = np.pad(u0.reshape(p.ny, p.nx), ((0, 0), (1, 1)))      # zero traces outside
    np.testing.assert_allclose(got, 0.5 * hy * (g[:, 2:] - g[:, :-2]), rtol=0, atol=1e-14)


def test_q1_dsa_operator_is_spd(orc):
    p = _problem(orc, 4, 3, lx=0.9, ly=1.3)
    st = 10.0 ** (2.0 * np.random.default_rng(7).uniform(size=p.Nx))
    sa = st * np.random.default_rng(8).uniform(0.01, 0.5, p.Nx)
    A = orc.dsa_matrix_q1(p, st, sa)
    assert np.max(np.abs(A - A.T)) <= 1e-13 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(A).min() > 0


def test_q1_sn_dsa_keeps_the_step_and_cuts_iterations(orc):
    c = workloads.small_case(5, 4, 1, 2, 8, seed=9, T0=1.0)
    c["sigma"] = np.full((4, 5), 1e3)
    res = []
    for dsa in (0, 1):
        p = oracle_problem(c)
        p.dsa, p.dsa_tol, p.dsa_max_iter = dsa, 0.1, 3
        T = c["T0"].reshape(-1).copy()
        psi = _q1_planck(p, T)
        psi, T, phi, it, *_ = orc.sn_step_q1(p, psi, T, si_tol=1e-12, si_max_iter=20000)
        res.append((T, psi, it))
    assert np.linalg.norm(res[1][0] - res[0][0]) <= 1e-9 * np.linalg.norm(res[0][0])
    assert np.linalg.norm(res[1][1] - res[0][1]) <= 1e-9 * np.linalg.norm(res[0][1])
    assert res[0][2] > 100 and res[1][2] * 5 < res[0][2], (res[0][2], res[1][2])


def _q1_mass_by_quadrature(p, coef):
    """int_K coef phi_i phi_j over each cell by 4 x 4 Gauss quadrature (the
    Legendre basis 1, xi, eta, xi eta), as a dense block-diagonal matrix."""
    hx, hy = p.lx / p.nx, p.ly / p.ny
    g, w = _gauss()
    M = np.zeros((4 * p.Nx, 4 * p.Nx))
    for c in range(p.Nx):
        B = np.zeros((4, 4))
        for gi, wi in zip(g, w):
            for gj, wj in zip(g, w):
                ph = np.array([1.0, gi, gj, gi * gj])
                B += wi * wj * np.outer(ph, ph) * hx * hy / 4
        M[4 * c:4 * c + 4, 4 * c:4 * c + 4] = coef[c] * B
    return M


def test_q1_dsa_operator_parts(orc):
    p = _problem(orc, 4, 5, lx=1.0, ly=1.2)
    rng = np.random.default_rng(11)
    st = rng.uniform(1.0, 30.0, p.Nx)
    sa = rng.uniform(0.1, 1.0, p.Nx)
    D = [orc.q1_deriv(p, 0), orc.q1_deriv(p, 1)]
    # M_a: the sigma_a-weighted Q1 mass matrix
    Ma = orc.dsa_matrix_q1(p, st, sa) - orc.dsa_matrix_q1(p, st, 0 * sa)
    np.testing.assert_allclose(Ma, _q1_mass_by_quadrature(p, sa), rtol=0, atol=1e-13)
    # (1/3) sum_j D_j^T M_t^-1 D_j: halving it by doubling sigma_t
    diff = orc.dsa_matrix_q1(p, st, sa) - orc.dsa_matrix_q1(p, 2 * st, sa)
    Mt_inv = np.linalg.inv(_q1_mass_by_quadrature(p, st))
    expect = sum(Dj.T @ Mt_inv @ Dj for Dj in D) / 6.0
    np.testing.assert_allclose(diff, expect, rtol=0, atol=1e-12 * np.abs(expect).max())
    # F0 penalises jumps only: zero on a continuous field away from the boundary
    F0 = orc.dsa_matrix_q1(p, np.full(p.Nx, 1e300), 0 * sa)
    u = _project(p, lambda x, y: 1 + x - 2 * y + x * y).reshape(-1)
    inner = np.zeros((p.ny, p.nx), bool)
    inner[1:-1, 1:-1] = True
    np.testing.assert_allclose((F0 @ u).reshape(-1, 4)[inner.reshape(-1)], 0.0, atol=1e-13)


def test_dlr_q1_dsa_keeps_the_step_and_cuts_iterations(orc):
    c = workloads.small_case(5, 4, 4, 2, 8, seed=10, T0=1.0)
    c["sigma"] = np.full((4, 5), 1e3)
    res = []
    for dsa in (0, 1):
        p = oracle_problem(c)
        p.dsa, p.dsa_tol, p.dsa_max_iter = dsa, 0.1, 3
        X = np.zeros((4 * p.Nx, 1))
        X[0::4, 0] = 1.0
        W = np.full((p.NOm, 1), 1.0 / np.sqrt(4 * np.pi))
        S = np.array([[orc.planck(p.a_rad, p.c, 1.0) * np.sqrt(4 * np.pi)]])
        T = c["T0"].reshape(-1).copy()
        T[:5] = 0.6                              # a cooler bottom row: not a 0-D problem
        X, S, W, T, phi, it, rc = orc.dlr_step_q1(p, X, S, W, T, si_tol=1e-12, si_max_iter=20000)
        assert rc == 0
        res.append((T, X @ S @ W.T, it))
    assert np.linalg.norm(res[1][0] - res[0][0]) <= 1e-9 * np.linalg.norm(res[0][0])
    assert np.linalg.norm(res[1][1] - res[0][1]) <= 1e-9 * np.linalg.norm(res[0][1])
    assert res[0][2] > 50 and res[1][2] * 3 < res[0][2], (res[0][2], res[1][2])
