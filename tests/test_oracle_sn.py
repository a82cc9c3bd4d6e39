"""Pins of the oracle's full-rank SN step: dense direct solve, exact energy
balance, equilibrium preservation (pins reading R1) and positivity."""
import numpy as np
import pytest

import workloads
from conftest import oracle_problem
from dense_ref import sn_dense


def _case(nx=4, ny=4, npol=2, naz=8, T0=0.4, seed=3):
    c = workloads.small_case(nx, ny, 1, npol, naz, seed=seed, T0=T0)
    return c


def test_sn_step_equals_dense_solve(orc):
    c = _case()
    p = oracle_problem(c)
    ox, oy, oz, w = orc.quadrature(c["n_polar"], c["n_azim"])
    T0 = c["T0"].reshape(-1)
    rng = np.random.default_rng(0)
    psi0 = rng.uniform(0.0, 0.5, (p.Nx, p.NOm))
    psi, T, phi, it, out, inn = orc.sn_step(p, psi0, T0, si_tol=1e-15)
    assert it > 0
    coef = orc.coefficients(p, T0)
    ref = sn_dense(p, coef, psi0, ox, oy, w)
    np.testing.assert_allclose(psi, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
    phi_ref = ref @ w
    Tref = T0 + p.dt * p.sigma.reshape(-1) * (phi_ref - 4 * np.pi * coef["B0"]) / coef["D"]
    np.testing.assert_allclose(T, Tref, rtol=1e-13)


@pytest.mark.parametrize("seed", [1, 2])
def test_sn_energy_balance(orc, seed):
    c = _case(nx=7, ny=5, npol=4, naz=8, T0=0.6, seed=seed)
    p = oracle_problem(c)
    p.psi_edge = (0.3, 0.0, 0.05, 0.0)
    ox, oy, oz, w = orc.quadrature(c["n_polar"], c["n_azim"])
    T = c["T0"].reshape(-1)
    psi = np.full((p.Nx, p.NOm), orc.planck(p.a_rad, p.c, 0.6))
    for _ in range(3):
        E0 = orc.energy(p, T, psi @ w)
        psi, T, phi, it, out, inn = orc.sn_step(p, psi, T, si_tol=1e-15)
        E1 = orc.energy(p, T, phi)
        assert abs(E1 - E0 + p.dt * (out - inn)) < 1e-12 * E1


def test_sn_equilibrium_preserved(orc):
    c = _case(nx=6, ny=6, npol=4, naz=8, T0=0.7)
    p = oracle_problem(c, psi_edge=[0] * 4)
    p.set_edge_temperatures([0.7] * 4)
    B = orc.planck(p.a_rad, p.c, 0.7)
    psi = np.full((p.Nx, p.NOm), B)
    T = np.full(p.Nx, 0.7)
    for _ in range(2):
        psi, T, phi, it, out, inn = orc.sn_step(p, psi, T, si_tol=1e-15)
    np.testing.assert_allclose(T, 0.7, rtol=1e-13)
    np.testing.assert_allclose(psi, B, rtol=1e-12)


def test_sn_positivity(orc):
    c = workloads.small_case(12, 10, 1, 4, 8, seed=5, T0=0.02)
    p = oracle_problem(c)
    psi = np.zeros((p.Nx, p.NOm))
    T = c["T0"].reshape(-1)
    for _ in range(3):
        psi, T, phi, it, out, inn = orc.sn_step(p, psi, T)
        assert psi.min() >= 0 and T.min() > 0
