"""Pins of the oracle's DG0 upwind sweep (reading R6) against closed forms
of the discrete scheme and against the continuum solution of the
pure-absorber transport equation (first-order convergence)."""
import math

import numpy as np
import pytest


def _absorber(orc, nx, ny, sigma, psi_edge, lx=1.0, ly=1.0):
    return orc.Problem(nx, ny, 2, 4, np.full(nx * ny, sigma), np.ones(nx * ny),
                       lx=lx, ly=ly, psi_edge=psi_edge)


@pytest.mark.parametrize("mu,edge", [(0.6, 0), (-0.35, 1)])
def test_grid_aligned_geometric_decay(orc, mu, edge):
    nx, ny, sig, pb = 17, 5, 3.0, 2.5
    pe = [0.0] * 4
    pe[edge] = pb
    p = _absorber(orc, nx, ny, sig, pe)
    psi = orc.sweep(p, mu, 0.0, np.full(nx * ny, sig), np.zeros(nx * ny)).reshape(ny, nx)
    h = 1.0 / nx
    i = np.arange(nx) if mu > 0 else np.arange(nx)[::-1]
    want = pb * (1.0 + sig * h / abs(mu)) ** (-(i + 1.0))
    for row in psi:
        np.testing.assert_allclose(row, want, rtol=1e-14, atol=0)


def _oblique_closed_form(nx, ny, ax, ay, sig, pb):
    """psi_{i,j} = pb sum_{j'<=j} a^{i+1} b^{j-j'} C(i+j-j', i): monotone
    lattice paths from the inflow column (sweep coordinates)."""
    a = ax / (sig + ax + ay)
    b = ay / (sig + ax + ay)
    out = np.zeros((ny, nx))
    for j in range(ny):
        for i in range(nx):
            out[j, i] = pb * sum(a ** (i + 1) * b ** (j - jp) * math.comb(i + j - jp, i)
                                 for jp in range(j + 1))
    return out


@pytest.mark.parametrize("ox,oy", [(0.5, 0.3), (-0.5, 0.3), (0.4, -0.7), (-0.2, -0.9)])
def test_oblique_binomial_closed_form(orc, ox, oy):
    nx, ny, sig, pb = 9, 7, 2.0, 1.5
    lx, ly = 1.3, 0.7
    pe = [0.0] * 4
    pe[0 if ox > 0 else 1] = pb  # inflow through the entering x-edge only
    p = _absorber(orc, nx, ny, sig, pe, lx, ly)
    psi = orc.sweep(p, ox, oy, np.full(nx * ny, sig), np.zeros(nx * ny)).reshape(ny, nx)
    want = _oblique_closed_form(nx, ny, abs(ox) / (lx / nx), abs(oy) / (ly / ny), sig, pb)
    if ox < 0:
        want = want[:, ::-1]
    if oy < 0:
        want = want[::-1, :]
    np.testing.assert_allclose(psi, want, rtol=1e-13, atol=0)


def test_y_inflow_closed_form(orc):
    nx, ny, sig, pb = 6, 8, 1.0, 0.8
    ox, oy = 0.3, 0.8
    p = _absorber(orc, nx, ny, sig, [0, 0, pb, 0])
    psi = orc.sweep(p, ox, oy, np.full(nx * ny, sig), np.zeros(nx * ny)).reshape(ny, nx)
    want = _oblique_closed_form(ny, nx, abs(oy) * ny, abs(ox) * nx, sig, pb).T
    np.testing.assert_allclose(psi, want, rtol=1e-13)


def test_uniform_source_interior_limit(orc):
    # no inflow, uniform source: far downstream psi -> src / sigma_t exactly
    nx = ny = 60
    p = _absorber(orc, nx, ny, 50.0, [0, 0, 0, 0])
    psi = orc.sweep(p, 0.6, 0.5, np.full(nx * ny, 50.0), np.full(nx * ny, 7.0)).reshape(ny, nx)
    assert abs(psi[-1, -1] - 7.0 / 50.0) < 1e-12


def test_first_order_convergence_grid_aligned(orc):
    sig, mu = 2.0, 0.7
    errs = []
    for n in (64, 128, 256, 512, 1024):
        p = _absorber(orc, n, 2, sig, [1.0, 0, 0, 0])
        psi = orc.sweep(p, mu, 0.0, np.full(2 * n, sig), np.zeros(2 * n)).reshape(2, n)[0]
        x = (np.arange(n) + 0.5) / n
        errs.append(np.max(np.abs(psi - np.exp(-sig * x / mu))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    # pre-asymptotic rates rise monotonically towards 1
    assert np.all(np.diff(rates) > 0) and 0.95 < rates[-1] < 1.05, rates


def test_first_order_convergence_oblique(orc):
    sig, ox, oy = 1.5, 0.8, 0.35
    tan = oy / ox
    errs = []
    for n in (32, 64, 128, 256):
        p = _absorber(orc, n, n, sig, [1.0, 0, 0, 0])
        psi = orc.sweep(p, ox, oy, np.full(n * n, sig), np.zeros(n * n)).reshape(n, n)
        x = (np.arange(n) + 0.5) / n
        X, Y = np.meshgrid(x, x)
        lit = (Y - X * tan > 0.3) & (X < 0.6)
        exact = np.exp(-sig * X / ox)
        errs.append(np.max(np.abs(psi - exact)[lit]))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 0.8) & (rates < 1.25)), rates
