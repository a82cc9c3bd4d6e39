"""Pins of the oracle's quadrature (reading R5) and Planck function."""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("npol,naz", [(2, 4), (8, 16), (16, 32), (32, 64)])
def test_gauss_legendre_matches_numpy(orc, npol, naz):
    ox, oy, oz, w = orc.quadrature(npol, naz)
    x, wp = np.polynomial.legendre.leggauss(npol)  # textbook routine
    mu = oz.reshape(npol, naz)[:, 0]
    np.testing.assert_allclose(mu, x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(w.reshape(npol, naz)[:, 0], wp * 2 * np.pi / naz, rtol=1e-13)


@pytest.mark.parametrize("npol,naz", [(2, 4), (8, 16), (16, 32)])
def test_moments(orc, npol, naz):
    ox, oy, oz, w = orc.quadrature(npol, naz)
    assert abs(w.sum() - 4 * np.pi) < 1e-13
    np.testing.assert_allclose(ox ** 2 + oy ** 2 + oz ** 2, 1.0, atol=1e-14)
    for f in (ox, oy, oz, ox * oy, ox * oz):
        assert abs(np.dot(w, f)) < 1e-13
    # second moments: int Om_i Om_j dOm = 4 pi / 3 delta_ij (appendix identity)
    for f in (ox * ox, oy * oy, oz * oz):
        assert abs(np.dot(w, f) - 4 * np.pi / 3) < 1e-13


def test_no_grid_aligned_directions(orc):
    ox, oy, oz, w = orc.quadrature(8, 16)
    assert np.min(np.abs(ox)) > 0.05 and np.min(np.abs(oy)) > 0.05


def test_planck_closed_form(orc):
    assert orc.planck(1.0, 1.0, 1.0) == pytest.approx(1 / (4 * math.pi), rel=1e-15)
    assert orc.planck(0.01372, 299.792458, 2.0) == pytest.approx(
        0.01372 * 299.792458 * 16 / (4 * math.pi), rel=1e-15)
