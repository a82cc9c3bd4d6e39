"""GPU parity of the hot kernel (the DG0 upwind sweep of Algorithm 1 step 4)
against the oracle's sweep and the discrete closed forms."""
import math

import numpy as np
import pytest

from gpu_util import rel_l2

pytestmark = pytest.mark.gpu


def _dirs():
    return np.array([[0.5, 0.3], [-0.5, 0.3], [0.4, -0.7], [-0.2, -0.9], [0.7, 0.0],
                     [-0.6, 0.0], [0.0, 0.8], [0.0, -0.3], [0.99, 0.01], [-0.01, 0.95]])


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 50), (50, 1), (32, 32), (37, 45), (70, 33),
                                   (33, 129), (256, 64), (1024, 40)])
@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_sweep_matches_oracle(orc, nx, ny, dtype):
    import torch
    import paper_2601_18705_gb300 as dlr
    rng = np.random.default_rng(nx * 1000 + ny)
    N = nx * ny
    dirs = _dirs()
    sig_t = rng.uniform(0.5, 300.0, N)
    src = rng.uniform(0.0, 2.0, (len(dirs), N))
    edge = np.array([0.7, 0.2, 0.4, 0.1])
    td = getattr(torch, dtype)
    psi = dlr.sweep(nx, ny, dirs, edge, torch.tensor(sig_t, dtype=td, device="cuda"),
                    torch.tensor(src.reshape(-1), dtype=td, device="cuda"), lx=1.3, ly=0.8)
    psi = psi.cpu().numpy().reshape(len(dirs), N)
    p = orc.Problem(nx, ny, 2, 4, np.ones(N), np.ones(N), lx=1.3, ly=0.8, psi_edge=tuple(edge))
    tol = 1e-13 if dtype == "float64" else 2e-6
    for d, (ox, oy) in enumerate(dirs):
        ref = orc.sweep(p, ox, oy, sig_t, src[d])
        assert rel_l2(psi[d], ref) < tol, (d, ox, oy, rel_l2(psi[d], ref))


def test_sweep_oblique_closed_form_on_gpu():
    import torch
    import paper_2601_18705_gb300 as dlr
    nx, ny, sig, pb = 40, 35, 2.0, 1.5
    ox, oy = 0.5, 0.3
    dirs = np.array([[ox, oy]])
    psi = dlr.sweep(nx, ny, dirs, [pb, 0, 0, 0], torch.full((nx * ny,), sig, dtype=torch.float64, device="cuda"),
                    torch.zeros(nx * ny, dtype=torch.float64, device="cuda")).cpu().numpy().reshape(ny, nx)
    ax, ay = ox * nx, oy * ny
    a, b = ax / (sig + ax + ay), ay / (sig + ax + ay)
    for j in (0, 5, 34):
        for i in (0, 7, 39):
            want = pb * sum(a ** (i + 1) * b ** (j - jp) * math.comb(i + j - jp, i) for jp in range(j + 1))
            assert abs(psi[j, i] - want) <= 1e-13 * want
