import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def oracle_problem(case, psi_edge=None):
    """oracle.Problem for a workloads case dict."""
    import oracle
    p = oracle.Problem(case["nx"], case["ny"], case["n_polar"], case["n_azim"],
                       case["sigma"], case["rho_cv"], dt=case["dt"], c=case["c"],
                       a_rad=case["a_rad"], lx=case.get("lx", 1.0), ly=case.get("ly", 1.0),
                       sigma_texp=case.get("sigma_texp", 0.0), cv_texp=case.get("cv_texp", 0.0),
                       T_ref=case.get("T_ref", 1.0))
    if psi_edge is not None:
        p.psi_edge = tuple(psi_edge)
    else:
        p.set_edge_temperatures(case["T_edge"])
    return p


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
