"""Failure detection on the GPU without a fault: a sweep unit is pointed at an
edge row that nothing writes (dlr_debug_lose_edge), so its bounded wait runs
out.  The step must end by itself, report the sticky DLR_ETIMEOUT, and leave
the context usable for the next solver."""
import time

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dlr():
    import paper_2601_18705_gb300 as m
    return m


def test_lost_edge_row_times_out_and_the_context_survives(dlr):
    case = workloads.small_case(64, 600, 4, 2, 8, seed=12)  # 19 bands: several units per angle
    spec = dlr.problem_from_case(case, precision=dlr.DLR_MIXED)
    with dlr.Solver(spec) as s:
        dlr.debug_lose_edge([s])
        t0 = time.perf_counter()
        with pytest.raises(dlr.DlrError) as e:
            s.step(1)
            s.T()
        el = time.perf_counter() - t0
        assert "ETIMEOUT" in str(e.value)
        assert el < 60.0
        assert s.stats()["status"] == dlr._lib.DLR_ETIMEOUT
    # a new solver on the same GPU steps normally
    with dlr.Solver(spec) as s2:
        s2.step(2)
        T = s2.T()
        assert np.all(np.isfinite(T)) and s2.stats()["status"] == dlr._lib.DLR_OK


def test_lose_edge_needs_a_split_angle(dlr):
    case = workloads.small_case(16, 40, 2, 2, 4)  # 2 bands: one unit per angle
    with dlr.Solver(dlr.problem_from_case(case, precision=dlr.DLR_MIXED)) as s:
        with pytest.raises(dlr.DlrError):
            dlr.debug_lose_edge([s])
