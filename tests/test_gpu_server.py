"""The continuous-batching server: every request's result is the same alone
and in the mix (requests join and leave the batch while others run), and a
small HBM budget makes requests wait for admission without changing results."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _requests(dlr, server_mod, n=6):
    reqs = []
    for i in range(n):
        case = workloads.small_case(20 + 9 * i, 16 + 7 * (i % 3), 4 + (i % 3) * 2, 4, 8,
                                    seed=40 + i, T0=0.3)
        reqs.append(server_mod.Request(rid=i, arrival=0.0, case=case, steps=3 + (i % 4),
                                       precision=dlr.DLR_MIXED))
    return reqs


def _alone(dlr, req):
    spec = dlr.problem_from_case(req.case, precision=req.precision, allow_nonpositive=1)
    with dlr.Solver(spec) as s:
        s.step(req.steps)
        return s.T()


def test_results_same_alone_and_in_the_mix():
    import paper_2601_18705_gb300 as dlr
    from paper_2601_18705_gb300 import server
    reqs = _requests(dlr, server)
    srv = server.Server(max_active=3, keep_results=True)
    rep = srv.run(reqs, realtime=False)
    assert len(rep.latencies) == len(reqs)
    assert rep.max_active == 3 and rep.admission_waits > 0
    for q in reqs:
        Ta = _alone(dlr, q)
        err = np.linalg.norm(q.result_T - Ta) / np.linalg.norm(Ta)
        assert err <= 2e-5, (q.rid, err)


def test_small_budget_serialises_admission():
    import paper_2601_18705_gb300 as dlr
    from paper_2601_18705_gb300 import server
    reqs = _requests(dlr, server, n=4)
    biggest = max(dlr.footprint_bytes(dlr.problem_from_case(q.case, precision=q.precision)) for q in reqs)
    srv = server.Server(max_active=8, hbm_budget=biggest, keep_results=True)
    rep = srv.run(reqs, realtime=False)
    assert len(rep.latencies) == 4 and rep.admission_waits > 0
    assert rep.peak_bytes <= biggest and rep.max_active < 4
    for q in reqs:
        assert np.linalg.norm(q.result_T - _alone(dlr, q)) <= 2e-5 * np.linalg.norm(q.result_T)
