"""Sweep work plans that split an angle's bands over several CTAs (edge rows
handed from CTA to CTA through tagged words in global memory), and the
autotuner that picks the plan.  A plan changes only which CTA sweeps which
band, never the arithmetic, so split and unsplit runs agree bit for bit; a
split run also matches the oracle within the path's tolerance."""
import numpy as np
import pytest

import workloads
from gpu_util import rel_l2, run_pair

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 2e-5}


@pytest.fixture(scope="module")
def dlr():
    import paper_2601_18705_gb300 as m
    return m


def _run(dlr, orc, case, prec, steps, split=None, tune=False, batch_with=None):
    """Steps from the oracle's initial factors; returns T, psi and the stats."""
    import torch
    from conftest import oracle_problem
    out = []
    cases = [case] + ([batch_with] if batch_with is not None else [])
    solvers = []
    st = torch.cuda.Stream()  # a batch shares one stream
    try:
        for c in cases:
            p = oracle_problem(c)
            X, S, W = orc.initial_factors(p, c["T0"].reshape(-1).copy(), c["r"])
            s = dlr.Solver(dlr.problem_from_case(c, precision=prec), stream=st)
            s.set_factors(X, S, W)
            solvers.append(s)
        if split is not None:
            dlr.set_split(solvers, split)
        tuned = dlr.autotune(solvers, iters=2, reps=1) if tune else None
        for _ in range(steps):
            dlr.step_batch(solvers, 1)
        for s in solvers:
            out.append((s.T(), s.psi(), s.stats()))
    finally:
        for s in solvers:
            s.close()
    return out, tuned


# (nx, ny, r): ny = 300 gives 10 bands with a ragged last one (12 rows), so
# the plans have units of 8 + 2 bands (FP32, 8 warps) or 4 + 4 + 2 (FP64, 4
# warps); ny = 1024 gives 32 whole bands
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(48, 300, 6), (37, 1024, 4)])
def test_split_equals_unsplit_bitwise(orc, dlr, prec, shape):
    nx, ny, r = shape
    case = workloads.small_case(nx, ny, r, 4, 8, seed=nx + ny, T0=0.4)
    ref, _ = _run(dlr, orc, case, prec, 3, split=0.0)
    for split in (1.0, 0.5):
        got, _ = _run(dlr, orc, case, prec, 3, split=split)
        (T0_, p0, s0), (T1, p1, s1) = ref[0], got[0]
        assert s1["si_iters_total"] == s0["si_iters_total"]
        assert np.array_equal(T1, T0_) and np.array_equal(p1, p0), split


@pytest.mark.parametrize("prec", [0, 1])
def test_split_parity_with_oracle(orc, dlr, prec):
    case = workloads.small_case(40, 290, 6, 4, 8, seed=5, T0=0.45)
    out, _ = run_pair(case, prec, 2, orc=orc, dlr=dlr, split=0.5)
    for eT, ep, oi, gi in out:
        assert eT < TOL[prec] and ep < TOL[prec], (eT, ep)


def test_split_in_a_batch_equals_each_alone(orc, dlr):
    big = workloads.small_case(64, 520, 6, 4, 8, seed=21, T0=0.5)
    small = workloads.small_case(30, 40, 4, 4, 8, seed=22, T0=0.3)
    alone_big, _ = _run(dlr, orc, big, 1, 2, split=0.0)
    alone_small, _ = _run(dlr, orc, small, 1, 2, split=0.0)
    both, _ = _run(dlr, orc, big, 1, 2, split=0.5, batch_with=small)
    for (Ta, pa, _), (Tb, pb, _) in zip([alone_big[0], alone_small[0]], both):
        assert np.array_equal(Ta, Tb) and np.array_equal(pa, pb)


def test_autotune_keeps_the_state(orc, dlr):
    case = workloads.small_case(40, 400, 6, 4, 8, seed=31, T0=0.6)
    ref, _ = _run(dlr, orc, case, 1, 2, split=0.0)
    got, tuned = _run(dlr, orc, case, 1, 2, tune=True)
    assert tuned["split"] in dlr.AUTOTUNE_CANDIDATES
    assert all(v > 0 for v in tuned["ms"].values()), tuned
    (Ta, pa, sa), (Tb, pb, sb) = ref[0], got[0]
    assert sb["si_iters_total"] == sa["si_iters_total"] and sb["steps"] == 2
    assert np.array_equal(Ta, Tb) and np.array_equal(pa, pb)
