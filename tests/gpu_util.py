"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_pair(case, precision, steps, *, orc, dlr, forced=None, si_fixed_iters=0, si_tol=None,
             selection=0, start=None, allow_nonpositive=0, split=None, augment=0, dsa=0,
             dsa_tol=0.1, dsa_max_iter=500, iters_out=None, sweep_mode=0, reflect=None):
    """Runs the oracle and the GPU solver side by side from the same state.
    Returns per-step (T error, psi error, oracle idx, gpu idx) and both states.
    When the GPU picks different angles than the oracle (a near-tie), the
    oracle step is repeated with the GPU's indices."""
    from conftest import oracle_problem
    p = oracle_problem(case)
    p.dsa, p.dsa_tol, p.dsa_max_iter = dsa, dsa_tol, dsa_max_iter
    kw = {}
    if reflect is not None:
        p.reflect = reflect
        kw["reflect"] = reflect
    if si_fixed_iters:
        kw["si_fixed_iters"] = si_fixed_iters
    spec = dlr.problem_from_case(case, precision=precision, selection=selection,
                                 allow_nonpositive=allow_nonpositive, augment=augment, dsa=dsa,
                                 dsa_tol=dsa_tol, dsa_max_iter=dsa_max_iter, sweep_mode=sweep_mode, **kw)
    if si_tol is not None:
        spec.si_tol = si_tol
    T = case["T0"].reshape(-1).copy()
    if start is None:
        X, S, W = orc.initial_factors(p, T, case["r"])
    else:
        X, S, W = start
    tol_o = 1e-13 if si_tol is None else si_tol
    out = []
    with dlr.Solver(spec) as s:
        s.set_factors(X, S, W)
        if split is not None:
            dlr.set_split([s], split)
        for _ in range(steps):
            X1, S1, W1, T1, res = orc.dlr_step(p, X, S, W, T, selection=selection,
                                               si_fixed_iters=si_fixed_iters, si_tol=tol_o,
                                               augment=augment)
            assert res.rc == 0, res
            s.step(1)
            gidx = s.selected()
            if sorted(gidx.tolist()) != sorted(res.idx.tolist()):
                X1, S1, W1, T1, res2 = orc.dlr_step(p, X, S, W, T, forced_idx=gidx,
                                                    si_fixed_iters=si_fixed_iters, si_tol=tol_o,
                                                    augment=augment)
                assert res2.rc == 0
            X, S, W, T = X1, S1, W1, T1
            if iters_out is not None:
                iters_out.append((res.iters, s.stats()["si_iters_last"], res.diag["dsa_iters"]))
            Tg = s.T()
            psig = s.psi()
            out.append((rel_l2(Tg, T), rel_l2(psig, X @ S @ W.T), res.idx.copy(), gidx.copy()))
        stats = s.stats()
    return out, stats
