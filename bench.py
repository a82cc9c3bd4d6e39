#!/usr/bin/env python3
"""Benchmark of the SN-like DLR time step (Algorithm 1 of Haut et al.) on GB300.

One "step" is one implicit DLR time step of the lognormal1024 workload (1024
x 1024 cells, log-normal opacity smoothed over 16 cells, central hot square
at T = 1, vacuum edges, rank 32, 32 x 64 angles), the largest single-GPU
configuration: angle selection, collocation sweeps with source iteration, QR
of Psi, projections, L-step, QR + SVD of L, temperature update, all in the
library's kernels with the state resident in HBM.

Printed JSON line (rank 0): cell-angle updates per second over the timed
steps (whole job for N GPUs; each rank steps its own replica, weak scaling),
the same measured through the public API with host buffers (e2e), DLR steps/s,
the all-FP64 GPU path on the same steps, the roofline of the
source-iteration kernel, the FP64 CPU oracle on all host cores on a bounded
sample (the first step) with the GPU paths' errors against it, and SM clocks
sampled during the timed region.  L2 is flushed between timed steps (value
and e2e alike).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "cell-angle updates/s"
WORKLOAD = "lognormal1024"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="dlr", choices=["dlr", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sn", action="store_true", help="skip the full-rank SN comparator")
    ap.add_argument("--no-aug", action="store_true", help="skip the augmented (rank-2r) step")
    ap.add_argument("--no-dsa", action="store_true", help="skip the DSA-accelerated step")
    ap.add_argument("--no-q1", action="store_true", help="skip the step on bilinear (Q1) elements")
    ap.add_argument("--q1", action="store_true", help="--kernel si: bilinear (Q1) elements")
    ap.add_argument("--dsa", action="store_true", help="served: every request with DSA")
    ap.add_argument("--dsa-max-iter", type=int, default=0, help="CG cap per DSA solve (0: the library's)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="CPU work of the oracle sample (checker256 and smaller)")
    ap.add_argument("--cpu-1thread", action="store_true",
                    help="also time the oracle sample on one thread")
    ap.add_argument("--kernel", default=None, choices=["sweep", "si"],
                    help="sweep: the hot kernel alone; si: two steps of the workload with the source "
                         "iteration fixed at --si-iters (a short run for profilers)")
    ap.add_argument("--si-iters", type=int, default=4, help="--kernel si: source iterations per step")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["lattice32", "checker256", "lognormal1024", "batch64", "served"])
    ap.add_argument("--requests", type=int, default=200, help="served: number of requests")
    ap.add_argument("--hbm-budget-gb", type=float, default=0.0, help="served: admission budget")
    ap.add_argument("--max-active", type=int, default=48, help="served: requests stepped together")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the sweep-plan autotuner (default plan: splitting threshold 1)")
    return ap.parse_args()


def case_config(case, precision):
    return {"workload": f"{case['name']}: {case['nx']}x{case['ny']} cells, rank {case['r']}, "
                        f"{case['n_polar']}x{case['n_azim']} angles, dt {case['dt']}",
            "nx": case["nx"], "ny": case["ny"], "rank": case["r"],
            "n_omega": case["n_polar"] * case["n_azim"], "precision": precision,
            "l2": "flushed between timed steps (256 MiB write), value and e2e alike",
            "inputs": "resident in HBM (value); host buffers each step (e2e)"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 50 ms) with host timestamps."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(device), "-lms", "50"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        win = [s for t, s in self.samples if t0 <= t <= t1] or [s for _, s in self.samples[-3:]]
        if not win:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(s[1]) for s in win if num(s[1]) is not None]
        mx = [num(s[2]) for s in win if num(s[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in win for i in range(4)
                          if len(s) > 5 + i and s[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(win)}


# ---------------------------------------------------------------- CPU

def si_traffic(workload, iters_per_launch):
    """DRAM bytes (read + write) per source-iteration launch from the
    committed ncu captures (profiles/k_si_traffic.json): bytes per iteration
    x this run's iterations per launch + the launch's fixed bytes; None when
    the capture is of another workload or the kernel sources changed since
    the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_si_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("workload") != workload:
            return None
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != rec["source_sha256"]:
            return None
        return rec["dram_bytes_per_si_iteration"] * iters_per_launch + rec.get("dram_bytes_per_launch_fixed", 0.0)
    except (OSError, KeyError, ValueError):
        return None


def _oracle_problem(case):
    import oracle
    p = oracle.Problem(case["nx"], case["ny"], case["n_polar"], case["n_azim"], case["sigma"],
                       case["rho_cv"], dt=case["dt"], c=case["c"], a_rad=case["a_rad"])
    p.set_edge_temperatures(case["T_edge"])
    return p


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_first_step(case, si_iters: int, threads: int):
    """The CPU baseline's sample: the FP64 oracle's first DLR step from the
    initial state with the source iteration fixed at si_iters (the count the
    GPU path took), on `threads` host threads.  Returns (updates/s, seconds,
    state after the step)."""
    import oracle
    oracle.set_threads(threads)
    p = _oracle_problem(case)
    T = case["T0"].reshape(-1).copy()
    X, S, W = oracle.initial_factors(p, T, case["r"])
    t0 = time.perf_counter()
    X, S, W, T, res = oracle.dlr_step(p, X, S, W, T, si_fixed_iters=si_iters)
    el = time.perf_counter() - t0
    if res.rc != 0:
        raise RuntimeError(f"oracle step failed: rc {res.rc}")
    return p.Nx * case["r"] * res.iters / el, el, (X, S, W, T, res.idx.copy())


def oracle_rate(case, seconds: float, steps=None, threads: int = 1):
    """FP64 CPU oracle: (updates/s, steps run, seconds) over whole steps from
    the initial state until `seconds` (or `steps`) are reached."""
    import oracle
    oracle.set_threads(threads)
    p = _oracle_problem(case)
    T = case["T0"].reshape(-1).copy()
    X, S, W = oracle.initial_factors(p, T, case["r"])
    upd, n, t0 = 0, 0, time.perf_counter()
    while True:
        X, S, W, T, res = oracle.dlr_step(p, X, S, W, T)
        upd += p.Nx * case["r"] * res.iters
        n += 1
        el = time.perf_counter() - t0
        if (steps is not None and n >= steps) or (steps is None and el >= seconds):
            break
    return upd / el, n, el


def psi_sample(X, S, W, ncols: int = 64):
    """psi = X S W^T at ncols evenly spaced angles (the full N x NOm array of
    the large workloads does not fit comfortably in host memory)."""
    cols = np.linspace(0, W.shape[0] - 1, ncols).astype(int)
    return X @ (S @ W[cols].T)


def rel_l2(a, b) -> float:
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


MIXED_SI_TOL = 1e-6  # the library's default stopping tolerance of the mixed path


def run_reference(args):
    """The oracle, as it stands, on all host cores (the base contract's
    reference arm): W untimed steps, then K timed steps of the same workload
    with the mixed path's stopping rule (max |d phi| <= 1e-6 max |phi|)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    case = workloads.CONFIGS[args.workload]()
    import oracle
    cores = host_cores()
    oracle.set_threads(cores)
    p = _oracle_problem(case)
    T = case["T0"].reshape(-1).copy()
    X, S, W = oracle.initial_factors(p, T, case["r"])
    kw = dict(si_tol=MIXED_SI_TOL, si_max_iter=case.get("si_max_iter", 1000))
    for _ in range(args.warmup):
        X, S, W, T, res = oracle.dlr_step(p, X, S, W, T, **kw)
    upd, t0 = 0, time.perf_counter()
    for _ in range(args.steps):
        X, S, W, T, res = oracle.dlr_step(p, X, S, W, T, **kw)
        upd += p.Nx * case["r"] * res.iters
    el = time.perf_counter() - t0
    v = upd / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": case_config(case, "fp64 (CPU oracle)"),
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": f"{args.steps} whole DLR steps of {case['name']} after "
                                       f"{args.warmup} warm-up steps, source iteration to "
                                       f"{MIXED_SI_TOL:g}, {oracle.get_threads()} threads"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- ranks
def reduce_over_ranks(total_ms: float, updates: float, dist=None):
    """Whole-job aggregate of a replicated run (each rank steps its own
    instance; no data-path collective): the slowest rank's time and the sum of
    all ranks' updates."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(total_ms), float(updates)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------- GPU
def timed_steps(dlr, torch, solver, K, flush):
    """K steps, each timed with CUDA events on the solver's stream, L2 flushed
    before each.  Returns (ms list)."""
    st = solver.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    for a, b in ev:
        with torch.cuda.stream(st):
            flush.fill_(1)
        a.record(st)
        solver.step(1)
        b.record(st)
    st.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def cpu_leg(args, dlr, case):
    """The CPU baseline and the GPU paths' errors against the FP64 oracle.

    Large workloads (beyond checker256): the sample is the first DLR step
    from the initial state.  Fresh GPU solvers (the library's own initial
    factors) take that step in mixed precision with the default stopping
    rule, then in FP64 with the same source-iteration count; the oracle
    takes it with that count on all host cores (timed: the baseline), and
    both GPU results are compared with it (T and psi on 64 sampled angles).
    Smaller workloads: whole oracle steps for about --cpu-seconds."""
    cores = host_cores()
    if case["nx"] * case["ny"] <= 256 * 256:
        v, n, el = oracle_rate(case, args.cpu_seconds, threads=cores)
        cpu = {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
               "sample": f"first {n} DLR steps of {case['name']} ({el:.1f} s, {cores} threads)"}
        return cpu, None
    gpu = {}
    with dlr.Solver(dlr.problem_from_case(case, precision=dlr.DLR_MIXED)) as s:
        s.step(1)
        n1 = s.stats()["si_iters_last"]
        X, S, W = s.factors()
        gpu["mixed"] = (s.T(), psi_sample(X, S, W), s.selected())
    with dlr.Solver(dlr.problem_from_case(case, precision=dlr.DLR_FP64, si_fixed_iters=n1)) as s:
        s.step(1)
        X, S, W = s.factors()
        gpu["fp64"] = (s.T(), psi_sample(X, S, W), s.selected())
    v, el, (Xo, So, Wo, To, idx) = oracle_first_step(case, n1, cores)
    po = psi_sample(Xo, So, Wo)
    cpu = {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
           "sample": f"first DLR step of {case['name']} from the initial state, source iteration "
                     f"fixed at the GPU's {n1} iterations ({el:.1f} s on {cores} threads)"}
    if args.cpu_1thread:
        v1, el1, _ = oracle_first_step(case, n1, 1)
        cpu["one_thread"] = {"value": v1, "seconds": el1}
    vs = {"sample": "first step from the library's own initial factors vs the oracle's, same "
                    f"source-iteration count ({n1}); psi = X S W^T at 64 sampled angles"}
    for k, (T, ps, sel) in gpu.items():
        vs[k] = {"rel_l2_T": rel_l2(T, To), "rel_l2_psi": rel_l2(ps, po),
                 "same_angles": sorted(sel.tolist()) == sorted(idx.tolist())}
    return cpu, vs


def run_gpu(args):
    import torch
    import paper_2601_18705_gb300 as dlr

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    case = workloads.CONFIGS[args.workload]()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # ---- main (mixed precision) ----
    solver = dlr.Solver(dlr.problem_from_case(case, precision=dlr.DLR_MIXED, allow_nonpositive=1))
    tuned = None if args.no_tune else dlr.autotune([solver])  # also applies to later solvers of this shape
    solver.step(args.warmup)
    solver.stream.synchronize()
    s0 = solver.stats()
    solver.set_timing(True)
    clk = ClockSampler(local) if rank == 0 else None
    time.sleep(0.15)
    barrier()
    tw0 = time.perf_counter()
    ms = timed_steps(dlr, torch, solver, args.steps, flush)
    barrier()
    tw1 = time.perf_counter()
    s1 = solver.stats()
    total_ms = float(sum(ms))
    updates = s1["cell_angle_updates"] - s0["cell_angle_updates"]
    iters = s1["si_iters_total"] - s0["si_iters_total"]
    si_ms = s1["ms_si_total"] - s0["ms_si_total"]
    si_launch = s1["si_launches"] - s0["si_launches"]
    launches = s1["kernel_launches"] - s0["kernel_launches"]
    grouped = bool(s1["sweep_grouped"])
    total_ms, updates_all = reduce_over_ranks(total_ms, updates, dist)
    if clk:
        time.sleep(0.1)
        clk.stop()
    value = updates_all / (total_ms / 1e3)
    T_mixed = solver.T()
    nonpos = solver.stats()["nonpositive_cells"]
    solver.close()

    # ---- e2e: public API with host buffers, copies inside the timed region,
    # timed like value (CUDA events on the solver's stream, L2 flushed
    # before each step) ----
    e2e = None
    if not args.no_e2e:
        s2 = dlr.Solver(dlr.problem_from_case(case, precision=dlr.DLR_MIXED, allow_nonpositive=1))
        s2.step(args.warmup)
        hostT = torch.empty(s2.N, dtype=torch.float64, pin_memory=True)
        s2.T_into(hostT)
        e0 = s2.stats()
        st2 = s2.stream
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier()
        for a, b in ev:
            with torch.cuda.stream(st2):
                flush.fill_(1)
            a.record(st2)
            s2.set_T(hostT)          # H2D of the step's input temperature (pinned host)
            s2.step(1)
            s2.T_into(hostT)         # D2H of the step's result (synchronises)
            b.record(st2)
        st2.synchronize()
        barrier()
        el_ms = float(sum(a.elapsed_time(b) for a, b in ev))
        e1 = s2.stats()
        s2.close()
        el_ms, eu = reduce_over_ranks(el_ms, e1["cell_angle_updates"] - e0["cell_angle_updates"], dist)
        e2e = {"value": eu / (el_ms / 1e3), "unit": METRIC, "h2d_bytes_per_step": 8 * case["nx"] * case["ny"],
               "d2h_bytes_per_step": 8 * case["nx"] * case["ny"], "ms_per_step": el_ms / args.steps,
               "timing": "CUDA events on the solver's stream around H2D + step + D2H, L2 flushed before each step"}

    # ---- the all-FP64 GPU path on the same steps ----
    fp64 = None
    if not args.no_fp64 and rank == 0:
        s3 = dlr.Solver(dlr.problem_from_case(case, precision=dlr.DLR_FP64, allow_nonpositive=1))
        s3.step(args.warmup)
        s3.stream.synchronize()
        f0 = s3.stats()
        ms64 = timed_steps(dlr, torch, s3, args.steps, flush)
        f1 = s3.stats()
        T64 = s3.T()
        s3.close()
        u64 = f1["cell_angle_updates"] - f0["cell_angle_updates"]
        t64 = sum(ms64)
        fp64 = {"value": u64 / (t64 / 1e3), "unit": METRIC, "ms_per_step": t64 / args.steps,
                "dlr_steps_per_s": args.steps / (t64 / 1e3),
                "mixed_vs_fp64_rel_l2_T": float(np.linalg.norm(T_mixed - T64) / np.linalg.norm(T64))}

    # ---- the full-rank SN step it approximates (all NOm angles), same steps ----
    sn = None
    if not args.no_sn and rank == 0:
        s4 = dlr.Solver(dlr.problem_from_case(case, precision=dlr.DLR_MIXED, allow_nonpositive=1,
                                              method=dlr.DLR_METHOD_SN))
        s4.step(args.warmup)
        s4.stream.synchronize()
        s4.set_timing(True)
        g0 = s4.stats()
        ms_sn = timed_steps(dlr, torch, s4, args.steps, flush)
        g1 = s4.stats()
        T_sn = s4.T()
        s4.close()
        usn = g1["cell_angle_updates"] - g0["cell_angle_updates"]
        tsn = sum(ms_sn)
        sn = {"method": f"full-rank SN over all {case['n_polar'] * case['n_azim']} angles, mixed",
              "value": usn / (tsn / 1e3), "unit": METRIC, "ms_per_step": tsn / args.steps,
              "dlr_steps_per_s": args.steps / (tsn / 1e3),
              "si_iters_per_step": (g1["si_iters_total"] - g0["si_iters_total"]) / args.steps,
              "T_rel_l2_dlr_vs_sn": float(np.linalg.norm(T_mixed - T_sn) / np.linalg.norm(T_sn))}
        # the same source-iteration kernel over all angles: per update it reads
        # the fixed source and writes psi (4 + 4 B), the scalar-flux phase
        # reads psi again (4 B), plus per-cell terms amortised over NOm angles
        K = case["n_polar"] * case["n_azim"]
        bpu = 12.0 + 16.0 / K
        nl = max(g1["si_launches"] - g0["si_launches"], 1)
        l_ms = (g1["ms_si_total"] - g0["ms_si_total"]) / nl
        ach = usn / nl * bpu / (l_ms / 1e3) / 1e9
        hbm_pk, pk_kind = peaks()
        sn["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm_pk, "unit": "GB/s",
                          "frac": ach / hbm_pk, "kernel": "k_si<float>", "peak_kind": pk_kind,
                          "bytes_per_update": bpu, "avg_launch_ms": l_ms}

    # ---- the same SN step with DSA-accelerated source iteration ----
    sn_dsa = None
    if not args.no_sn and not args.no_dsa and rank == 0:
        s7 = dlr.Solver(dlr.problem_from_case(case, precision=dlr.DLR_MIXED, allow_nonpositive=1,
                                              method=dlr.DLR_METHOD_SN, dsa=1,
                                              dsa_max_iter=args.dsa_max_iter))
        s7.step(args.warmup)
        s7.stream.synchronize()
        h0 = s7.stats()
        ms_snd = timed_steps(dlr, torch, s7, args.steps, flush)
        h1 = s7.stats()
        T_snd = s7.T()
        s7.close()
        si_s = h1["si_iters_total"] - h0["si_iters_total"]
        tsd = sum(ms_snd)
        sn_dsa = {"method": f"full-rank SN, DSA (at most {args.dsa_max_iter or 3} CG iterations per solve), mixed",
                  "ms_per_step": tsd / args.steps, "si_iters_per_step": si_s / args.steps,
                  "cg_iters_per_si_iter": (h1["dsa_iters_total"] - h0["dsa_iters_total"]) / max(si_s, 1),
                  "step_speedup_vs_sn": (sn["ms_per_step"] / (tsd / args.steps)) if sn else None,
                  "T_rel_l2_vs_sn": float(np.linalg.norm(T_snd - T_sn) / np.linalg.norm(T_sn)) if sn else None}

    # ---- the augmented step (rank-2r basis truncated to r), same steps ----
    aug = None
    if not args.no_aug and rank == 0 and 2 * case["r"] <= 32 and case["n_polar"] * case["n_azim"] <= 1024:
        s5 = dlr.Solver(dlr.problem_from_case(case, precision=dlr.DLR_MIXED, allow_nonpositive=1, augment=1))
        s5.step(args.warmup)
        s5.stream.synchronize()
        a0 = s5.stats()
        ms_aug = timed_steps(dlr, torch, s5, args.steps, flush)
        a1 = s5.stats()
        T_aug = s5.T()
        s5.close()
        ua = a1["cell_angle_updates"] - a0["cell_angle_updates"]
        ta = sum(ms_aug)
        aug = {"method": f"augmented step, rank {2 * case['r']} basis truncated to {case['r']}, mixed",
               "value": ua / (ta / 1e3), "unit": METRIC, "ms_per_step": ta / args.steps,
               "dlr_steps_per_s": args.steps / (ta / 1e3),
               "si_iters_per_step": (a1["si_iters_total"] - a0["si_iters_total"]) / args.steps}
        if sn is not None:
            aug["T_rel_l2_vs_sn"] = float(np.linalg.norm(T_aug - T_sn) / np.linalg.norm(T_sn))

    # ---- the same steps with DSA-accelerated source iteration (Section 4.5) ----
    dsa = None
    if not args.no_dsa and rank == 0:
        s6 = dlr.Solver(dlr.problem_from_case(case, precision=dlr.DLR_MIXED, allow_nonpositive=1, dsa=1,
                                              dsa_max_iter=args.dsa_max_iter))
        s6.step(args.warmup)
        s6.stream.synchronize()
        d0 = s6.stats()
        ms_dsa = timed_steps(dlr, torch, s6, args.steps, flush)
        d1 = s6.stats()
        T_dsa = s6.T()
        s6.close()
        ud = d1["cell_angle_updates"] - d0["cell_angle_updates"]
        td = sum(ms_dsa)
        si_d = d1["si_iters_total"] - d0["si_iters_total"]
        dsa = {"method": "DSA-accelerated source iteration (Jacobi-PCG, dsa_tol 0.1, at most "
                         f"{args.dsa_max_iter or 3} CG iterations per solve), mixed",
               "ms_per_step": td / args.steps, "dlr_steps_per_s": args.steps / (td / 1e3),
               "si_iters_per_step": si_d / args.steps,
               "cg_iters_per_si_iter": (d1["dsa_iters_total"] - d0["dsa_iters_total"]) / max(si_d, 1),
               "step_speedup_vs_plain": (total_ms / args.steps) / (td / args.steps),
               "T_rel_l2_vs_plain": float(np.linalg.norm(T_dsa - T_mixed) / np.linalg.norm(T_mixed)),
               "cell_angle_updates_per_s": ud / (td / 1e3)}

    # ---- the same steps on bilinear (Q1) elements (Section 4.4), mixed ----
    q1 = None
    if not args.no_q1 and rank == 0:
        s8 = dlr.Solver(dlr.problem_from_case(case, precision=dlr.DLR_MIXED, allow_nonpositive=1, element=1))
        s8.step(args.warmup)
        s8.stream.synchronize()
        s8.set_timing(True)
        q0 = s8.stats()
        ms_q1 = timed_steps(dlr, torch, s8, args.steps, flush)
        q1s = s8.stats()
        T_q1 = s8.T()
        s8.close()
        uq = q1s["cell_angle_updates"] - q0["cell_angle_updates"]
        tq = sum(ms_q1)
        nlq = max(q1s["si_launches"] - q0["si_launches"], 1)
        lq_ms = (q1s["ms_si_total"] - q0["ms_si_total"]) / nlq
        # per cell-angle update (FP32): the 4 fixed-source coefficients read,
        # the 4 psi coefficients written by the sweep and read back by the
        # scalar-flux phase; per cell sigma_t, sigma_s/4pi, phi read by the
        # sweep and the scalar-flux phase and written once, amortised over r
        bpq = 48.0 + 56.0 / case["r"]
        achq = uq / nlq * bpq / (lq_ms / 1e3) / 1e9
        hbm_q, kind_q = peaks()
        q1 = {"method": "SN-like DLR step on bilinear (Q1) elements, 4 coefficients per cell, mixed",
              "value": uq / (tq / 1e3), "unit": METRIC, "ms_per_step": tq / args.steps,
              "dlr_steps_per_s": args.steps / (tq / 1e3),
              "si_iters_per_step": (q1s["si_iters_total"] - q0["si_iters_total"]) / args.steps,
              "T_rel_l2_vs_dg0": float(np.linalg.norm(T_q1 - T_mixed) / np.linalg.norm(T_mixed)),
              "roofline": {"bound": "hbm", "achieved": achq, "peak": hbm_q, "unit": "GB/s",
                           "frac": achq / hbm_q, "kernel": "k_q1_si<float>", "peak_kind": kind_q,
                           "bytes_per_update": bpq, "avg_launch_ms": lq_ms}}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    hbm, kind = peaks()
    si_kernel = ("grouped source iteration (graph loop of k_grp_sweep, k_grp_qsum, k_grp_phi + last sweep)"
                 if grouped else "k_si<float> (per-angle source iteration)")
    traffic = si_traffic(args.workload, iters / max(si_launch, 1)) if grouped else None
    r = case["r"]
    bytes_per_update = 4.0 + 16.0 / r  # fixed-source read + amortised per-cell terms (FP32)
    per_launch_ms = si_ms / max(si_launch, 1)
    per_launch_updates = updates / max(si_launch, 1)
    achieved = per_launch_updates * bytes_per_update / (per_launch_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "kernel": si_kernel,
                "peak_kind": kind, "bytes_per_update": bytes_per_update,
                "avg_launch_ms": per_launch_ms,
                "traffic_note": "DRAM bytes per launch from profiles/k_si_traffic.json (ncu graph-level "
                                "captures of the same kernel sources at 2 and 6 iterations), at this "
                                "run's iterations per launch"}
    cpu, vs_oracle = None, None
    if not args.no_cpu_baseline and world == 1:
        cpu, vs_oracle = cpu_leg(args, dlr, case)
    clocks = clk.summary(tw0, tw1) if clk else None
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic", "config": case_config(case, "mixed: FP32 sweeps/projections, FP64 small LA and T"),
            "dlr_steps_per_s": world * args.steps / (total_ms / 1e3),
            "si_iters_per_step": iters / args.steps,
            "roofline": roofline, "cpu_baseline": cpu, "vs_oracle": vs_oracle, "e2e": e2e, "fp64_gpu": fp64, "sn_gpu": sn, "sn_dsa_gpu": sn_dsa, "augmented_gpu": aug, "dsa_gpu": dsa, "q1_gpu": q1,
            "clocks": clocks, "gpu_launches": int(launches),
            "nonpositive_cells_at_end": int(nonpos), "sweep_plan": tuned}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def run_kernel_sweep(args):
    """The hot kernel alone: r DG0 upwind sweeps (dlr_sweep) on the workload's
    mesh, directions of its quadrature, random sources; one CTA per direction."""
    import torch
    import paper_2601_18705_gb300 as dlr
    case = workloads.CONFIGS[args.workload]()
    nx, ny, r = case["nx"], case["ny"], case["r"]
    N = nx * ny
    td = torch.float32 if args.precision == "mixed" else torch.float64
    rng = np.random.default_rng(0)
    K = case["n_polar"] * case["n_azim"]
    k = rng.choice(K, r, replace=False)
    mu, wp = np.polynomial.legendre.leggauss(case["n_polar"])
    p, a = k // case["n_azim"], k % case["n_azim"]
    phi = (a + 0.5) * 2 * np.pi / case["n_azim"]
    s = np.sqrt(1 - mu[p] ** 2)
    dirs = np.stack([s * np.cos(phi), s * np.sin(phi)], 1)
    sig_t = torch.tensor(case["sigma"].reshape(-1) + 1 / (case["c"] * case["dt"]), dtype=td, device="cuda")
    src = torch.rand(r * N, dtype=td, device="cuda")
    for _ in range(args.warmup):
        dlr.sweep(nx, ny, dirs, [1, 0, 0, 0], sig_t, src)
    torch.cuda.synchronize()
    t = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dlr.sweep(nx, ny, dirs, [1, 0, 0, 0], sig_t, src)
        e1.record()
        torch.cuda.synchronize()
        t.append(e0.elapsed_time(e1))
    ms = statistics.median(t)
    print(json.dumps({"kernel": "sweep", "workload": args.workload, "precision": args.precision,
                      "directions": r, "cells": N, "ms_median": ms,
                      "cell_angle_updates_per_s": r * N / (ms / 1e3),
                      "ns_per_wavefront_step": ms * 1e6 / (nx + 1.25 * ny)}))


def run_kernel_si(args):
    """Two DLR steps of the workload (mixed precision, splitting threshold 2;
    --q1: on bilinear elements) with the source iteration fixed at
    --si-iters iterations: a short, repeatable run for profilers (e.g. ncu
    --graph-profiling graph)."""
    import paper_2601_18705_gb300 as dlr
    case = workloads.CONFIGS[args.workload]()
    spec = dlr.problem_from_case(case, precision=dlr.DLR_MIXED, si_fixed_iters=args.si_iters,
                                 element=1 if args.q1 else 0)
    with dlr.Solver(spec) as s:
        if not args.q1:
            dlr.set_split([s], 2.0)
        s.step(2)
        st = s.stats()
        print(json.dumps({"kernel": "si", "workload": args.workload, "element": "q1" if args.q1 else "dg0",
                          "si_iters_per_step": args.si_iters, "steps": st["steps"],
                          "sweep_grouped": st["sweep_grouped"], "T_min": float(s.T().min())}))


def run_batch64(args):
    """64 independent instances stepped as one batch (one launch per kernel
    per step for all of them), against the plain FP64 path run one instance
    at a time on the same steps."""
    import torch
    import paper_2601_18705_gb300 as dlr
    cases = workloads.batch64(steps=args.warmup + args.steps)
    st = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    solvers = [dlr.Solver(dlr.problem_from_case(c, precision=dlr.DLR_MIXED, allow_nonpositive=1),
                          stream=st) for c in cases]
    tuned = None if args.no_tune else dlr.autotune(solvers)
    dlr.step_batch(solvers, args.warmup)
    st.synchronize()
    u0 = sum(s.stats()["cell_angle_updates"] for s in solvers)
    ms = 0.0
    for _ in range(args.steps):
        with torch.cuda.stream(st):
            flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        dlr.step_batch(solvers, 1)
        e1.record(st)
        st.synchronize()
        ms += e0.elapsed_time(e1)
    u1 = sum(s.stats()["cell_angle_updates"] for s in solvers)
    for s in solvers:
        s.close()
    value = (u1 - u0) / (ms / 1e3)
    # plain FP64, one instance at a time, same steps
    fp_ms, fp_upd = 0.0, 0
    if not args.no_fp64:
        for c in cases:
            with dlr.Solver(dlr.problem_from_case(c, precision=dlr.DLR_FP64, allow_nonpositive=1)) as s:
                s.step(args.warmup)
                a = s.stats()["cell_angle_updates"]
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s.stream)
                s.step(args.steps)
                e1.record(s.stream)
                s.stream.synchronize()
                fp_ms += e0.elapsed_time(e1)
                fp_upd += s.stats()["cell_angle_updates"] - a
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batch64: 64 instances, sides {64..512}, ranks {8..32}, "
                                   "128..1024 angles, one launch per kernel per step",
                       "precision": "mixed", "l2": "flushed between timed steps"},
            "dlr_steps_per_s": 64 * args.steps / (ms / 1e3),
            "fp64_one_at_a_time": None if args.no_fp64 else {
                "value": fp_upd / (fp_ms / 1e3), "dlr_steps_per_s": 64 * args.steps / (fp_ms / 1e3),
                "ms_total": fp_ms},
            "sweep_plan": tuned}
    print(json.dumps(line))


def run_served(args):
    """Poisson arrivals (mean gap 50 ms); continuous batching with admission
    by HBM footprint; latency = completion - arrival."""
    import paper_2601_18705_gb300 as dlr
    from paper_2601_18705_gb300 import server
    reqs = [server.Request(rid=q["id"], arrival=t, case=workloads.materialize(q), steps=q["steps"])
            for t, q in workloads.served_requests(n=args.requests)]
    if args.dsa:
        for q in reqs:
            q.spec = dlr.problem_from_case(q.case, precision=q.precision, allow_nonpositive=1, dsa=1,
                                           dsa_max_iter=args.dsa_max_iter)
    srv = server.Server(max_active=args.max_active, hbm_budget=int(args.hbm_budget_gb * 2 ** 30))
    rep = srv.run(reqs, realtime=True)
    s = rep.summary()
    line = {"metric": METRIC, "value": s["cell_angle_updates_per_s"], "unit": METRIC, "n_gpus": 1,
            "steps": s["ticks"], "warmup": 0, "ms_per_step": 1e3 * s["wall_s"] / max(s["ticks"], 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"served: {args.requests} requests, Poisson 20/s, sides "
                                   "U{128..1024}, ranks {8,16,32}, 50-200 steps, 16x32 angles",
                       "precision": "mixed", "hbm_budget_gb": args.hbm_budget_gb,
                       "max_active": args.max_active, "dsa": int(args.dsa)},
            "served": s}
    print(json.dumps(line))


def main():
    args = parse()
    if args.kernel == "sweep":
        run_kernel_sweep(args)
        return
    if args.kernel == "si":
        run_kernel_si(args)
        return
    if args.workload == "batch64" and args.impl != "reference":
        run_batch64(args)
        return
    if args.workload == "served" and args.impl != "reference":
        run_served(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
