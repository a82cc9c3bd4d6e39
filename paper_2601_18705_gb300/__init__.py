"""GB300-native SN-like dynamic-low-rank (DLR) solver for gray thermal
radiative transfer in 2-D (Haut et al., Section 4 and Algorithm 1).

The Python layer marshals arguments for the C ABI of include/dlr.h; every
step of the method runs in the CUDA kernels of libdlr_gb300.so.  PyTorch
supplies device memory (through the allocator callback) and streams.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import (DLR_FP64, DLR_METHOD_DLR, DLR_METHOD_SN, DLR_MIXED, DLR_SEL_DEIM,  # noqa: F401
                   DLR_SEL_QDEIM, DlrError,
                   check, load)

__all__ = ["Solver", "step_batch", "autotune", "set_split", "sweep", "tc_gemm", "footprint_bytes", "DlrError", "DLR_FP64",
           "DLR_MIXED", "DLR_SEL_QDEIM", "DLR_SEL_DEIM", "DLR_METHOD_DLR", "DLR_METHOD_SN",
           "problem_from_case"]


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


@dataclass
class ProblemSpec:
    nx: int
    ny: int
    n_polar: int
    n_azim: int
    rank: int
    sigma: np.ndarray
    rho_cv: np.ndarray
    T0: np.ndarray
    T_edge: tuple = (-1.0, -1.0, -1.0, -1.0)
    lx: float = 1.0
    ly: float = 1.0
    dt: float = 1e-3
    c: float = 299.792458
    a_rad: float = 0.01372
    precision: int = DLR_FP64
    selection: int = DLR_SEL_QDEIM
    si_tol: float = 0.0
    si_max_iter: int = 0
    si_fixed_iters: int = 0
    allow_nonpositive: int = 0
    method: int = DLR_METHOD_DLR
    augment: int = 0     # 1: augmented step (rank-2r basis truncated back to rank r)
    sigma_texp: float = 0.0  # sigma(T) = sigma (T/T_ref)^-sigma_texp, at each step's T0
    cv_texp: float = 0.0     # rho c_v(T) = rho_cv (T/T_ref)^cv_texp
    T_ref: float = 1.0
    dsa: int = 0             # 1: diffusion synthetic acceleration of the source iteration
    dsa_tol: float = 0.0     # CG stop ||r|| <= dsa_tol ||b|| (0: 0.1)
    dsa_max_iter: int = 0    # CG cap per solve (0: 3)
    reflect: tuple = (0, 0, 0, 0)  # reflective edges L, R, B, T (full-rank SN only)
    sweep_mode: int = 0      # mixed DLR source iteration: 0 autotuned, 1 one angle per warp, 2 grouped
    element: int = 0         # 0 DG0 cells, 1 bilinear (Q1) elements (4 coefficients per cell)

    def cstruct(self):
        keep = [_f64(self.sigma), _f64(self.rho_cv), _f64(self.T0)]
        N = self.nx * self.ny
        for a in keep:
            if a.size != N:
                raise ValueError("field size does not match nx*ny")
        p = _lib.DlrProblem()
        p.nx, p.ny, p.lx, p.ly = self.nx, self.ny, self.lx, self.ly
        p.n_polar, p.n_azim, p.rank = self.n_polar, self.n_azim, self.rank
        p.dt, p.c, p.a_rad = self.dt, self.c, self.a_rad
        dp = C.POINTER(C.c_double)
        p.sigma, p.rho_cv, p.T0 = (a.ctypes.data_as(dp) for a in keep)
        for e in range(4):
            p.T_edge[e] = float(self.T_edge[e])
        p.precision, p.selection, p.augment = self.precision, self.selection, int(self.augment)
        p.si_tol, p.si_max_iter, p.si_fixed_iters = self.si_tol, self.si_max_iter, self.si_fixed_iters
        p.allow_nonpositive = 1 if self.allow_nonpositive else 0
        p.method = self.method
        p.sigma_texp, p.cv_texp, p.T_ref = self.sigma_texp, self.cv_texp, self.T_ref
        p.dsa, p.dsa_tol, p.dsa_max_iter = int(self.dsa), float(self.dsa_tol), int(self.dsa_max_iter)
        for e in range(4):
            p.reflect[e] = int(self.reflect[e])
        p.sweep_mode = int(self.sweep_mode)
        p.element = int(self.element)
        return p, keep


def problem_from_case(case: dict, precision=None, **kw) -> ProblemSpec:
    """ProblemSpec of a workloads case dict."""
    prec = case.get("precision", "fp64") if precision is None else precision
    if isinstance(prec, str):
        prec = DLR_MIXED if prec == "mixed" else DLR_FP64
    spec = ProblemSpec(nx=case["nx"], ny=case["ny"], n_polar=case["n_polar"],
                       n_azim=case["n_azim"], rank=case["r"], sigma=case["sigma"],
                       rho_cv=case["rho_cv"], T0=case["T0"], T_edge=tuple(case["T_edge"]),
                       lx=case.get("lx", 1.0), ly=case.get("ly", 1.0), dt=case["dt"],
                       c=case["c"], a_rad=case["a_rad"], precision=prec,
                       si_max_iter=case.get("si_max_iter", 0),
                       sigma_texp=case.get("sigma_texp", 0.0), cv_texp=case.get("cv_texp", 0.0),
                       T_ref=case.get("T_ref", 1.0))
    for k, v in kw.items():
        setattr(spec, k, v)
    return spec


def footprint_bytes(spec: ProblemSpec) -> int:
    p, keep = spec.cstruct()
    return int(load().dlr_footprint_bytes(C.byref(p)))


class _TorchArena:
    """Device memory for a handle from PyTorch's caching allocator."""

    def __init__(self, device, stream):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream
        self.blocks = {}
        self._alloc = _lib.ALLOC_FN(self.alloc)
        self._free = _lib.FREE_FN(self.free)

    def alloc(self, nbytes, ctx):
        try:
            with self.torch.cuda.stream(self.stream):
                t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        ptr = t.data_ptr()
        self.blocks[ptr] = t
        return ptr

    def free(self, ptr, ctx):
        self.blocks.pop(ptr, None)


class Solver:
    """One SN-like DLR instance (or, with spec.method = DLR_METHOD_SN, one
    full-rank SN instance) resident on the GPU.

    spec: ProblemSpec; use_torch_memory: allocate device state from PyTorch
    (else cudaMalloc); stream: a torch.cuda.Stream (a new one by default);
    hbm_budget: reject problems whose footprint exceeds it (bytes, 0 = none).
    """

    def __init__(self, spec: ProblemSpec, *, use_torch_memory: bool = True, stream=None,
                 hbm_budget: int = 0):
        import torch
        L = load()
        self.spec = spec
        self.N = spec.nx * spec.ny
        self.K = spec.n_polar * spec.n_azim
        self.sn = spec.method == DLR_METHOD_SN
        self.r = self.K if self.sn else spec.rank
        # rows of X and psi: one per cell, four (Legendre coefficients) on bilinear elements
        self.rows = self.N * (4 if getattr(spec, "element", 0) == 1 else 1)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        rt = _lib.DlrRuntime()
        rt.stream = C.c_void_p(self.stream.cuda_stream)
        self._arena = None
        if use_torch_memory:
            self._arena = _TorchArena(torch.device("cuda", torch.cuda.current_device()), self.stream)
            rt.alloc, rt.free = self._arena._alloc, self._arena._free
        rt.hbm_budget = int(hbm_budget)
        p, keep = spec.cstruct()
        h = C.c_void_p()
        check(L.dlr_create(C.byref(p), C.byref(rt), C.byref(h)))
        self._rt = rt
        self.h = h

    # -- lifetime --
    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            load().dlr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- stepping --
    def step(self, nsteps: int = 1) -> None:
        check(load().dlr_step(self.h, int(nsteps)))

    # -- state --
    def T(self) -> np.ndarray:
        out = np.empty(self.N)
        check(load().dlr_get_T(self.h, out.ctypes.data, 0))
        return out

    def T_into(self, tensor) -> None:
        check(load().dlr_get_T(self.h, C.c_void_p(tensor.data_ptr()), 1 if tensor.is_cuda else 0))

    def set_T(self, T) -> None:
        if hasattr(T, "data_ptr"):
            check(load().dlr_set_T(self.h, C.c_void_p(T.data_ptr()), 1 if T.is_cuda else 0))
        else:
            a = _f64(T)
            check(load().dlr_set_T(self.h, a.ctypes.data, 0))

    def factors(self):
        X = np.empty((self.rows, self.r), order="F")
        S = np.empty((self.r, self.r), order="F")
        W = np.empty((self.K, self.r), order="F")
        r = C.c_int32()
        check(load().dlr_get_factors(self.h, X.ctypes.data, S.ctypes.data, W.ctypes.data,
                                     C.byref(r), 0))
        return X, S, W

    def set_factors(self, X, S, W) -> None:
        X = np.asfortranarray(X, dtype=np.float64)
        S = np.asfortranarray(S, dtype=np.float64)
        W = np.asfortranarray(W, dtype=np.float64)
        assert X.shape == (self.rows, self.r) and S.shape == (self.r, self.r) and W.shape == (self.K, self.r)
        check(load().dlr_set_factors(self.h, X.ctypes.data, S.ctypes.data, W.ctypes.data, 0))

    def psi(self) -> np.ndarray:
        """psi (rows x NOm; rows = Nx, or 4 Nx Legendre coefficients on
        bilinear elements): the full-rank state of an SN instance, or X S W^T
        of a DLR instance (formed on the device)."""
        out = np.empty((self.rows, self.K), order="F")
        check(load().dlr_get_psi(self.h, out.ctypes.data, 0))
        return out

    def set_psi(self, psi) -> None:
        """Replaces the angular flux of an SN instance (rows x NOm)."""
        a = np.asfortranarray(psi, dtype=np.float64)
        assert a.shape == (self.rows, self.K)
        check(load().dlr_set_psi(self.h, a.ctypes.data, 0))

    def quadrature(self):
        om = np.empty((self.K, 3))
        w = np.empty(self.K)
        dp = C.POINTER(C.c_double)
        check(load().dlr_get_quadrature(self.h, om.ctypes.data_as(dp), w.ctypes.data_as(dp)))
        return om, w

    def selected(self) -> np.ndarray:
        idx = np.empty(self.r, dtype=np.int32)
        check(load().dlr_get_selected(self.h, idx.ctypes.data_as(C.POINTER(C.c_int32))))
        return idx

    def stats(self) -> dict:
        s = _lib.DlrStats()
        check(load().dlr_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _lib.DlrStats._fields_}

    def set_timing(self, on: bool) -> None:
        check(load().dlr_set_timing(self.h, 1 if on else 0))

    def set_edge_inflow(self, edge: int, psi_iso: float) -> None:
        check(load().dlr_set_edge_inflow(self.h, int(edge), float(psi_iso)))


def step_batch(solvers, nsteps: int = 1) -> None:
    """Steps several solvers as one batch (shared launches)."""
    arr = (C.c_void_p * len(solvers))(*[s.h.value for s in solvers])
    check(load().dlr_step_batch(arr, len(solvers), int(nsteps)))


AUTOTUNE_CANDIDATES = (0.0, 2.0, 1.0, 0.5)  # splitting thresholds, in dlr_autotune's order


def autotune(solvers, *, iters: int = 12, reps: int = 3) -> dict:
    """Autotunes the sweep work plan of the batch `solvers` (the same list
    later passed to step_batch; one solver for Solver.step): times each
    candidate -- the per-angle and the grouped source-iteration kernel, each
    with every splitting threshold -- on the device and keeps the fastest.
    Each timed launch runs `iters` source iterations: a count near a step's
    own, so that the fixed cost of a launch (the grouped kernel's set-up and
    its last sweep, which writes psi) weighs as it does in a step.
    Returns {"split": chosen threshold (0 = no split), "grouped": whether
    the grouped kernel was chosen, "ms": {threshold: ms per launch} of the
    per-angle kernel, "ms_grouped": the same for the grouped kernel (-1:
    the batch cannot take it)}."""
    arr = (C.c_void_p * len(solvers))(*[s.h.value for s in solvers])
    chosen = C.c_double(0.0)
    nc = len(AUTOTUNE_CANDIDATES)
    ms = (C.c_double * (2 * nc))()
    check(load().dlr_autotune(arr, len(solvers), int(iters), int(reps), C.byref(chosen), ms))
    ms = list(ms)
    grouped = min(ms[nc:]) >= 0 and min(ms[nc:]) < min(ms[:nc])
    return {"split": chosen.value, "grouped": bool(grouped),
            "ms": dict(zip(AUTOTUNE_CANDIDATES, ms[:nc])),
            "ms_grouped": dict(zip(AUTOTUNE_CANDIDATES, ms[nc:]))}


def debug_lose_edge(solvers) -> None:
    """Testing aid: the next step of the batch `solvers` waits for an edge row
    that nothing writes, gives up after its time bound and reports ETIMEOUT."""
    arr = (C.c_void_p * len(solvers))(*[s.h.value for s in solvers])
    check(load().dlr_debug_lose_edge(arr, len(solvers)))


def tc_gemm(A, B, *, stream=None):
    """Testing aid: D = A B^T (A: m x k, B: n x k, contiguous float32 CUDA
    tensors; m in {128, 256}, n in {16, 32}, k a multiple of 32) by the
    fifth-generation tensor cores (tcgen05, split TF32 products)."""
    import torch
    m, k = A.shape
    n = B.shape[0]
    D = torch.empty(m, n, dtype=torch.float32, device=A.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    check(load().dlr_debug_tc_gemm(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()), m, n, k,
                                   C.c_void_p(D.data_ptr()), C.c_void_p(st.cuda_stream)))
    return D


def set_split(solvers, split: float) -> None:
    """Sets the splitting threshold of the sweep work plan of the batch
    `solvers` (0 = one work unit per angle) without timing."""
    arr = (C.c_void_p * len(solvers))(*[s.h.value for s in solvers])
    check(load().dlr_set_split(arr, len(solvers), float(split)))


def sweep(nx, ny, dirs, psi_edge, sigma_t, src, *, lx=1.0, ly=1.0, stream=None):
    """DG0 upwind sweeps of the hot kernel for n_dir directions.  sigma_t (N)
    and src (n_dir*N) are CUDA tensors of float64 (FP64) or float32 (mixed);
    returns psi (n_dir*N) of the same dtype."""
    import torch
    dirs = _f64(dirs)
    n_dir = dirs.size // 2
    edge = _f64(psi_edge)
    prec = DLR_MIXED if sigma_t.dtype == torch.float32 else DLR_FP64
    psi = torch.empty(n_dir * nx * ny, dtype=sigma_t.dtype, device=sigma_t.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    dp = C.POINTER(C.c_double)
    check(load().dlr_sweep(nx, ny, lx, ly, n_dir, dirs.ctypes.data_as(dp), edge.ctypes.data_as(dp),
                           prec, C.c_void_p(sigma_t.data_ptr()), C.c_void_p(src.data_ptr()),
                           C.c_void_p(psi.data_ptr()), C.c_void_p(st.cuda_stream)))
    return psi
