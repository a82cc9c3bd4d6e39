"""FP64 CPU oracle of the SN-like DLR time step (Haut et al., Section 4,
Algorithm 1), as a ctypes binding over the plain C code in ``oracle.c``.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product package never imports
it, and it imports nothing from the product package.  It shares no code with
the CUDA path.

Parity status per function (what pins it, in ``tests/test_oracle_*.py``):
  quadrature          pinned (numpy Gauss-Legendre, exact moments)
  coefficients        pinned (equilibrium preservation, 0-D recurrence)
  sweep               pinned (discrete closed forms, first-order convergence)
  lu / qr / svd       pinned (numpy / LAPACK)
  qdeim / deim        pinned (LAPACK dgeqp3 pivots, brute-force max volume,
                      DEIM interpolation property)
  lstep               pinned (dense solve of the coupled r*NOm system)
  dlr_step            pinned (= full SN at r = Nx; 0-D recurrence; equilibrium;
                      energy balance; positivity; collocation dense solve)
  sn_step             pinned (dense solve of the assembled SN system)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    stale = (not os.path.exists(_OUT)) or max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_OUT)
    if force or stale:
        tmp = _OUT + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        # OpenMP where the compiler has it (same results with any thread count)
        if subprocess.call(base + ["-fopenmp"], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _OUT)
    return _OUT


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (n <= 0: all processors)."""
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("lx", C.c_double),
                ("ly", C.c_double), ("n_polar", C.c_int), ("n_azim", C.c_int),
                ("dt", C.c_double), ("c", C.c_double), ("a_rad", C.c_double),
                ("sigma", _dp), ("rho_cv", _dp),
                ("psi_edge", C.c_double * 4), ("sigma_texp", C.c_double),
                ("cv_texp", C.c_double), ("T_ref", C.c_double),
                ("dsa", C.c_int), ("dsa_tol", C.c_double), ("dsa_max_iter", C.c_int),
                ("reflect", C.c_int * 4)]


class _Opts(C.Structure):
    _fields_ = [("selection", C.c_int), ("forced_idx", _ip),
                ("si_tol", C.c_double), ("si_max_iter", C.c_int),
                ("si_fixed_iters", C.c_int), ("canonicalize", C.c_int),
                ("augment", C.c_int)]


class _Diag(C.Structure):
    _fields_ = [("iters", C.c_int), ("dsa_iters", C.c_int), ("E_before", C.c_double),
                ("E_after", C.c_double), ("outflow", C.c_double),
                ("inflow", C.c_double), ("residual", C.c_double),
                ("min_T", C.c_double), ("min_phi", C.c_double),
                ("What_cond1", C.c_double), ("R_diag_ratio", C.c_double)]


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.oracle_planck.restype = C.c_double
        L.oracle_planck.argtypes = [C.c_double, C.c_double, C.c_double]
        L.oracle_quadrature.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp]
        L.oracle_coefficients.argtypes = [C.POINTER(_Problem), _dp, _dp, _dp, _dp, _dp]
        L.oracle_sweep.argtypes = [C.POINTER(_Problem), C.c_double, C.c_double, _dp, _dp, _dp]
        L.oracle_lu_solve.argtypes = [C.c_int, _dp, C.c_int, _dp, _dp]
        L.oracle_householder_qr.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
        L.oracle_jacobi_svd.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
        L.oracle_qdeim.argtypes = [C.c_int, C.c_int, _dp, _ip]
        L.oracle_deim.argtypes = [C.c_int, C.c_int, _dp, _ip]
        L.oracle_initial_factors.argtypes = [C.POINTER(_Problem), _dp, C.c_int, _dp, _dp, _dp]
        L.oracle_lstep.argtypes = [C.POINTER(_Problem), C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        L.oracle_dlr_step.argtypes = [C.POINTER(_Problem), C.c_int, _dp, _dp, _dp, _dp,
                                      C.POINTER(_Opts), _ip, _dp, C.POINTER(_Diag)]
        L.oracle_collocation.argtypes = [C.POINTER(_Problem), C.c_int, _dp, _dp, _dp, _dp, _ip,
                                         C.c_double, C.c_int, C.c_int, _dp, _ip]
        L.oracle_sn_step.argtypes = [C.POINTER(_Problem), _dp, _dp, C.c_double, C.c_int,
                                     _dp, _dp, _dp]
        L.oracle_sweep_in.argtypes = [C.POINTER(_Problem), C.c_double, C.c_double, _dp, _dp, _dp,
                                      _dp, _dp]
        L.oracle_reflect_index.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
        L.oracle_sn_step_q1.argtypes = [C.POINTER(_Problem), _dp, _dp, C.c_double, C.c_int,
                                        _dp, _dp, _dp]
        L.oracle_dlr_step_q1.argtypes = [C.POINTER(_Problem), C.c_int, _dp, _dp, _dp, _dp,
                                         C.c_double, C.c_int, _ip, _dp]
        L.oracle_q1_deriv.argtypes = [C.POINTER(_Problem), C.c_int, _dp]
        L.oracle_dsa_matrix_q1.argtypes = [C.POINTER(_Problem), _dp, _dp, _dp]
        L.oracle_sweep_q1.argtypes = [C.POINTER(_Problem), C.c_double, C.c_double, _dp, _dp, _dp,
                                      _dp, _dp]
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_get_threads.restype = C.c_int
        L.oracle_dsa_kappa.restype = C.c_double
        L.oracle_dsa_kappa.argtypes = [C.c_int, C.c_int, C.c_int]
        L.oracle_dsa_apply.argtypes = [C.POINTER(_Problem), _dp, _dp, _dp, _dp]
        L.oracle_dsa_diag.argtypes = [C.POINTER(_Problem), _dp, _dp, _dp]
        L.oracle_dsa_solve.argtypes = [C.POINTER(_Problem), _dp, _dp, _dp, C.c_double,
                                       C.c_int, _dp]
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _fortran(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _fptr(a: np.ndarray):
    assert a.flags.f_contiguous
    return a.ctypes.data_as(_dp)


def planck(a_rad: float, c: float, T: float) -> float:
    return lib().oracle_planck(a_rad, c, T)


@dataclass
class Problem:
    """Mesh, quadrature, constants and material fields of one TRT problem.
    ``sigma`` and ``rho_cv`` are (ny, nx) or flat Nx arrays, c = iy*nx + ix."""
    nx: int
    ny: int
    n_polar: int
    n_azim: int
    sigma: np.ndarray
    rho_cv: np.ndarray
    dt: float = 1e-3
    c: float = 299.792458
    a_rad: float = 0.01372
    lx: float = 1.0
    ly: float = 1.0
    psi_edge: tuple = (0.0, 0.0, 0.0, 0.0)
    sigma_texp: float = 0.0   # sigma(T) = sigma (T/T_ref)^-sigma_texp (reading R16)
    cv_texp: float = 0.0      # rho c_v(T) = rho_cv (T/T_ref)^cv_texp
    T_ref: float = 1.0
    dsa: int = 0              # diffusion synthetic acceleration (Section 4.5, reading R17)
    dsa_tol: float = 0.1      # CG stop: ||r||_2 <= dsa_tol ||b||_2
    dsa_max_iter: int = 3
    reflect: tuple = (0, 0, 0, 0)  # reflective edges L, R, B, T (reading R18, SN only)
    _keep: list = field(default_factory=list, repr=False)

    @property
    def Nx(self) -> int:
        return self.nx * self.ny

    @property
    def NOm(self) -> int:
        return self.n_polar * self.n_azim

    def set_edge_temperatures(self, T_edge) -> None:
        """psi_edge from edge temperatures (isotropic Planck inflow, reading
        R4); a negative temperature means vacuum."""
        self.psi_edge = tuple(planck(self.a_rad, self.c, t) if t >= 0 else 0.0
                              for t in T_edge)

    def cstruct(self) -> _Problem:
        sig = _f64(self.sigma).reshape(-1)
        rho = _f64(self.rho_cv).reshape(-1)
        assert sig.size == self.Nx and rho.size == self.Nx
        self._keep = [sig, rho]
        s = _Problem()
        s.nx, s.ny, s.lx, s.ly = self.nx, self.ny, self.lx, self.ly
        s.n_polar, s.n_azim = self.n_polar, self.n_azim
        s.dt, s.c, s.a_rad = self.dt, self.c, self.a_rad
        s.sigma, s.rho_cv = _ptr(sig), _ptr(rho)
        s.sigma_texp, s.cv_texp, s.T_ref = self.sigma_texp, self.cv_texp, self.T_ref
        s.dsa, s.dsa_tol, s.dsa_max_iter = int(self.dsa), float(self.dsa_tol), int(self.dsa_max_iter)
        for e in range(4):
            s.reflect[e] = int(self.reflect[e])
        for e in range(4):
            s.psi_edge[e] = float(self.psi_edge[e])
        return s


def quadrature(n_polar: int, n_azim: int):
    n = n_polar * n_azim
    ox, oy, oz, w = (np.zeros(n) for _ in range(4))
    lib().oracle_quadrature(n_polar, n_azim, _ptr(ox), _ptr(oy), _ptr(oz), _ptr(w))
    return ox, oy, oz, w


def coefficients(p: Problem, T0):
    T0 = _f64(T0).reshape(-1)
    out = [np.zeros(p.Nx) for _ in range(4)]
    lib().oracle_coefficients(C.byref(p.cstruct()), _ptr(T0), *map(_ptr, out))
    return dict(sigma_s=out[0], q=out[1], B0=out[2], D=out[3],
                sigma_t=_f64(p.sigma).reshape(-1) + 1.0 / (p.c * p.dt))


def sweep(p: Problem, ox: float, oy: float, sigma_t, src) -> np.ndarray:
    st, s = _f64(sigma_t).reshape(-1), _f64(src).reshape(-1)
    psi = np.zeros(p.Nx)
    lib().oracle_sweep(C.byref(p.cstruct()), float(ox), float(oy), _ptr(st), _ptr(s), _ptr(psi))
    return psi


def sweep_in(p: Problem, ox: float, oy: float, sigma_t, src, in_x, in_y) -> np.ndarray:
    st, s, ix, iy = (_f64(a).reshape(-1) for a in (sigma_t, src, in_x, in_y))
    psi = np.zeros(p.Nx)
    lib().oracle_sweep_in(C.byref(p.cstruct()), float(ox), float(oy), _ptr(st), _ptr(s), _ptr(ix),
                          _ptr(iy), _ptr(psi))
    return psi


def sweep_q1(p: Problem, ox: float, oy: float, sigma_t, src, in_x, in_y) -> np.ndarray:
    """Q1 DG sweep: src (Nx, 4) Legendre coefficients per cell, in_x (ny, 2),
    in_y (nx, 2) inflow traces; returns psi (Nx, 4)."""
    st = _f64(sigma_t).reshape(-1)
    s, ix, iy = (_f64(a).reshape(-1) for a in (src, in_x, in_y))
    assert s.size == 4 * p.Nx and ix.size == 2 * p.ny and iy.size == 2 * p.nx
    psi = np.zeros(4 * p.Nx)
    lib().oracle_sweep_q1(C.byref(p.cstruct()), float(ox), float(oy), _ptr(st), _ptr(s), _ptr(ix),
                          _ptr(iy), _ptr(psi))
    return psi.reshape(p.Nx, 4)


def sn_step_q1(p: Problem, psi, T, *, si_tol: float = 1e-14, si_max_iter: int = 5000):
    """One full-rank SN step on Q1 elements.  psi is (NOm, Nx, 4); returns
    new copies (psi, T, phi (Nx, 4), iterations, outflow, inflow)."""
    psi = _f64(psi).reshape(-1).copy()
    assert psi.size == 4 * p.Nx * p.NOm
    T = _f64(T).reshape(-1).copy()
    phi = np.zeros(4 * p.Nx)
    out, inn = C.c_double(), C.c_double()
    it = lib().oracle_sn_step_q1(C.byref(p.cstruct()), _ptr(psi), _ptr(T), si_tol, si_max_iter,
                                 _ptr(phi), C.byref(out), C.byref(inn))
    return psi.reshape(p.NOm, p.Nx, 4), T, phi.reshape(p.Nx, 4), it, out.value, inn.value


def dlr_step_q1(p: Problem, X, S, W, T, *, si_tol: float = 1e-13, si_max_iter: int = 5000):
    """One SN-like DLR step on Q1 elements.  X (4 Nx, r) Q1 coefficients,
    S (r, r), W (NOm, r), T (Nx).  Returns new copies (X, S, W, T, phi
    (Nx, 4), iterations, rc)."""
    X = _fortran(X).copy(order="F")
    S = _fortran(S).copy(order="F")
    W = _fortran(W).copy(order="F")
    T = _f64(T).reshape(-1).copy()
    r = X.shape[1]
    phi = np.zeros(4 * p.Nx)
    it = C.c_int(0)
    rc = lib().oracle_dlr_step_q1(C.byref(p.cstruct()), r, _fptr(X), _fptr(S), _fptr(W), _ptr(T),
                                  si_tol, si_max_iter, C.byref(it), _ptr(phi))
    return X, S, W, T, phi.reshape(p.Nx, 4), it.value, rc


def q1_deriv(p: Problem, axis: int) -> np.ndarray:
    """The Q1 DG derivative D_j as a dense (4 Nx, 4 Nx) matrix (reading R20)."""
    n = 4 * p.Nx
    D = np.zeros(n * n)
    lib().oracle_q1_deriv(C.byref(p.cstruct()), int(axis), _ptr(D))
    return D.reshape(n, n).T.copy()


def dsa_matrix_q1(p: Problem, sigma_t, sigma_a) -> np.ndarray:
    n = 4 * p.Nx
    st, sa = (_f64(a).reshape(-1) for a in (sigma_t, sigma_a))
    A = np.zeros(n * n)
    lib().oracle_dsa_matrix_q1(C.byref(p.cstruct()), _ptr(st), _ptr(sa), _ptr(A))
    return A.reshape(n, n).T.copy()


def reflect_index(n_polar: int, n_azim: int, k: int, axis: int) -> int:
    return lib().oracle_reflect_index(n_polar, n_azim, k, axis)


def dsa_kappa(n_polar: int, n_azim: int, axis: int) -> float:
    return lib().oracle_dsa_kappa(n_polar, n_azim, axis)


def dsa_apply(p: Problem, sigma_t, sigma_a, u) -> np.ndarray:
    st, sa, uu = (_f64(a).reshape(-1) for a in (sigma_t, sigma_a, u))
    out = np.zeros(p.Nx)
    lib().oracle_dsa_apply(C.byref(p.cstruct()), _ptr(st), _ptr(sa), _ptr(uu), _ptr(out))
    return out


def dsa_diag(p: Problem, sigma_t, sigma_a) -> np.ndarray:
    st, sa = (_f64(a).reshape(-1) for a in (sigma_t, sigma_a))
    d = np.zeros(p.Nx)
    lib().oracle_dsa_diag(C.byref(p.cstruct()), _ptr(st), _ptr(sa), _ptr(d))
    return d


def dsa_solve(p: Problem, sigma_t, sigma_a, b, tol: float = 1e-12, max_iter: int = 10000):
    """Jacobi-PCG solve of the DSA system A x = b; returns (x, iterations)."""
    st, sa, bb = (_f64(a).reshape(-1) for a in (sigma_t, sigma_a, b))
    x = np.zeros(p.Nx)
    it = lib().oracle_dsa_solve(C.byref(p.cstruct()), _ptr(st), _ptr(sa), _ptr(bb), float(tol),
                                int(max_iter), _ptr(x))
    return x, it


def lu_solve(A, B) -> np.ndarray:
    A = _fortran(A)
    B = _fortran(B if np.ndim(B) == 2 else np.asarray(B)[:, None])
    Xo = np.zeros_like(B, order="F")
    rc = lib().oracle_lu_solve(A.shape[0], _fptr(A), B.shape[1], _fptr(B), _fptr(Xo))
    if rc:
        raise np.linalg.LinAlgError("singular")
    return Xo


def householder_qr(A):
    A = _fortran(A)
    m, n = A.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    lib().oracle_householder_qr(m, n, _fptr(A), _fptr(Q), _fptr(R))
    return Q, R


def jacobi_svd(A):
    A = _fortran(A)
    n = A.shape[0]
    U = np.zeros((n, n), order="F")
    V = np.zeros((n, n), order="F")
    s = np.zeros(n)
    lib().oracle_jacobi_svd(n, _fptr(A), _fptr(U), _ptr(s), _fptr(V))
    return U, s, V


def qdeim(W) -> np.ndarray:
    W = _fortran(W)
    n, r = W.shape
    idx = np.zeros(r, dtype=np.int32)
    if lib().oracle_qdeim(n, r, _fptr(W), idx.ctypes.data_as(_ip)):
        raise np.linalg.LinAlgError("no finite pivot")
    return idx


def deim(W) -> np.ndarray:
    W = _fortran(W)
    n, r = W.shape
    idx = np.zeros(r, dtype=np.int32)
    if lib().oracle_deim(n, r, _fptr(W), idx.ctypes.data_as(_ip)):
        raise np.linalg.LinAlgError("singular interpolation matrix")
    return idx


def initial_factors(p: Problem, T0, r: int):
    T0 = _f64(T0).reshape(-1)
    X = np.zeros((p.Nx, r), order="F")
    S = np.zeros((r, r), order="F")
    W = np.zeros((p.NOm, r), order="F")
    if lib().oracle_initial_factors(C.byref(p.cstruct()), _ptr(T0), r, _fptr(X), _fptr(S), _fptr(W)):
        raise ValueError("rank too large for the mesh / quadrature")
    return X, S, W


def lstep(p: Problem, X, sigma_t, sigma_s, q, Lt0) -> np.ndarray:
    X = _fortran(X)
    r = X.shape[1]
    Lt0 = _fortran(Lt0)
    L = np.zeros((r, p.NOm), order="F")
    a = [_f64(v).reshape(-1) for v in (sigma_t, sigma_s, q)]
    if lib().oracle_lstep(C.byref(p.cstruct()), r, _fptr(X), *map(_ptr, a), _fptr(Lt0), _fptr(L)):
        raise np.linalg.LinAlgError("singular L-step system")
    return L


@dataclass
class StepResult:
    rc: int
    idx: np.ndarray
    phi: np.ndarray
    iters: int
    diag: dict


def dlr_step(p: Problem, X, S, W, T, *, selection: int = 0, forced_idx=None,
             si_tol: float = 1e-13, si_max_iter: int = 1000,
             si_fixed_iters: int = 0, canonicalize: int = 1, augment: int = 0):
    """One SN-like DLR step (augment=1: the augmented rank-2r step truncated
    back to rank r, reading R15).  Returns new (X, S, W, T) copies and a
    StepResult; the inputs are not modified."""
    X = _fortran(X).copy(order="F")
    S = _fortran(S).copy(order="F")
    W = _fortran(W).copy(order="F")
    T = _f64(T).reshape(-1).copy()
    r = X.shape[1]
    o = _Opts()
    o.selection, o.si_tol, o.si_max_iter = selection, si_tol, si_max_iter
    o.si_fixed_iters, o.canonicalize, o.augment = si_fixed_iters, canonicalize, augment
    fi = None
    if forced_idx is not None:
        fi = np.ascontiguousarray(forced_idx, dtype=np.int32)
        o.forced_idx = fi.ctypes.data_as(_ip)
    idx = np.zeros(r, dtype=np.int32)
    phi = np.zeros(p.Nx)
    d = _Diag()
    rc = lib().oracle_dlr_step(C.byref(p.cstruct()), r, _fptr(X), _fptr(S), _fptr(W),
                               _ptr(T), C.byref(o), idx.ctypes.data_as(_ip), _ptr(phi),
                               C.byref(d))
    diag = {k: getattr(d, k) for k, _ in _Diag._fields_}
    return X, S, W, T, StepResult(rc, idx, phi, d.iters, diag)


def collocation(p: Problem, X0, S0, W0, T0, idx, *, si_tol: float = 1e-14,
                si_max_iter: int = 5000, si_fixed_iters: int = 0):
    """Steps 1-4 of Algorithm 1 at the given angles; returns (Psi, iters)."""
    X0, S0, W0 = _fortran(X0), _fortran(S0), _fortran(W0)
    r = X0.shape[1]
    T0 = _f64(T0).reshape(-1)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    Psi = np.zeros((p.Nx, r), order="F")
    it = C.c_int()
    rc = lib().oracle_collocation(C.byref(p.cstruct()), r, _fptr(X0), _fptr(S0), _fptr(W0),
                                  _ptr(T0), idx.ctypes.data_as(_ip), si_tol, si_max_iter,
                                  si_fixed_iters, _fptr(Psi), C.byref(it))
    if rc == -1:
        raise np.linalg.LinAlgError("singular What")
    return Psi, it.value, rc


def sn_step(p: Problem, psi, T, *, si_tol: float = 1e-14, si_max_iter: int = 5000):
    """One full-rank SN step.  psi is (Nx, NOm); returns new copies."""
    psi = _fortran(psi).copy(order="F")
    T = _f64(T).reshape(-1).copy()
    phi = np.zeros(p.Nx)
    out, inn = C.c_double(), C.c_double()
    it = lib().oracle_sn_step(C.byref(p.cstruct()), _fptr(psi), _ptr(T), si_tol, si_max_iter,
                              _ptr(phi), C.byref(out), C.byref(inn))
    return psi, T, phi, it, out.value, inn.value


def energy(p: Problem, T, phi) -> float:
    """E = sum_c h^2 (rho_cv T + phi / c) (Section 2.1 energy balance)."""
    h2 = (p.lx / p.nx) * (p.ly / p.ny)
    return float(h2 * np.sum(_f64(p.rho_cv).reshape(-1) * _f64(T).reshape(-1)
                             + _f64(phi).reshape(-1) / p.c))
