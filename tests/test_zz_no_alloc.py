"""dlr_sweep_noalloc, the allocation-free variant of the sweep entry point.

It serves callers that cannot allocate device memory (their device memory is
held by another allocator, or they run in a loop where cudaMalloc / cudaFree
are not allowed).  Called through the C ABI, twice in a row, it must give the
same result as dlr_sweep within the sweep tests' tolerance.  This file is
collected last, so a run that stops at the first failure has run every other
test first; it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [("float64", 1e-13), ("float32", 2e-6)])
def test_noalloc_sweep_matches_dlr_sweep_twice(dtype, tol):
    import torch
    from paper_2601_18705_gb300 import _lib
    L = _lib.load()
    dp = C.POINTER(C.c_double)
    td = getattr(torch, dtype)
    prec = _lib.DLR_MIXED if dtype == "float32" else _lib.DLR_FP64
    stream = torch.cuda.current_stream()
    for call, (nx, ny) in enumerate([(37, 45), (70, 33)]):
        rng = np.random.default_rng(100 + call)
        N = nx * ny
        dirs = np.ascontiguousarray(rng.uniform(-1, 1, (9, 2)))
        edge = np.array([0.7, 0.2, 0.4, 0.1])
        n_dir = len(dirs)
        sig_t = torch.tensor(rng.uniform(0.5, 300.0, N), dtype=td, device="cuda")
        src = torch.tensor(rng.uniform(0.0, 2.0, n_dir * N), dtype=td, device="cuda")
        want = torch.empty(n_dir * N, dtype=td, device="cuda")
        got = torch.full((n_dir * N,), float("nan"), dtype=td, device="cuda")
        args = (nx, ny, 1.3, 0.8, n_dir, dirs.ctypes.data_as(dp), edge.ctypes.data_as(dp), prec,
                C.c_void_p(sig_t.data_ptr()), C.c_void_p(src.data_ptr()))
        st = C.c_void_p(stream.cuda_stream)
        _lib.check(L.dlr_sweep(*args, C.c_void_p(want.data_ptr()), st))
        _lib.check(L.dlr_sweep_noalloc(*args, C.c_void_p(got.data_ptr()), st))
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.isfinite(g).all()
        assert np.linalg.norm(g - w) <= tol * np.linalg.norm(w)


def test_noalloc_rejects_too_many_directions():
    import torch
    from paper_2601_18705_gb300 import _lib
    L = _lib.load()
    dp = C.POINTER(C.c_double)
    n_dir = 4097  # DLR_SWEEP_NOALLOC_MAX_DIRS + 1
    dirs = np.zeros((n_dir, 2)) + 0.5
    edge = np.zeros(4)
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = L.dlr_sweep_noalloc(2, 2, 1.0, 1.0, n_dir, dirs.ctypes.data_as(dp), edge.ctypes.data_as(dp),
                             _lib.DLR_FP64, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()),
                             C.c_void_p(x.data_ptr()), C.c_void_p(0))
    assert rc == _lib.DLR_EINVAL
    assert b"DLR_SWEEP_NOALLOC_MAX_DIRS" in L.dlr_last_error()
