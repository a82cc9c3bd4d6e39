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


def _cudart():
    """The CUDA runtime library this process already loaded (the DLR
    library links it), found through the process's mappings."""
    with open("/proc/self/maps") as f:
        paths = {ln.split()[-1] for ln in f if "libcudart.so" in ln}
    if not paths:
        pytest.skip("libcudart not mapped in this process")
    return C.CDLL(sorted(paths)[0])


def _device_memory_state(rt, dev):
    """(free bytes, reserved and used bytes of the default stream-ordered
    memory pool) of the device."""
    free, total = C.c_size_t(), C.c_size_t()
    assert rt.cudaMemGetInfo(C.byref(free), C.byref(total)) == 0
    pool = C.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(C.byref(pool), dev) == 0
    vals = []
    for attr in (5, 7):  # cudaMemPoolAttrReservedMemCurrent, cudaMemPoolAttrUsedMemCurrent
        v = C.c_uint64()
        assert rt.cudaMemPoolGetAttribute(pool, attr, C.byref(v)) == 0
        vals.append(v.value)
    return free.value, vals


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


def _sweep_args(nx, ny, n_dir, td, prec, seed):
    import torch
    rng = np.random.default_rng(seed)
    N = nx * ny
    dirs = np.ascontiguousarray(rng.uniform(-1, 1, (n_dir, 2)))
    edge = np.array([0.7, 0.2, 0.4, 0.1])
    sig_t = torch.tensor(rng.uniform(0.5, 300.0, N), dtype=td, device="cuda")
    src = torch.tensor(rng.uniform(0.0, 2.0, n_dir * N), dtype=td, device="cuda")
    return dirs, edge, sig_t, src


def test_noalloc_allocates_nothing():
    """After a first call (which may load the device code), further calls
    leave the device's free memory and its default memory pool unchanged."""
    import torch
    from paper_2601_18705_gb300 import _lib
    L = _lib.load()
    dp = C.POINTER(C.c_double)
    nx, ny, n_dir = 64, 48, 12
    dirs, edge, sig_t, src = _sweep_args(nx, ny, n_dir, torch.float32, _lib.DLR_MIXED, 7)
    out = torch.empty(n_dir * nx * ny, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    args = (nx, ny, 1.0, 1.0, n_dir, dirs.ctypes.data_as(dp), edge.ctypes.data_as(dp), _lib.DLR_MIXED,
            C.c_void_p(sig_t.data_ptr()), C.c_void_p(src.data_ptr()), C.c_void_p(out.data_ptr()),
            C.c_void_p(stream.cuda_stream))
    _lib.check(L.dlr_sweep_noalloc(*args))
    torch.cuda.synchronize()
    rt = _cudart()
    dev = torch.cuda.current_device()
    before = _device_memory_state(rt, dev)
    for _ in range(3):
        _lib.check(L.dlr_sweep_noalloc(*args))
    torch.cuda.synchronize()
    after = _device_memory_state(rt, dev)
    assert after[1] == before[1]
    assert after[0] >= before[0] - (2 << 20)


def test_noalloc_rejects_too_wide_mesh_then_works():
    """A mesh wider than the sweep's shared memory allows is refused with
    DLR_EINVAL before anything is enqueued, like dlr_sweep; the next valid
    call still succeeds and matches dlr_sweep."""
    import torch
    from paper_2601_18705_gb300 import _lib
    L = _lib.load()
    dp = C.POINTER(C.c_double)
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    dirs = np.full((1, 2), 0.5)
    edge = np.zeros(4)
    for fn in (L.dlr_sweep, L.dlr_sweep_noalloc):
        rc = fn(100000, 1, 1.0, 1.0, 1, dirs.ctypes.data_as(dp), edge.ctypes.data_as(dp), _lib.DLR_MIXED,
                C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), C.c_void_p(0))
        assert rc == _lib.DLR_EINVAL
        assert b"too large" in L.dlr_last_error()
    nx, ny, n_dir = 40, 37, 5
    dirs, edge, sig_t, src = _sweep_args(nx, ny, n_dir, torch.float32, _lib.DLR_MIXED, 9)
    want = torch.empty(n_dir * nx * ny, dtype=torch.float32, device="cuda")
    got = torch.full_like(want, float("nan"))
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (nx, ny, 1.0, 1.0, n_dir, dirs.ctypes.data_as(dp), edge.ctypes.data_as(dp), _lib.DLR_MIXED,
            C.c_void_p(sig_t.data_ptr()), C.c_void_p(src.data_ptr()))
    _lib.check(L.dlr_sweep(*args, C.c_void_p(want.data_ptr()), st))
    _lib.check(L.dlr_sweep_noalloc(*args, C.c_void_p(got.data_ptr()), st))
    w, g = want.cpu().numpy(), got.cpu().numpy()
    assert np.linalg.norm(g - w) <= 2e-6 * np.linalg.norm(w)
