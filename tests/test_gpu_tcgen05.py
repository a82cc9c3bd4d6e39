"""The fifth-generation tensor-core (tcgen05) form of the contraction of the
mixed-precision projections (MMAs of kind TF32, operands split into two
TF32 parts, FP32 accumulator in tensor memory) on plain arrays, against an
FP64 product: D = A B^T.  The
bound per entry is relative to sum_k |a_ik| |b_jk|: about 2^-20 for the
split products plus FP32 accumulation over k (k 2^-24), written below with
a factor 4 of margin.  On failure the message tells which layout mistakes
the result matches (a transposed core matrix, swapped operands, a wrong
accumulator lane map), since those are the plausible ones."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dlr():
    import paper_2601_18705_gb300 as m
    return m


def _operands(m, n, k, seed):
    rng = np.random.default_rng(seed)
    # entries spread over several binades, some exactly representable
    A = (rng.standard_normal((m, k)) * np.exp2(rng.integers(-6, 6, (m, 1)))).astype(np.float32)
    B = (rng.standard_normal((n, k)) * np.exp2(rng.integers(-6, 6, (1, k)))).astype(np.float32)
    A[0, :] = 1.0
    B[:, 0] = 0.0
    return A, B


def _diagnose(D, A, B):
    """Which entries are wrong, and whether the result is the product with
    the K order inside each 8-wide k-step permuted (a core-matrix layout
    mistake) or only the hi parts multiplied (a split mistake)."""
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = A64 @ B64.T
    scale = np.abs(A64) @ np.abs(B64).T + 1e-30
    bad = np.abs(D - ref) > 1e-3 * scale
    notes = [f"bad entries {bad.sum()} of {bad.size}; rows {np.unique(np.nonzero(bad)[0])[:16]}; "
             f"cols {np.unique(np.nonzero(bad)[1])[:16]}",
             f"max relative error {np.max(np.abs(D - ref) / scale):.3e}"]
    k = A.shape[1]
    perm = np.arange(k).reshape(-1, 2, 4)[:, ::-1, :].reshape(-1)  # the two core matrices of a k-step swapped
    alt = A64 @ B64[:, perm].T
    notes.append(f"matches A B^T with swapped K core matrices of B: {np.allclose(D, alt, rtol=1e-4, atol=0)}")
    hi = lambda X: ((X.view(np.uint32) + np.uint32(0x1000)) & np.uint32(0xffffe000)).view(np.float32)
    notes.append(f"matches hi(A) hi(B)^T: {np.allclose(D, hi(A).astype(np.float64) @ hi(B).astype(np.float64).T, rtol=1e-5)}")
    notes.append(f"matches the transpose of a square result: {D.shape[0] == D.shape[1] and np.allclose(D, ref.T)}")
    return "; ".join(notes)


@pytest.mark.parametrize("m,n,k", [(128, 32, 32), (128, 16, 64), (256, 32, 256), (256, 16, 96)])
def test_tc_gemm_matches_fp64(dlr, m, n, k):
    import torch
    A, B = _operands(m, n, k, seed=m + n + k)
    Dg = dlr.tc_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    bound = 4 * (2.0 ** -20 + k * 2.0 ** -24) * scale
    assert np.all(np.abs(Dg - ref) <= bound + 1e-30), _diagnose(Dg, A, B)


def test_tc_gemm_split_beats_plain_tf32(dlr):
    # the three split products are far more accurate than one TF32 product:
    # the error stays below 2^-15 of the scale where plain TF32 reaches 2^-12
    import torch
    m, n, k = 128, 32, 128
    A, B = _operands(m, n, k, seed=7)
    Dg = dlr.tc_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    assert np.max(np.abs(Dg - ref) / scale) < 2.0 ** -15


def test_tc_gemm_rejects_bad_shapes(dlr):
    import torch
    A = torch.zeros(64, 32, device="cuda")
    B = torch.zeros(32, 32, device="cuda")
    with pytest.raises(dlr.DlrError):
        dlr.tc_gemm(A, B)
    A = torch.zeros(128, 40, device="cuda")
    B = torch.zeros(32, 40, device="cuda")
    with pytest.raises(dlr.DlrError):
        dlr.tc_gemm(A, B)
