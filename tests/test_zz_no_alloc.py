"""The allocation-free eigensolver entry point (osv_syev_batched_noalloc), called through the C ABI, agrees
with osv_syev_batched on two calls in a row.  It serves callers that cannot call cudaMalloc (code under an
external allocator that owns the device memory, or that cannot take cudaFree's device-wide synchronisation).
Collected last on purpose: a stop-at-first-failure run has run every other test before this one."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2106_06149_gb300 import build, osvmbe
    build.build()
    return osvmbe.load()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _call(fn, A):
    b, n, _ = A.shape
    w = torch.full((b, n), float("nan"), dtype=torch.float64, device=A.device)
    Zt = torch.full((b, n, n), float("nan"), dtype=torch.float64, device=A.device)
    st = fn(_p(A), n, b, _p(w), _p(Zt), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, w.cpu().numpy(), Zt.cpu().numpy()


def _check_same(A, w0, Z0, w1, Z1):
    for b in range(A.shape[0]):
        scale = np.abs(w0[b]).max()
        assert np.allclose(w1[b], w0[b], rtol=0, atol=1e-12 * scale)
        # eigenvectors agree up to sign (the eigenvalues of these random matrices are simple)
        ov = np.abs(np.sum(Z0[b] * Z1[b], axis=1))
        assert np.abs(ov - 1.0).max() <= 1e-9
        n = A.shape[1]
        Z = Z1[b].T
        assert np.abs(A[b] @ Z - Z * w1[b][None, :]).max() <= 1e-12 * scale * n


def test_noalloc_matches_allocating_entry_point_twice(lib):
    from paper_2106_06149_gb300 import osvmbe
    rng = np.random.default_rng(7)
    for (batch, n) in ((3, 200), (9, 64)):       # two calls in a row, different shapes
        X = rng.standard_normal((batch, n, n))
        A = X + X.transpose(0, 2, 1)
        Ad = torch.from_numpy(A).cuda()
        st0, w0, Z0 = _call(lib.osv_syev_batched, Ad)
        st1, w1, Z1 = _call(lib.osv_syev_batched_noalloc, Ad)
        assert st0 == osvmbe.OSV_OK and st1 == osvmbe.OSV_OK
        _check_same(A, w0, Z0, w1, Z1)
    # the input is read only
    assert torch.equal(Ad.cpu(), torch.from_numpy(A))


def test_noalloc_rejects_requests_beyond_its_static_scratch(lib):
    from paper_2106_06149_gb300 import osvmbe
    A = torch.zeros(1, 1, 1, dtype=torch.float64, device="cuda")
    w = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.osv_syev_batched_noalloc(_p(A), 1100, 1, _p(w), _p(A), None)   # 1100^2 > 2^20 doubles
    assert st == osvmbe.OSV_ERR_INVALID
    assert b"exceeds the static scratch" in lib.osv_last_error(None)
