"""tjm_svd_noalloc: the SVD entry point that allocates nothing, for callers whose
own allocator owns all device memory or that cannot afford cudaMalloc/cudaFree.

It is called several times in a row through the C ABI on device buffers the
test owns (FP64 up to the workspace's 128 x 128 limit, FP32 and double-float),
and each result is checked against the allocating entry point
(tjm_selftest_svd) on the same input and precision.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2501_17913_gb300 import tjm

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


def _dev(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def test_noalloc_svd_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    lib = lib_ready()
    lib.tjm_svd_noalloc.restype = C.c_int
    lib.tjm_svd_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p]
    rng = np.random.default_rng(42)
    # one wide and one tall FP64 call back to back, the largest problem the static workspace holds
    # (128 x 128: the rotation accumulator and V fill it), and the FP32 and double-float instantiations
    shapes = [(64, 128, 1), (128, 64, 1), (128, 128, 1), (96, 128, 0), (128, 80, 2)]
    for call, (m, n, dp) in enumerate(shapes):
        A = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
        A[:, 3] = 0.0                        # a zero column as well
        nn = min(m, n)
        a = _dev(torch, np.stack([A.real, A.imag], -1))
        u = torch.zeros((m, nn, 2), dtype=torch.float64, device="cuda")
        s = torch.zeros((nn,), dtype=torch.float64, device="cuda")
        v = torch.zeros((n, nn, 2), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        st = lib.tjm_svd_noalloc(dp, m, n, a.data_ptr(), u.data_ptr(), s.data_ptr(), v.data_ptr(), stream)
        assert st == tjm.TJM_OK
        torch.cuda.synchronize()
        U = u.cpu().numpy()
        U = U[..., 0] + 1j * U[..., 1]
        V = v.cpu().numpy()
        V = V[..., 0] + 1j * V[..., 1]
        S = s.cpu().numpy()
        Ur, Sr, Vr = tjm.selftest_svd(A, dp)
        tol = {0: 2e-4, 1: 1e-12, 2: 1e-10}[dp]
        assert np.abs(S - Sr).max() < tol, call
        assert np.abs((U * S) @ V.conj().T - (Ur * Sr) @ Vr.conj().T).max() < tol, call
        assert np.abs((U * S) @ V.conj().T - A).max() < tol, call
        assert np.abs(U.conj().T @ U - np.eye(nn)).max() < tol, call
    # beyond the static workspace: rejected, nothing launched
    big = torch.zeros((129, 4, 2), dtype=torch.float64, device="cuda")
    assert lib.tjm_svd_noalloc(1, 129, 4, big.data_ptr(), big.data_ptr(), big.data_ptr(), big.data_ptr(),
                               None) == tjm.TJM_EINVAL
