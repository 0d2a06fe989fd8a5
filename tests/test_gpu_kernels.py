"""Kernel-level parity of the CTA building blocks (through the C ABI self tests).

QR and SVD are checked through what defines them (orthonormal factors,
reconstruction, triangularity, singular values equal to LAPACK's), so the
gauge freedom of the factors does not matter.  Each runs in the three
factorization precisions: FP32 (dp=0), FP64 (dp=1) and double-float emulated
FP64 (dp=2), whose 48-bit significand must give FP64-class results.
"""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle.philox import uniforms
from paper_2501_17913_gb300 import tjm

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


def _rand(rng, m, n):
    return rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))


def _cases():
    rng = np.random.default_rng(0)
    out = [('square', _rand(rng, 8, 8)), ('tall', _rand(rng, 128, 64)), ('wide', _rand(rng, 64, 128)),
           ('tiny', _rand(rng, 2, 1)), ('max', _rand(rng, 128, 128)), ('odd', _rand(rng, 37, 13))]
    A = _rand(rng, 8, 8)
    A[1] = 0                                    # a zero row
    A[:, 3] = 0                                 # and a zero column
    out.append(('zero_rows_cols', A))
    B = _rand(rng, 16, 4) @ _rand(rng, 4, 12)   # rank 4
    out.append(('rank4', B))
    C = np.zeros((4, 4), complex)
    C[0, 0] = 1.0
    out.append(('rank1_unit', C))
    D = np.diag([3.0, 1.0, 1.0, 1e-7]).astype(complex)   # degenerate pair, tiny value
    out.append(('degenerate', D))
    return out


TOL = {0: 5e-5, 1: 1e-12, 2: 1e-11}


@pytest.mark.parametrize("dp", [1, 0, 2])
def test_qr_block(dp):
    lib_ready()
    tol = TOL[dp]
    for name, A in _cases():
        Q, R = tjm.selftest_qr(A, dp)
        k = min(A.shape)
        scale = max(1.0, np.abs(A).max())
        assert np.abs(Q.conj().T @ Q - np.eye(k)).max() < tol * 10, name
        assert np.abs(Q @ R - A).max() < tol * 10 * scale, name
        assert np.abs(np.tril(R, -1)).max() == 0.0, name


@pytest.mark.parametrize("dp", [1, 0, 2])
def test_svd_block(dp):
    lib_ready()
    tol = TOL[dp]
    for name, A in _cases():
        U, S, V = tjm.selftest_svd(A, dp)
        nn = min(A.shape)
        scale = max(1.0, np.abs(A).max())
        ref = np.linalg.svd(A, compute_uv=False)
        assert np.all(np.diff(S) <= 0), name
        assert np.abs(S - ref).max() < tol * 10 * scale, name
        assert np.abs(U.conj().T @ U - np.eye(nn)).max() < tol * 100, name
        assert np.abs(V.conj().T @ V - np.eye(nn)).max() < tol * 100, name
        assert np.abs((U * S) @ V.conj().T - A).max() < tol * 10 * scale, name


def test_expm_tridiagonal_block():
    lib_ready()
    rng = np.random.default_rng(3)
    for k in (1, 2, 5, 17, 30, 32):
        for theta in (-0.05, 0.05, -0.7, 2.5):
            a = rng.uniform(-30, 30, k)
            b = rng.uniform(0.1, 5, k - 1)
            T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
            ref = expm(1j * theta * T)[:, 0]
            c = tjm.selftest_expm_tridiag(a, b, theta)
            assert np.abs(c - ref).max() < 1e-12, (k, theta)


def test_philox_stream_bit_exact():
    lib_ready()
    rng = np.random.default_rng(1)
    traj = np.concatenate([np.arange(50), rng.integers(0, 2 ** 63, 50, dtype=np.uint64)]).astype(np.uint64)
    step = rng.integers(0, 2 ** 32, 100, dtype=np.uint64).astype(np.uint32)
    step[:20] = np.arange(20)
    branch = (np.arange(100) % 2).astype(np.uint32)
    for seed in (0, 7, 0xDEADBEEFCAFEF00D):
        u1, u2 = tjm.selftest_philox(seed, traj, step, branch)
        for i in range(100):
            r1, r2 = uniforms(seed, int(traj[i]), int(step[i]), int(branch[i]))
            assert u1[i] == r1 and u2[i] == r2, i


def test_svd_rank_deficient_after_projection():
    """Rank-deficient inputs whose null directions hold only rounding noise (as after a sigma^- jump)
    must still give orthonormal factors: the noise columns may not be driven into denormals."""
    lib_ready()
    rng = np.random.default_rng(5)
    for (m, n, r) in [(8, 8, 4), (16, 16, 3), (64, 128, 20), (128, 128, 64), (32, 8, 2)]:
        Qa, _ = np.linalg.qr(_rand(rng, m, m))
        Qb, _ = np.linalg.qr(_rand(rng, n, n))
        s = np.sort(rng.uniform(0.01, 1.0, r))[::-1]
        A = (Qa[:, :r] * s) @ Qb[:, :r].conj().T          # exact rank r, noise in the null space
        for dp in (1, 0, 2):
            U, S, V = tjm.selftest_svd(A, dp)
            nn = min(m, n)
            tol = TOL[dp]
            assert np.abs(U.conj().T @ U - np.eye(nn)).max() < 100 * tol, (m, n, r, dp)
            assert np.abs(V.conj().T @ V - np.eye(nn)).max() < 100 * tol, (m, n, r, dp)
            assert np.abs((U * S) @ V.conj().T - A).max() < 100 * tol, (m, n, r, dp)
            assert np.abs(S[:r] - s).max() < 10 * tol, (m, n, r, dp)


def test_qr_rank_deficient_noise_columns():
    """A column that vanishes up to rounding must not produce an overflowing reflector (FP32 and FP64)."""
    lib_ready()
    rng = np.random.default_rng(9)
    for (m, n, r) in [(8, 7, 6), (16, 8, 3), (128, 64, 40), (64, 64, 1)]:
        Qa, _ = np.linalg.qr(_rand(rng, m, m))
        Qb, _ = np.linalg.qr(_rand(rng, n, n))
        A = (Qa[:, :r] * rng.uniform(0.1, 1.0, r)) @ Qb[:, :r].conj().T
        for dp in (1, 0, 2):
            Q, R = tjm.selftest_qr(A, dp)
            tol = TOL[dp]
            k = min(m, n)
            assert np.isfinite(Q).all() and np.isfinite(R).all()
            assert np.abs(Q.conj().T @ Q - np.eye(k)).max() < 100 * tol, (m, n, r, dp)
            assert np.abs(Q @ R - A).max() < 100 * tol, (m, n, r, dp)


def test_emulated_fp64_factorizations_equal_native_fp64():
    """Double-float QR and SVD give the native FP64 results (singular values, the projector U U^H,
    R up to the column phases of Q) on the factorization shapes of the sweeps, to ~1e-11 relative:
    the 48-bit significand (2^-48 = 3.6e-15 per operation) over O(10^3) operations per entry."""
    lib_ready()
    rng = np.random.default_rng(11)
    for (m, n) in [(128, 64), (64, 128), (128, 128), (32, 16)]:
        A = _rand(rng, m, n) / np.sqrt(n)
        U1, S1, V1 = tjm.selftest_svd(A, 1)
        U2, S2, V2 = tjm.selftest_svd(A, 2)
        assert np.abs(S1 - S2).max() < 1e-11 * S1[0], (m, n)
        r = min(m, n) // 2
        assert np.abs(U1[:, :r] @ U1[:, :r].conj().T - U2[:, :r] @ U2[:, :r].conj().T).max() < 1e-10, (m, n)
        Q1, R1 = tjm.selftest_qr(A, 1)
        Q2, R2 = tjm.selftest_qr(A, 2)
        assert np.abs(np.abs(R1) - np.abs(R2)).max() < 1e-11 * np.abs(R1).max(), (m, n)
        assert np.abs(Q1 @ R1 - Q2 @ R2).max() < 1e-11, (m, n)
