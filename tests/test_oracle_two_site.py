"""Oracle pins for the two-site observables (paper Fig. 4b, <X_i X_{i+1}>) and the TFIM Hamiltonian
(Sec. "Benchmarking").

* local_expectations with a 4 x 4 operator on (i, i+1) equals the dense
  <psi| I..I (x) O (x) I..I |psi> of the contracted state vector, for a random
  non-canonical MPS (so no gauge assumption can hide an index mistake), and a
  product of two one-site operators equals the product of the one-site values
  on a product state.
* tfim_mpo contracts to -J sum Z Z - g sum X built from Kronecker products.
"""
import numpy as np

from oracle import dense as O2
from oracle import mps_tjm as O1
from paper_2501_17913_gb300 import inputs as I


def _dense(mps):
    psi = mps[0]
    for M in mps[1:]:
        psi = np.tensordot(psi, M, ([psi.ndim - 1], [0]))
    return psi.reshape(-1)


def _pair_operator(op4, site, L):
    return np.kron(np.kron(np.eye(2 ** site), op4), np.eye(2 ** (L - site - 2)))


def test_two_site_expectation_equals_dense():
    rng = np.random.default_rng(4)
    L, chi = 5, 3
    bonds = [1, 2, 3, 3, 2, 1]
    mps = [rng.standard_normal((bonds[l], 2, bonds[l + 1])) + 1j * rng.standard_normal((bonds[l], 2, bonds[l + 1]))
           for l in range(L)]
    psi = _dense(mps)
    A = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    ops = [(l, A) for l in range(L - 1)] + I.xx_observables(L) + [(2, I.Z)]
    vals, norm2 = O1.local_expectations(mps, ops)
    assert abs(norm2 - np.vdot(psi, psi).real) < 1e-10
    for (site, op), v in zip(ops, vals):
        op = np.asarray(op)
        full = _pair_operator(op, site, L) if op.shape == (4, 4) else O2.site_operator(op, site, L)
        assert abs(v - np.vdot(psi, full @ psi)) < 1e-10 * max(1.0, abs(v)), (site, op.shape)


def test_two_site_product_state_factorises():
    phis = I.haar_product(4, np.random.default_rng(2))
    mps = O1.product_mps(phis)
    x = O1.measure(mps, [(l, I.X) for l in range(4)])
    xx = O1.measure(mps, I.xx_observables(4))
    assert np.allclose(xx, x[:-1] * x[1:], atol=1e-13)


def test_tfim_mpo_equals_pauli_sum():
    L, J, g = 4, 1.3, 0.7
    H = np.zeros((2 ** L, 2 ** L), complex)
    for i in range(L - 1):
        H -= J * O2.site_operator(I.Z, i, L) @ O2.site_operator(I.Z, i + 1, L)
    for j in range(L):
        H -= g * O2.site_operator(I.X, j, L)
    assert np.allclose(O2.mpo_to_dense(I.tfim_mpo(L, J, g)), H, atol=1e-13)
