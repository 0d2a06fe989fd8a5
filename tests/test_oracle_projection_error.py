"""Oracle pins for the projection error of 1TDVP (paper Sec. "Error measures",
eps = ||(I - P) H psi||).

* Neel product state |0101...>: H psi leaves the product-state tangent space only
  through the spin flips of X X + Y Y on each bond (2 J |..10..> per bond, all
  orthogonal), so eps = 2 |J| sqrt(L - 1) whatever the field g.
* |0...0> under the same H: X X + Y Y annihilates it, Z Z and X stay tangent: eps = 0.
* At full bond dimension the tangent space is the whole space: eps = 0 for a
  random MPS.
* The projector is orthogonal (P^2 = P = P^dag) and fixes every tangent vector of a
  random complex MPS -- the state with one site tensor replaced by an arbitrary
  tensor -- so a conjugated or transposed block projector fails it (eps of H = I,
  which is 0, does not see such a mistake).
"""
import math

import numpy as np

from oracle import mps_tjm as O1
from paper_2501_17913_gb300 import inputs as I


def test_neel_product_state_closed_form():
    for L, J, g in [(4, 1.0, 0.5), (6, 0.7, 0.0), (5, -1.0, 1.3)]:
        eps = O1.projection_error(O1.product_mps(I.neel(L)), I.xxx_mpo(L, J, g))
        assert abs(eps - 2 * abs(J) * math.sqrt(L - 1)) < 1e-12, (L, J, g, eps)


def test_all_zero_state_has_no_projection_error():
    eps = O1.projection_error(O1.product_mps(I.all_zero(5)), I.xxx_mpo(5, 1.0, 0.5))
    assert eps < 1e-12


def test_full_bond_dimension_has_no_projection_error():
    rng = np.random.default_rng(3)
    L = 6
    chi = [min(2 ** b, 2 ** (L - b)) for b in range(L + 1)]
    mps = [rng.standard_normal((chi[l], 2, chi[l + 1])) + 1j * rng.standard_normal((chi[l], 2, chi[l + 1]))
           for l in range(L)]
    assert O1.projection_error(mps, I.xxx_mpo(L, 1.0, 0.5)) < 1e-10


def test_truncated_state_has_error_and_identity_has_none():
    rng = np.random.default_rng(5)
    L = 6
    chi = [1, 2, 2, 2, 2, 2, 1]
    mps = [rng.standard_normal((chi[l], 2, chi[l + 1])) + 1j * rng.standard_normal((chi[l], 2, chi[l + 1]))
           for l in range(L)]
    assert O1.projection_error(mps, I.xxx_mpo(L, 1.0, 0.5)) > 1e-3
    # an MPO of the identity: H psi = psi lies in the tangent space
    Wid = [np.eye(2, dtype=complex).reshape(1, 1, 2, 2) for _ in range(L)]
    assert O1.projection_error(mps, Wid) < 1e-12


def test_projector_fixes_tangent_vectors_of_a_complex_state():
    rng = np.random.default_rng(8)
    L = 5
    chi = [1, 2, 3, 3, 2, 1]
    mps = [rng.standard_normal((chi[l], 2, chi[l + 1])) + 1j * rng.standard_normal((chi[l], 2, chi[l + 1]))
           for l in range(L)]
    P, psi = O1.tangent_projector(mps)
    assert np.abs(P @ P - P).max() < 1e-12 and np.abs(P - P.conj().T).max() < 1e-12
    assert np.abs(P @ psi - psi).max() < 1e-12
    for l in range(L):
        var = [m.copy() for m in mps]
        var[l] = rng.standard_normal(mps[l].shape) + 1j * rng.standard_normal(mps[l].shape)
        t = var[0]
        for M in var[1:]:
            t = np.tensordot(t, M, ([t.ndim - 1], [0]))
        t = t.reshape(-1)
        assert np.abs(P @ t - t).max() < 1e-10 * np.abs(t).max(), l
    # and the rank of P is the tangent-space dimension: sum_l chi_l d chi_{l+1} - sum_bonds chi^2
    dim = sum(chi[l] * 2 * chi[l + 1] for l in range(L)) - sum(chi[b] ** 2 for b in range(1, L))
    assert round(np.trace(P).real) == dim
