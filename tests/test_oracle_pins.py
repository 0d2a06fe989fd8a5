"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests uses the CUDA library.  Each one checks the oracle against
something other than itself: a library routine on a special case, a closed
form, an exactly solvable limit, an invariant, or an independent dense
computation.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

from oracle import dense as O2
from oracle import mps_tjm as O1
from oracle.philox import philox4x32_10, u53, uniforms
from paper_2501_17913_gb300 import inputs as I


# ---------------------------------------------------------------- Philox
def _curand():
    candidates = ["/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")]
    for path in candidates:
        if not path:
            continue
        try:
            return ctypes.CDLL(path)
        except OSError:
            pass
    return None


@pytest.mark.parametrize("seed", [0, 0x123456789ABCDEF0, 20250130])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox4_32_10 (a library) fills block i from counter (i // 65536, 0, i % 65536, 0)."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0   # CURAND_RNG_PSEUDO_PHILOX4_32_10
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    n_blocks = 131072
    out = np.zeros(4 * n_blocks, dtype=np.uint32)
    assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    lib.curandDestroyGenerator(gen)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in list(range(0, 70)) + list(range(65530, 65600)) + [131071]:
        ctr = (i // 65536, 0, i % 65536, 0)
        assert philox4x32_10(ctr, key) == [int(x) for x in out[4 * i:4 * i + 4]], i


def test_u53_range_and_resolution():
    assert u53(0, 0) == 0.0
    top = u53(0xFFFFFFFF, 0xFFFFFFFF)
    assert top < 1.0 and 1.0 - top == 2.0 ** -53
    us = [uniforms(7, t, s, b)[0] for t in range(20) for s in range(10) for b in range(2)]
    assert all(0.0 <= u < 1.0 for u in us)
    assert abs(np.mean(us) - 0.5) < 0.05


# ---------------------------------------------------------------- model inputs
def _kron_chain(ops):
    out = np.ones((1, 1), dtype=np.complex128)
    for o in ops:
        out = np.kron(out, o)
    return out


def _xxx_dense(L, J, g):
    """H = J sum (XX + YY + ZZ) + g sum X written out with Kronecker products."""
    H = np.zeros((2 ** L, 2 ** L), dtype=np.complex128)
    for i in range(L - 1):
        for P in (I.X, I.Y, I.Z):
            ops = [I.I2] * L
            ops[i] = P
            ops[i + 1] = P
            H += J * _kron_chain(ops)
    for i in range(L):
        ops = [I.I2] * L
        ops[i] = I.X
        H += g * _kron_chain(ops)
    return H


@pytest.mark.parametrize("L,J,g", [(2, 1.0, 0.5), (4, 0.7, -0.3), (5, 1.0, 0.5)])
def test_mpo_equals_pauli_sum(L, J, g):
    assert np.allclose(O2.mpo_to_dense(I.xxx_mpo(L, J, g)), _xxx_dense(L, J, g), atol=1e-13)


def test_dissipator_closed_form():
    """sigma^- and Z at rates g1, g2: D = diag(e^{-g2 tau/2}, e^{-(g1+g2) tau/2})."""
    g1, g2, tau = 0.3, 0.17, 0.05
    prob = O1.Problem(I.xxx_mpo(3), [(1, I.SM, g1), (1, I.Z, g2), (0, I.Z, g2)], 0.1, 4)
    D = O1.dissipator_site(prob, 1, tau)
    assert np.allclose(D, np.diag([math.exp(-g2 * tau / 2), math.exp(-(g1 + g2) * tau / 2)]), atol=1e-15)
    D2 = O1.dissipator_site(prob, 2, tau)
    assert np.allclose(D2, np.eye(2), atol=1e-15)


# ---------------------------------------------------------------- Lanczos
@pytest.mark.parametrize("n,coef", [(40, -0.3j), (64, +0.05j), (7, -2.0j)])
def test_lanczos_matches_dense_expm(n, coef):
    from scipy.linalg import expm
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = (A + A.conj().T) / 2
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y, k = O1.expm_lanczos(lambda x: H @ x, v, coef, 1e-13, 60)
    ref = expm(coef * H) @ v
    assert np.linalg.norm(y - ref) < 1e-10 * np.linalg.norm(v)
    assert 1 <= k <= 60


def test_lanczos_breakdown_cases():
    v = np.array([1.0, 2.0j, -1.0])
    y, k = O1.expm_lanczos(lambda x: 0 * x, v, -0.7j, 1e-12, 30)
    assert k == 1 and np.allclose(y, v)
    # v an eigenvector: one matvec, exact phase
    H = np.diag([1.0, 2.0, 3.0])
    e = np.array([0, 1.0 + 0j, 0])
    y, k = O1.expm_lanczos(lambda x: H @ x, e, -0.4j, 1e-12, 30)
    assert k == 1 and np.allclose(y, np.exp(-0.8j) * e, atol=1e-14)


def test_trunc_rank_rule():
    prob = O1.Problem(I.xxx_mpo(3), [], 0.1, chi_max=10, trunc_eps=1e-4)
    S = np.array([1.0, 0.5, 1e-2, 5e-3, 1e-3])
    total = np.sum(S ** 2)
    r = O1.trunc_rank(S, prob)
    assert np.sum(S[r:] ** 2) <= 1e-4 * total < np.sum(S[r - 1:] ** 2)
    assert r == 3
    prob.chi_max = 2
    assert O1.trunc_rank(S, prob) == 2
    prob.chi_max, prob.trunc_eps = 10, 0.0
    assert O1.trunc_rank(np.array([1.0, 0.1, 0.0]), prob) == 2
    prob.exact = True
    assert O1.trunc_rank(np.array([1.0, 0.1, 0.0]), prob) == 3
    prob.exact, prob.trunc_eps = False, 0.99
    assert O1.trunc_rank(S, prob) == 1


# ---------------------------------------------------------------- environments / H_eff
def _random_mps(L, chis, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((chis[l], 2, chis[l + 1])) + 1j * rng.standard_normal((chis[l], 2, chis[l + 1]))
            for l in range(L)]


def _left_states(mps, upto):
    """Dense vectors of the left block basis (sites 0..upto-1): shape (2^upto, chi)."""
    acc = np.ones((1, 1), dtype=np.complex128)
    for l in range(upto):
        a, d, b = mps[l].shape
        acc = np.einsum('Pa,asb->Psb', acc, mps[l]).reshape(-1, b)
    return acc


def _right_states(mps, frm):
    """Dense vectors of the right block basis (sites frm..L-1): shape (chi, 2^(L-frm))."""
    acc = np.ones((1, 1), dtype=np.complex128)
    for l in range(len(mps) - 1, frm - 1, -1):
        a, d, b = mps[l].shape
        acc = np.einsum('asb,bP->asP', mps[l], acc).reshape(a, -1)
    return acc


def test_heff_matches_projected_dense_hamiltonian():
    """H_eff built from environments equals P^dag H P for the local isometry P (Sec. 1TDVP)."""
    L = 5
    W = I.xxx_mpo(L, 0.9, 0.4)
    H = O2.mpo_to_dense(W)
    mps = _random_mps(L, [1, 2, 4, 4, 2, 1], 3)
    c = 2   # orthogonality centre
    for l in range(c):
        O1.qr_move_right(mps, l)
    for l in range(L - 1, c, -1):
        O1.rq_move_left(mps, l)
    sw = O1.Sweeper(O1.Problem(W, [], 0.1, 8))
    for l in range(c):
        sw.Lenv[l + 1] = O1.env_left_update(sw.Lenv[l], mps[l], W[l])
    sw.build_right_envs(mps)
    Lb, Rb = _left_states(mps, c), _right_states(mps, c + 1)
    assert np.allclose(Lb.conj().T @ Lb, np.eye(Lb.shape[1]), atol=1e-12)
    assert np.allclose(Rb @ Rb.conj().T, np.eye(Rb.shape[0]), atol=1e-12)
    # one site
    shape = mps[c].shape
    P = np.einsum('Pa,st,bQ->PtQasb', Lb, np.eye(2), Rb).reshape(2 ** L, -1)
    Hd = P.conj().T @ H @ P
    n = int(np.prod(shape))
    He = np.stack([O1.heff1(sw.Lenv[c], W[c], sw.Renv[c + 1], np.eye(n)[k].reshape(shape)).reshape(-1)
                   for k in range(n)], axis=1)
    assert np.allclose(He, Hd, atol=1e-12)
    # two sites (c, c+1)
    Rb2 = _right_states(mps, c + 2)
    sh2 = (shape[0], 2, 2, mps[c + 1].shape[2])
    P2 = np.einsum('Pa,st,uv,bQ->PtvQasub', Lb, np.eye(2), np.eye(2), Rb2).reshape(2 ** L, -1)
    Hd2 = P2.conj().T @ H @ P2
    n2 = int(np.prod(sh2))
    He2 = np.stack([O1.heff2(sw.Lenv[c], W[c], W[c + 1], sw.Renv[c + 2], np.eye(n2)[k].reshape(sh2)).reshape(-1)
                    for k in range(n2)], axis=1)
    assert np.allclose(He2, Hd2, atol=1e-12)
    # bond between c and c+1: move the centre right first
    O1.qr_move_right(mps, c)
    sw.Lenv[c + 1] = O1.env_left_update(sw.Lenv[c], mps[c], W[c])
    Lb1 = _left_states(mps, c + 1)
    chb = Lb1.shape[1]
    P0 = np.einsum('Pa,bQ->PQab', Lb1, Rb).reshape(2 ** L, -1)
    Hd0 = P0.conj().T @ H @ P0
    He0 = np.stack([O1.heff0(sw.Lenv[c + 1], sw.Renv[c + 1], np.eye(chb * Rb.shape[0])[k].reshape(chb, -1)).reshape(-1)
                    for k in range(chb * Rb.shape[0])], axis=1)
    assert np.allclose(He0, Hd0, atol=1e-12)


def _energy(mps, H):
    psi = _left_states(mps, len(mps))[:, 0]
    return float(np.vdot(psi, H @ psi).real / np.vdot(psi, psi).real), float(np.vdot(psi, psi).real)


def test_one_site_tdvp_conserves_norm_and_energy():
    """1TDVP on a fixed manifold conserves norm and energy (Methods, Sec. TDVP overview)."""
    L = 6
    W = I.xxx_mpo(L, 1.0, 0.5)
    H = O2.mpo_to_dense(W)
    mps = _random_mps(L, [1, 2, 3, 3, 3, 2, 1], 11)
    for l in range(L - 1, 0, -1):
        O1.rq_move_left(mps, l)
    mps[0] /= np.linalg.norm(mps[0])
    prob = O1.Problem(W, [], 0.1, chi_max=2)    # every bond >= 2: one-site everywhere
    sw = O1.Sweeper(prob)
    sw.build_right_envs(mps)
    e0, n0 = _energy(mps, H)
    for _ in range(3):
        sw.sweep(mps, 0.05)
        sw.build_right_envs(mps)
    e1, n1 = _energy(mps, H)
    assert sw.updates['two_site'] == 0 and sw.updates['one_site'] == 3 * 2 * L
    assert abs(n1 - 1.0) < 1e-11
    assert abs(e1 - e0) < 1e-10


def _prepared(L, bonds, seed):
    mps = _random_mps(L, bonds, seed)
    for l in range(L - 1, 0, -1):
        O1.rq_move_left(mps, l)
    mps[0] /= np.linalg.norm(mps[0])
    return mps


def test_dynamic_tdvp_switch_is_per_bond_and_exact_without_truncation():
    """The dynamic switch of Sec. "Dynamic TDVP": a two-site update exactly where the bond is below
    chi_max, a one-site update elsewhere.  Bonds [1, 2, 4, 4, 4, 2, 1] at chi_max = 4: the two edge
    bonds are below chi_max but already at full rank (2), so each sweep makes 2 two-site and 3
    one-site updates per half sweep, none truncates, and every substep is the exponential of a
    Hermitian effective operator or an exact refactorization: norm and energy are conserved to the
    Lanczos accuracy.  Testing `<=` instead of `<` would make every update two-site and truncate."""
    L = 6
    W = I.xxx_mpo(L, 1.0, 0.5)
    H = O2.mpo_to_dense(W)
    mps = _prepared(L, [1, 2, 4, 4, 4, 2, 1], 13)
    prob = O1.Problem(W, [], 0.1, chi_max=4)
    sw = O1.Sweeper(prob)
    sw.build_right_envs(mps)
    e0, _ = _energy(mps, H)
    for _ in range(3):
        sw.sweep(mps, 0.05)
        sw.build_right_envs(mps)
    e1, n1 = _energy(mps, H)
    assert sw.updates == {'two_site': 3 * 4, 'one_site': 3 * 6}, sw.updates
    assert [m.shape[2] for m in mps] == [2, 4, 4, 4, 2, 1]
    assert abs(n1 - 1.0) < 1e-11
    assert abs(e1 - e0) < 1e-10


def test_dynamic_tdvp_bonds_grow_to_chi_max_without_truncation():
    """From bonds of 2 everywhere with chi_max = 4, the left-to-right half sweep is two-site at all
    five bonds; a two-site block between two bonds of 2 has rank <= 4, so the interior bonds grow
    to 4 (generic state) without any truncation.  The switch is taken when the sweep reaches a
    bond, so the right-to-left half sweep finds the three interior bonds at chi_max (one-site) and
    the two full-rank edge bonds at 2 (two-site).  Norm and energy are conserved.  Keeping the old
    bond dimension, or truncating below chi_max, would leave the bonds at 2 or change the energy."""
    L = 6
    W = I.xxx_mpo(L, 1.0, 0.5)
    H = O2.mpo_to_dense(W)
    mps = _prepared(L, [1, 2, 2, 2, 2, 2, 1], 17)
    prob = O1.Problem(W, [], 0.1, chi_max=4)
    sw = O1.Sweeper(prob)
    sw.build_right_envs(mps)
    e0, _ = _energy(mps, H)
    sw.sweep(mps, 0.05)
    sw.build_right_envs(mps)
    e1, n1 = _energy(mps, H)
    bonds = [m.shape[2] for m in mps[:-1]]
    assert sw.updates == {'two_site': 5 + 2, 'one_site': 3}, sw.updates
    assert bonds[0] == 2 and bonds[-1] == 2 and max(bonds) == 4 and all(b <= 4 for b in bonds), bonds
    assert abs(n1 - 1.0) < 1e-11
    assert abs(e1 - e0) < 1e-10


def test_padded_product_state_is_right_canonical_and_exact():
    phis = I.haar_product(5, np.random.default_rng(4))
    mps = O1.padded_product_mps(phis)
    assert [m.shape[2] for m in mps[:-1]] == [2, 4, 4, 2]
    for l in range(1, 5):
        a, d, b = mps[l].shape
        M = mps[l].reshape(a, d * b)
        assert np.allclose(M @ M.conj().T, np.eye(a), atol=1e-12)
    psi = _left_states(mps, 5)[:, 0]
    assert np.allclose(psi, O2.product_state(phis), atol=1e-12)


# ---------------------------------------------------------------- exact mode: O1 == O2
@pytest.mark.parametrize("chi_max,expect", [(16, 'two'), (2, 'one'), (4, 'mixed')])
def test_exact_mode_mps_tjm_equals_dense_strang_mcwf(chi_max, expect):
    """With bonds at full dimension TDVP is exact, so O1 must equal O2 per trajectory (Thm. 1 setting)."""
    L, n = 5, 8
    W = I.xxx_mpo(L, 1.0, 0.5)
    jumps = I.noise(L, 0.2, 0.1)
    phis = I.neel(L)
    obs = I.z_observables(L) + [(2, I.X)]
    prob = O1.Problem(W, jumps, 0.1, chi_max, 0.0, exact=True)
    ds = O2.DenseStrang(O2.mpo_to_dense(W), jumps, 0.1, L)
    for traj in range(3):
        v1, st = O1.run_trajectory(prob, O1.padded_product_mps(phis), traj, 5, obs, n, range(n + 1))
        v2, recs = ds.run(O2.product_state(phis), traj, 5, obs, n, range(n + 1))
        assert np.abs(v1 - v2).max() < 1e-10
        assert [r['jump'] for r in st['records']] == [r['jump'] for r in recs]
        up = st['updates']
        assert {'two': up['one_site'] == 0, 'one': up['two_site'] == 0,
                'mixed': up['one_site'] > 0 and up['two_site'] > 0}[expect]


# ---------------------------------------------------------------- H = 0: exactly solvable jump chain
def _basis_chain(L, bits, g_relax, g_deph, dt, n, seed, traj):
    """Trajectory of a computational basis state under H = 0 with sigma^- and Z noise, by hand.

    D[tau] scales a basis state with k excited sites by exp(-(k g_relax + L g_deph) tau / 2),
    so dp = 1 - exp(-(k g_relax + L g_deph) tau); a jump picks, in site-major
    order, sigma^- on an excited site (weight g_relax) or Z on any site (g_deph).
    """
    bits = list(bits)

    def dj(bits, tau, u1, u2):
        k = sum(bits)
        dp = 1.0 - math.exp(-(k * g_relax + L * g_deph) * tau)
        if not (u1 < dp):
            return bits
        w = []
        for l in range(L):
            w.append(('m', l, g_relax * bits[l]))
            w.append(('z', l, g_deph))
        total = sum(x[2] for x in w)
        acc = 0.0
        for kind, l, x in w:
            acc += x
            if u2 * total < acc:
                if kind == 'm':
                    bits = bits.copy()
                    bits[l] = 0
                return bits
        return bits

    out = [[1.0 - 2 * b for b in bits]]
    bits = dj(bits, dt / 2, *uniforms(seed, traj, 0, 0))
    for j in range(1, n + 1):
        X = dj(bits, dt / 2, *uniforms(seed, traj, j, 1))
        out.append([1.0 - 2 * b for b in X])
        if j < n:
            bits = dj(bits, dt, *uniforms(seed, traj, j, 0))
    return np.array(out)


def test_zero_hamiltonian_jump_chain_per_trajectory():
    L, n, dt = 6, 30, 0.2
    W = I.xxx_mpo(L, 0.0, 0.0)
    jumps = []
    for l in range(L):
        jumps.append((l, I.SM, 0.4))
        jumps.append((l, I.Z, 0.1))
    prob = O1.Problem(W, jumps, dt, 4, 1e-10)
    bits = [1, 1, 0, 1, 1, 1]
    phis = [np.array([1.0 - b, b], dtype=complex) for b in bits]
    for traj in range(6):
        v, st = O1.run_trajectory(prob, O1.product_mps(phis), traj, 3, I.z_observables(L), n, range(n + 1))
        ref = _basis_chain(L, bits, 0.4, 0.1, dt, n, 3, traj)
        assert np.abs(v - ref).max() < 1e-12
        assert st['matvecs']['heff1'] + st['matvecs']['heff2'] + st['matvecs']['heff0'] > 0


def test_dephasing_flips_x_per_trajectory():
    """H = 0, Z noise only, |+>^L: each Z jump flips <X> on its site; dp = 1 - exp(-L gamma tau)."""
    L, n, dt, g = 4, 20, 0.3, 0.25
    W = I.xxx_mpo(L, 0.0, 0.0)
    jumps = [(l, I.Z, g) for l in range(L)]
    prob = O1.Problem(W, jumps, dt, 4, 1e-10)
    plus = [np.array([1.0, 1.0]) / math.sqrt(2)] * L
    obs = [(l, I.X) for l in range(L)]
    for traj in range(4):
        v, st = O1.run_trajectory(prob, O1.product_mps(plus), traj, 1, obs, n, range(n + 1))
        signs = np.ones(L)
        ref = [signs.copy()]

        def dj(signs, tau, u1, u2):
            if u1 < 1.0 - math.exp(-L * g * tau):
                s = signs.copy()
                s[min(int(u2 * L), L - 1)] *= -1
                return s
            return signs
        signs = dj(signs, dt / 2, *uniforms(1, traj, 0, 0))
        for j in range(1, n + 1):
            ref.append(dj(signs, dt / 2, *uniforms(1, traj, j, 1)))
            if j < n:
                signs = dj(signs, dt, *uniforms(1, traj, j, 0))
        assert np.abs(v - np.array(ref)).max() < 1e-12


# ---------------------------------------------------------------- O2 and O3 pins
def test_dense_unitary_and_conservation_laws():
    from scipy.linalg import expm
    L = 4
    H = _xxx_dense(L, 1.0, 0.0)
    ds = O2.DenseStrang(H, [], 0.1, L)
    assert np.allclose(ds.U, expm(-0.1j * H), atol=1e-12)
    psi = O2.product_state(I.neel(L))
    Ztot = sum(O2.site_operator(I.Z, l, L) for l in range(L))
    e0, m0 = np.vdot(psi, H @ psi).real, np.vdot(psi, Ztot @ psi).real
    for _ in range(20):
        psi = ds.U @ psi
    assert abs(np.linalg.norm(psi) - 1) < 1e-12
    assert abs(np.vdot(psi, H @ psi).real - e0) < 1e-11
    assert abs(np.vdot(psi, Ztot @ psi).real - m0) < 1e-11


def _liouvillian(H, jumps_dense):
    """Column-stacking vectorisation: vec(A rho B) = (B^T kron A) vec(rho)."""
    n = H.shape[0]
    Id = np.eye(n)
    Lv = -1j * (np.kron(Id, H) - np.kron(H.T, Id))
    for (Lm, g) in jumps_dense:
        LdL = Lm.conj().T @ Lm
        Lv += g * (np.kron(Lm.conj(), Lm) - 0.5 * np.kron(Id, LdL) - 0.5 * np.kron(LdL.T, Id))
    return Lv


def test_lindblad_integrator_against_liouvillian_exponential():
    from scipy.linalg import expm
    L = 2
    H = _xxx_dense(L, 1.0, 0.5)
    jumps = I.noise(L, 0.3, 0.2)
    jd = [(O2.site_operator(op, s, L), g) for (s, op, g) in jumps]
    psi = O2.product_state([np.array([0.6, 0.8j]), np.array([1.0, 0.0])])
    rho0 = np.outer(psi, psi.conj())
    times = [0.0, 0.5, 1.3, 2.0]
    rhos = O2.lindblad_evolve(H, jumps, L, rho0, times)
    Lv = _liouvillian(H, jd)
    for t, r in zip(times, rhos):
        ref = (expm(t * Lv) @ rho0.reshape(-1, order='F')).reshape(4, 4, order='F')
        assert np.allclose(r, ref, atol=1e-10)
        assert abs(np.trace(r) - 1) < 1e-11
        assert np.allclose(r, r.conj().T, atol=1e-12)
        assert np.linalg.eigvalsh((r + r.conj().T) / 2).min() > -1e-11


def test_lindblad_pure_relaxation_closed_form():
    """H = 0, sigma^- at rate g: <Z>(t) = 1 - 2 p1(0) exp(-g t); steady state |0..0>."""
    L, g = 3, 0.7
    H = np.zeros((8, 8), dtype=complex)
    jumps = [(l, I.SM, g) for l in range(L)]
    p1 = [0.2, 1.0, 0.55]
    phis = [np.array([math.sqrt(1 - p), math.sqrt(p)]) for p in p1]
    psi = O2.product_state(phis)
    times = [0.0, 0.4, 1.5, 30.0]
    rhos = O2.lindblad_evolve(H, jumps, L, np.outer(psi, psi.conj()), times)
    for t, r in zip(times, rhos):
        for l in range(L):
            assert abs(O2.expect(r, I.Z, l, L) - (1 - 2 * p1[l] * math.exp(-g * t))) < 1e-10
    assert abs(rhos[-1][0, 0].real - 1.0) < 1e-8


# ---------------------------------------------------------------- energy shift (a global phase)
def _shifted_mpo(W, c):
    """The MPO with -c*I added to every site's on-site entry (row 0, last column): H - c*L*I."""
    out = []
    for l, w in enumerate(W):
        w = np.array(w, dtype=np.complex128)
        w[0, w.shape[1] - 1] -= c * np.eye(2)
        out.append(w)
    return out


def test_energy_shift_changes_only_the_global_phase():
    """The kernels may evolve with H - E*I (E per trajectory); in the method this is a global phase.

    First the finite-state MPO with -c on every on-site channel is H - c*L*I (dense check); then
    whole truncated TJM trajectories (dynamic TDVP, dissipation, jumps, sampling) with H and with
    the shifted MPO give the same observables."""
    L, c = 5, 0.37
    W = I.xxx_mpo(L, 1.0, 0.5)
    Ws = _shifted_mpo(W, c)
    assert np.allclose(O2.mpo_to_dense(Ws), O2.mpo_to_dense(W) - c * L * np.eye(2 ** L), atol=1e-13)
    jumps, obs = I.noise(L, 0.2, 0.1), I.z_observables(L) + [(2, I.X)]
    for traj in range(4):
        vals = []
        for WW in (W, Ws):
            prob = O1.Problem(WW, jumps, 0.1, 4, 1e-10)
            v, st = O1.run_trajectory(prob, O1.product_mps(I.neel(L)), traj, 7, obs, 8, list(range(9)))
            vals.append(v)
        assert np.abs(vals[0] - vals[1]).max() < 1e-10, traj


# ---------------------------------------------------------------- truncated TDVP converges with chi
def test_truncated_dynamic_tdvp_converges_to_the_exact_evolution():
    """Below full bond dimension the TDVP projection error has no closed form, but it must vanish as
    chi_max grows: with no noise (pure Hamiltonian evolution from Neel, L = 8) the oracle's
    observables approach the dense exp(-iH t) evolution monotonically in chi_max (full dimension at
    the centre bond is 16; the exact-mode test covers padded full bonds at 1e-10)."""
    L, n = 8, 6
    W = I.xxx_mpo(L, 1.0, 0.5)
    jumps = I.noise(L, 0.0, 0.0)
    phis = I.neel(L)
    obs = I.z_observables(L) + [(3, I.X)]
    ds = O2.DenseStrang(O2.mpo_to_dense(W), jumps, 0.1, L)
    exact, _ = ds.run(O2.product_state(phis), 0, 5, obs, n, range(n + 1))
    errs = []
    for chi in (2, 4, 8, 16):
        prob = O1.Problem(W, jumps, 0.1, chi, 1e-14)
        v, _ = O1.run_trajectory(prob, O1.product_mps(phis), 0, 5, obs, n, range(n + 1))
        errs.append(float(np.abs(v - exact).max()))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[0] > 1e-2 and errs[-1] < 2e-3, errs
