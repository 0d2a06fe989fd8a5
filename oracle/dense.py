"""O2 (dense Strang-ordered MCWF) and O3 (dense Lindblad) for small chains.

TEST INFRASTRUCTURE ONLY (see the package docstring).

O2 runs the same step schedule, the same jump rule and the same random
numbers as O1 (oracle.mps_tjm), but on the full 2^L state vector with the
exact unitary exp(-i H0 dt).  With MPS bonds at full dimension, TDVP is exact,
so O1 must then reproduce O2 trajectory by trajectory (Thm. 1's full bond
dimension setting).

O3 integrates the Lindblad master equation (Eq. Lindblad) for the density
matrix; the trajectory average converges to it (Thm. 1, App. A).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp
from scipy.linalg import expm as _scipy_expm

from .philox import uniforms


def mpo_to_dense(W):
    """Contract an MPO [W_l (Dl, Dr, d, d)] into the dense d^L x d^L operator."""
    acc = W[0][0]                                  # (Dr, d, d): first site has Dl = 1
    for Wl in W[1:]:
        # acc[v, T, S] x Wl[v, u, t, s] -> acc[u, (T t), (S s)]
        acc = np.einsum('vTS,vuts->uTtSs', acc, Wl)
        u, a, b, c, e = acc.shape
        acc = acc.reshape(u, a * b, c * e)
    return acc[0]


def site_operator(op, site, L, d=2):
    """I x ... x op (at `site`, site 0 most significant) x ... x I."""
    out = np.ones((1, 1), dtype=np.complex128)
    for l in range(L):
        out = np.kron(out, op if l == site else np.eye(d))
    return out


def _operator(op, site, L, d=2):
    """A one-site (d x d) or nearest-neighbour two-site (d^2 x d^2, on site, site + 1) operator, dense."""
    op = np.asarray(op, dtype=np.complex128)
    if op.shape == (d, d):
        return site_operator(op, site, L, d)
    return np.kron(np.kron(np.eye(d ** site), op), np.eye(d ** (L - site - 2)))


def apply_site(op, psi, site, L, d=2):
    """Apply a d x d operator to one site of a dense state vector."""
    t = psi.reshape([d] * L)
    t = np.tensordot(op, t, axes=([1], [site]))
    t = np.moveaxis(t, 0, site)
    return t.reshape(-1)


def product_state(phis):
    psi = np.ones(1, dtype=np.complex128)
    for v in phis:
        v = np.asarray(v, dtype=np.complex128)
        psi = np.kron(psi, v / np.linalg.norm(v))
    return psi


class DenseStrang:
    """O2: the TJM step schedule on a dense vector (Eqs. TimeEvolutionFunctions, SimulationStep)."""

    def __init__(self, H, jumps, dt, L, d=2):
        self.L, self.d, self.dt = L, d, dt
        H = np.asarray(H, dtype=np.complex128)
        ev, V = np.linalg.eigh(H)
        self.U = (V * np.exp(-1j * dt * ev)) @ V.conj().T
        self.jumps = [(int(s), np.asarray(op, dtype=np.complex128), float(g)) for (s, op, g) in jumps]
        self.order = sorted(range(len(self.jumps)), key=lambda m: (self.jumps[m][0], m))

    def dissipator(self, site, tau):
        A = np.zeros((self.d, self.d), dtype=np.complex128)
        for (s, op, g) in self.jumps:
            if s == site:
                A += g * (op.conj().T @ op)
        return _scipy_expm(-0.5 * tau * A)

    def dj(self, psi, tau, u1, u2):
        """psi <- J_eps(D[tau] psi) with the same decision rule as O1."""
        for l in range(self.L):
            psi = apply_site(self.dissipator(l, tau), psi, l, self.L, self.d)
        norm2 = float(np.vdot(psi, psi).real)
        dp = 1.0 - norm2
        rec = {'dp': dp, 'margin1': abs(u1 - dp), 'jump': -1, 'margin2': math.inf}
        if not (u1 < dp):
            return psi / math.sqrt(norm2), rec
        w = []
        for m in self.order:
            s, op, g = self.jumps[m]
            phi = apply_site(op, psi, s, self.L, self.d)
            w.append(g * float(np.vdot(phi, phi).real))
        total, csum = 0.0, []
        for x in w:
            total += x
            csum.append(total)
        target = u2 * total
        pick = len(w) - 1
        for i, c in enumerate(csum):
            if target < c:
                pick = i
                break
        rec['margin2'] = min(abs(target - c) for c in csum) / total
        m = self.order[pick]
        rec['jump'] = m
        s, op, g = self.jumps[m]
        psi = math.sqrt(g) * apply_site(op, psi, s, self.L, self.d)
        return psi / np.linalg.norm(psi), rec

    def run(self, psi0, traj_id, seed, observables, n_steps, sample_steps, order=2):
        """order 2: the TJM schedule; order 1: Psi(j dt) = J(D[dt] U Psi((j-1) dt)) measured directly,
        the first-order baseline (same readings as O1's run_trajectory)."""
        psi = np.asarray(psi0, dtype=np.complex128)
        psi = psi / np.linalg.norm(psi)
        obs = [_operator(op, s, self.L, self.d) for (s, op) in observables]

        def meas(p):
            return np.array([np.vdot(p, O @ p).real for O in obs]) / float(np.vdot(p, p).real)

        want = set(sample_steps)
        vals, recs = {}, []
        if 0 in want:
            vals[0] = meas(psi)
        if order == 1:
            for j in range(1, n_steps + 1):
                u1, u2 = uniforms(seed, traj_id, j, 0)
                psi, r = self.dj(self.U @ psi, self.dt, u1, u2)
                recs.append(r)
                if j in want:
                    vals[j] = meas(psi)
            return np.array([vals[s] for s in sample_steps]), recs
        if n_steps > 0:
            u1, u2 = uniforms(seed, traj_id, 0, 0)
            psi, r = self.dj(psi, 0.5 * self.dt, u1, u2)
            recs.append(r)
        for j in range(1, n_steps + 1):
            psi = self.U @ psi
            if j in want:
                u1, u2 = uniforms(seed, traj_id, j, 1)
                X, r = self.dj(psi.copy(), 0.5 * self.dt, u1, u2)
                recs.append(r)
                vals[j] = meas(X)
            if j < n_steps:
                u1, u2 = uniforms(seed, traj_id, j, 0)
                psi, r = self.dj(psi, self.dt, u1, u2)
                recs.append(r)
        out = np.array([vals[s] for s in sample_steps])
        return out, recs


def lindblad_rhs(H, jumps_dense):
    """d rho/dt of Eq. Lindblad as a function on a flattened complex matrix."""
    n = H.shape[0]
    LdL = sum(g * (Lm.conj().T @ Lm) for (Lm, g) in jumps_dense) if jumps_dense else np.zeros_like(H)
    Heff = H - 0.5j * LdL

    def f(rho):
        r = rho.reshape(n, n)
        out = -1j * (Heff @ r - r @ Heff.conj().T)
        for (Lm, g) in jumps_dense:
            out = out + g * (Lm @ r @ Lm.conj().T)
        return out.reshape(-1)
    return f


def lindblad_evolve(H, jumps, L, rho0, times, d=2, rtol=1e-12, atol=1e-13):
    """O3: rho(t) at the requested times by an adaptive 8th-order Runge-Kutta integration."""
    H = np.asarray(H, dtype=np.complex128)
    jd = [(site_operator(np.asarray(op, dtype=np.complex128), s, L, d), float(g)) for (s, op, g) in jumps]
    f = lindblad_rhs(H, jd)
    n = H.shape[0]

    def real_f(t, y):
        z = f(y[:n * n] + 1j * y[n * n:])
        return np.concatenate([z.real, z.imag])

    r0 = np.asarray(rho0, dtype=np.complex128).reshape(-1)
    y0 = np.concatenate([r0.real, r0.imag])
    times = np.asarray(times, dtype=np.float64)
    sol = solve_ivp(real_f, (0.0, float(times[-1])), y0, method='DOP853', t_eval=times,
                    rtol=rtol, atol=atol)
    out = [(sol.y[:n * n, i] + 1j * sol.y[n * n:, i]).reshape(n, n) for i in range(len(times))]
    return out


def lindblad_steady_state(H, jumps, L, d=2):
    """O3 steady state: the trace-one solution of L(rho) = 0 (Eq. Lindblad with d rho/dt = 0).

    The Liouvillian is assembled as a sparse superoperator on row-major vec(rho)
    (vec(A rho B) = (A kron B^T) vec(rho)); one of its rows is replaced by the
    trace condition sum_i rho_ii = 1 and the linear system is solved directly.
    Assumes a unique steady state (as for the boundary-driven chain).
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    H = np.asarray(H, dtype=np.complex128)
    n = H.shape[0]
    jd = [(site_operator(np.asarray(op, dtype=np.complex128), s, L, d), float(g)) for (s, op, g) in jumps]
    LdL = sum(g * (Lm.conj().T @ Lm) for (Lm, g) in jd) if jd else np.zeros_like(H)
    Heff = sp.csr_matrix(H - 0.5j * LdL)
    Id = sp.identity(n, format='csr', dtype=np.complex128)
    # d rho/dt = -i (Heff rho - rho Heff^dag) + sum_m g L rho L^dag
    Lv = -1j * (sp.kron(Heff, Id) - sp.kron(Id, Heff.conj()))
    for (Lm, g) in jd:
        Ls = sp.csr_matrix(Lm)
        Lv = Lv + g * sp.kron(Ls, Ls.conj())
    A = Lv.tolil()
    A[0, :] = 0
    for i in range(n):
        A[0, i * n + i] = 1.0
    b = np.zeros(n * n, dtype=np.complex128)
    b[0] = 1.0
    return spl.spsolve(A.tocsc(), b).reshape(n, n)


def expect(rho, op, site, L, d=2):
    return float(np.trace(rho @ _operator(op, site, L, d)).real)
