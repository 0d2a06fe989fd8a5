"""Oracle pins for the boundary-driven XXX chain (paper Sec. "Validating convergence against
analytical results", Fig. edge-driven XXX).

* The steady state found by solving L(rho) = 0 equals the long-time limit of the
  time-stepped Lindblad integration (two independent routes of O3).
* It is a density matrix, antisymmetric in <Z_j> under reflection of the chain
  (the model maps to itself under spin flip + reflection), and within 0.01 of
  the paper's closed form <Z_j> = cos(pi (j-1)/(L-1)) already at L = 4..6
  (the form is exact in the limit of strong driving and long chains); a wrong
  orientation of sigma^+- or a wrong sign of J fails this by O(1).
* The dense TJM schedule (O2: the Strang-ordered MCWF with at most one jump per
  step) reaches the same steady state within its standard error at dt = 0.1.
"""
import math

import numpy as np

from oracle import dense as O
from paper_2501_17913_gb300 import inputs as I


def _model(L):
    wl = I.edge_driven_xxx(L=L, chi_max=64, n_traj=1, T=1.0)
    return O.mpo_to_dense(wl.W), wl.jumps


def test_steady_state_equals_long_time_limit():
    L = 3
    H, jumps = _model(L)
    rho_ss = O.lindblad_steady_state(H, jumps, L)
    rho0 = np.zeros((8, 8), complex)
    rho0[0, 0] = 1.0
    rho_t = O.lindblad_evolve(H, jumps, L, rho0, [80.0])[0]      # gap 0.49: converged to e^-39
    assert np.abs(rho_ss - rho_t).max() < 1e-8


def test_steady_state_matches_the_closed_form_profile():
    for L in (4, 5, 6):
        H, jumps = _model(L)
        rho = O.lindblad_steady_state(H, jumps, L)
        assert abs(np.trace(rho) - 1.0) < 1e-12
        assert np.abs(rho - rho.conj().T).max() < 1e-10
        assert np.linalg.eigvalsh(0.5 * (rho + rho.conj().T)).min() > -1e-10
        z = np.array([O.expect(rho, I.Z, l, L) for l in range(L)])
        assert np.abs(z + z[::-1]).max() < 1e-9
        cos = np.cos(np.pi * np.arange(L) / (L - 1))
        assert np.abs(z - cos).max() < 0.01, (L, z)


def test_dense_tjm_schedule_reaches_the_steady_state():
    L, N, T, dt = 4, 64, 12.0, 0.1
    H, jumps = _model(L)
    rho = O.lindblad_steady_state(H, jumps, L)
    z_ss = np.array([O.expect(rho, I.Z, l, L) for l in range(L)])
    sim = O.DenseStrang(H, jumps, dt, L)
    n = int(round(T / dt))
    samples = list(range(0, n + 1, 5))
    psi0 = O.product_state(I.all_zero(L))
    window = [k for k, s in enumerate(samples) if s * dt >= 6.0]      # gap 0.32: relaxed by t = 6
    per_traj = []
    for t in range(N):
        v, _ = sim.run(psi0, t, 3, I.z_observables(L), n, samples)
        per_traj.append(v[window].mean(axis=0))
    per_traj = np.array(per_traj)
    m = per_traj.mean(axis=0)
    se = per_traj.std(axis=0, ddof=1) / math.sqrt(N)
    assert (np.abs(m - z_ss) <= 3 * se + 0.003).all(), (m, z_ss, se)
