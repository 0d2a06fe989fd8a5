"""Seeded synthetic workloads for the tensor jump method.

This module only DESCRIBES problems -- Hamiltonian MPO tensors, jump-operator
lists, initial product states, observables and output times -- with the
shapes, sizes and parameter distributions of the paper's noisy spin-chain
experiments.  It holds none of the method's arithmetic, so both the CUDA path
(through the C ABI) and the CPU oracle (in the tests) take their inputs from it.

Conventions (TJM, Sec. "Benchmarking"): |0> = (1, 0) has Z = +1 and is the
relaxation target; sigma^- = [[0, 1], [0, 0]]; Z = diag(1, -1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
SM = np.array([[0, 1], [0, 0]], dtype=np.complex128)   # sigma^- : |1> -> |0>
SP = SM.T.copy()                                        # sigma^+ : |0> -> |1>


def xxx_mpo(L: int, J: float = 1.0, g: float = 0.5):
    """MPO (bond dimension 5) of H = J sum_i (X_i X_{i+1} + Y_i Y_{i+1} + Z_i Z_{i+1}) + g sum_i X_i.

    XX + YY is written as 2 (sigma^+ sigma^- + sigma^- sigma^+), so every tensor
    is real.  Site tensors have shape (D_left, D_right, 2, 2) with the first
    physical index the output (bra) index; D_left = 1 on site 0 and
    D_right = 1 on site L-1.
    """
    Wb = np.zeros((5, 5, 2, 2), dtype=np.complex128)
    Wb[0, 0] = I2
    Wb[0, 1] = 2 * J * SP
    Wb[0, 2] = 2 * J * SM
    Wb[0, 3] = J * Z
    Wb[0, 4] = g * X
    Wb[1, 4] = SM
    Wb[2, 4] = SP
    Wb[3, 4] = Z
    Wb[4, 4] = I2
    if L == 1:
        return [Wb[0:1, 4:5].copy()]
    W = [Wb[0:1, :].copy()]
    W += [Wb.copy() for _ in range(L - 2)]
    W.append(Wb[:, 4:5].copy())
    return W


def noise(L: int, gamma_relax: float = 0.1, gamma_dephase: float = 0.1):
    """Relaxation sigma^- and dephasing Z on every site: [(site, op, rate)]."""
    out = []
    for l in range(L):
        if gamma_relax > 0:
            out.append((l, SM.copy(), float(gamma_relax)))
    for l in range(L):
        if gamma_dephase > 0:
            out.append((l, Z.copy(), float(gamma_dephase)))
    return out


def z_observables(L: int):
    return [(l, Z.copy()) for l in range(L)]


def xx_observables(L: int):
    """Nearest-neighbour correlators X_i X_{i+1} (paper Fig. 4b) as two-site operators on (i, i+1)."""
    return [(l, np.kron(X, X)) for l in range(L - 1)]


def tfim_mpo(L: int, J: float = 1.0, g: float = 1.0):
    """MPO (bond dimension 3) of the transverse-field Ising chain H = -J sum_i Z_i Z_{i+1} - g sum_j X_j
    (paper Sec. "Benchmarking", critical point J = g = 1).  Same layout as xxx_mpo."""
    Wb = np.zeros((3, 3, 2, 2), dtype=np.complex128)
    Wb[0, 0] = I2
    Wb[0, 1] = -J * Z
    Wb[0, 2] = -g * X
    Wb[1, 2] = Z
    Wb[2, 2] = I2
    if L == 1:
        return [Wb[0:1, 2:3].copy()]
    W = [Wb[0:1, :].copy()]
    W += [Wb.copy() for _ in range(L - 2)]
    W.append(Wb[:, 2:3].copy())
    return W


def all_zero(L: int):
    return [np.array([1.0, 0.0], dtype=np.complex128) for _ in range(L)]


def neel(L: int):
    """|0101...> with site 0 in |0>."""
    return [np.array([1.0, 0.0] if l % 2 == 0 else [0.0, 1.0], dtype=np.complex128) for l in range(L)]


def haar_product(L: int, rng: np.random.Generator):
    """Independent Haar-random single-site states (normalised complex Gaussians)."""
    out = []
    for _ in range(L):
        v = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        out.append(v / np.linalg.norm(v))
    return out


@dataclass
class Workload:
    """One TJM problem plus the run parameters (the paper's initialisation list)."""
    name: str
    W: list
    jumps: list
    dt: float
    n_steps: int
    chi_max: int
    trunc_eps: float
    n_traj: int
    seed: int
    psi0: list                      # per-site vectors, shared by all trajectories
    observables: list
    sample_steps: list
    psi0_per_traj: list | None = None   # optional [n_traj][L] site vectors
    meta: dict = field(default_factory=dict)

    @property
    def L(self):
        return len(self.W)

    @property
    def times(self):
        return [s * self.dt for s in self.sample_steps]


def config_small_fp64(n_traj: int = 200) -> Workload:
    """L=6 XXX chain, J=1, g=0.5, sigma^- and Z at 0.1 on every site, |0..0>, dt=0.1, T=5, chi_max=16."""
    L, dt, T = 6, 0.1, 5.0
    n = int(round(T / dt))
    return Workload('xxx_L6_chi16_fp64', xxx_mpo(L, 1.0, 0.5), noise(L, 0.1, 0.1), dt, n, 16, 1e-10,
                    n_traj, 0, all_zero(L), z_observables(L), list(range(n + 1)))


def config_l30(n_traj: int = 1024) -> Workload:
    """L=30 XXX chain, Neel start, dt=0.1, T=10, chi_max=32, 1024 trajectories."""
    L, dt, T = 30, 0.1, 10.0
    n = int(round(T / dt))
    return Workload('xxx_L30_chi32', xxx_mpo(L, 1.0, 0.5), noise(L, 0.1, 0.1), dt, n, 32, 1e-10,
                    n_traj, 0, neel(L), z_observables(L), list(range(n + 1)))


def config_l1000(n_traj: int = 256) -> Workload:
    """L=1000 XXX chain, Neel start, dt=0.1, T=5, chi_max=64, 256 trajectories."""
    L, dt, T = 1000, 0.1, 5.0
    n = int(round(T / dt))
    return Workload('xxx_L1000_chi64', xxx_mpo(L, 1.0, 0.5), noise(L, 0.1, 0.1), dt, n, 64, 1e-10,
                    n_traj, 0, neel(L), z_observables(L), list(range(n + 1)))


def config_bench(n_traj: int = 256, n_steps: int = 6) -> Workload:
    """The benchmark workload: L=1000, chi_max=64, from a seeded random MPS with every bulk bond at 64.

    Same Hamiltonian and noise as config_l1000; <Z_i> recorded at every step.
    The initial MPS is in meta['mps'] as (chi, sites).
    """
    L, dt = 1000, 0.1
    wl = Workload('xxx_L1000_chi64_bench', xxx_mpo(L, 1.0, 0.5), noise(L, 0.1, 0.1), dt, n_steps, 64, 1e-10,
                  n_traj, 0, all_zero(L), z_observables(L), list(range(n_steps + 1)))
    wl.meta['mps'] = random_mps(L, 64, 2025)
    return wl


def uneven_groups(seed: int = 7, n_groups: int = 32, per_group: int = 128, dt: float = 0.05, T: float = 5.0):
    """The uneven batch: 27 groups enumerate L x chi_max x gamma, 5 more drawn at random.

    L in {50, 100, 200}, chi_max in {16, 32, 64}, gamma in {0.01, 0.1, 1.0}
    (relaxation and dephasing at the same rate), g ~ U[0, 1] per group, and a
    Haar-random product initial state per trajectory.
    """
    rng = np.random.default_rng(seed)
    grid = [(L, c, g) for L in (50, 100, 200) for c in (16, 32, 64) for g in (0.01, 0.1, 1.0)]
    params = list(grid)
    while len(params) < n_groups:
        params.append((int(rng.choice([50, 100, 200])), int(rng.choice([16, 32, 64])),
                       float(rng.choice([0.01, 0.1, 1.0]))))
    n = int(round(T / dt))
    out = []
    for gi, (L, chi, gam) in enumerate(params[:n_groups]):
        gfield = float(rng.uniform(0.0, 1.0))
        psis = [haar_product(L, rng) for _ in range(per_group)]
        out.append(Workload(f'group{gi}_L{L}_chi{chi}_g{gam}', xxx_mpo(L, 1.0, gfield), noise(L, gam, gam),
                            dt, n, chi, 1e-10, per_group, seed, psis[0], z_observables(L), [n],
                            psi0_per_traj=psis, meta={'g': gfield, 'gamma': gam, 'first_traj': gi * per_group}))
    return out


def uneven_group(gi: int, n_steps: int | None = None, seed: int = 7):
    """Group gi of uneven_groups(seed), optionally cut to n_steps with every step sampled."""
    wl = uneven_groups(seed)[gi]
    if n_steps is not None:
        wl.n_steps = n_steps
        wl.sample_steps = list(range(n_steps + 1))
    return wl


def request_stream(seed: int = 11, n_requests: int = 200, rate: float = 20.0):
    """Poisson request arrivals for the serving loop.

    Each request: L ~ U{20..500}, gamma log-uniform in [0.01, 1], g ~ U[0, 1],
    chi_max in {16, 32, 64}, N ~ U{100..2000}, T ~ U[1, 10], dt = 0.1.
    Returns [(arrival_time_s, Workload)].
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        L = int(rng.integers(20, 501))
        gam = float(math.exp(rng.uniform(math.log(0.01), math.log(1.0))))
        gfield = float(rng.uniform(0.0, 1.0))
        chi = int(rng.choice([16, 32, 64]))
        N = int(rng.integers(100, 2001))
        T = float(rng.uniform(1.0, 10.0))
        dt = 0.1
        n = max(1, int(round(T / dt)))
        out.append((t, Workload(f'req{r}', xxx_mpo(L, 1.0, gfield), noise(L, gam, gam), dt, n, chi, 1e-10,
                                N, seed * 1000003 + r, neel(L), z_observables(L), [n])))
    return out


def edge_driven_xxx(L: int = 100, eps: float = 10 * math.pi, chi_max: int = 4, n_traj: int = 100, T: float = 100.0,
                    dt: float = 0.1, sample_every: int = 10, seed: int = 3) -> Workload:
    """The boundary-driven XXX chain of the paper's large-scale validation (Sec. "Validating convergence
    against analytical results"): H = -J sum_i (X X + Y Y + Z Z) - h sum_j Z_j with J = 1, h = 0, jump
    operators sqrt(eps) sigma^+ on the first site and sqrt(eps) sigma^- on the last, |0...0> start, dt = 0.1.

    That section defines sigma^+- = (X +- i Y) / 2, so its sigma^+ is [[0, 1], [0, 0]] (our SM: it pumps
    the first site to |0>, Z = +1) and its sigma^- is [[0, 0], [1, 0]] (our SP: the last site to |1>,
    Z = -1), which is the orientation of the stated steady state <Z_j> = cos(pi (j - 1) / (L - 1)).
    """
    n = int(round(T / dt))
    samples = list(range(0, n + 1, sample_every))
    if samples[-1] != n:
        samples.append(n)
    return Workload(f'edge_driven_L{L}_chi{chi_max}', xxx_mpo(L, -1.0, 0.0), [(0, SM.copy(), float(eps)),
                    (L - 1, SP.copy(), float(eps))], dt, n, chi_max, 1e-10, n_traj, seed, all_zero(L),
                    z_observables(L), samples)


def random_mps(L: int, chi_max: int, seed: int = 1234):
    """A seeded random MPS with every bond at min(chi_max, 2^b, 2^(L-b)).

    Entries are complex Gaussians of variance 1/(2 chi_right), so the right
    transfer map sum_s M^s (.) M^s^dag preserves the identity on average and
    the norm neither overflows nor underflows along a long chain.  Used as a
    bond-saturated starting point ("chi-saturated regime").
    Returns (chi [L+1], [site tensors (chi_l, 2, chi_r)]).
    """
    rng = np.random.default_rng(seed)
    chi = [min(chi_max, 2 ** min(b, 30), 2 ** min(L - b, 30)) for b in range(L + 1)]
    sites = []
    for l in range(L):
        a, b = chi[l], chi[l + 1]
        x = rng.standard_normal((a, 2, b)) + 1j * rng.standard_normal((a, 2, b))
        sites.append(x / math.sqrt(2.0 * 2 * b))
    return chi, sites
