"""The oracle's trajectory average against the exact Lindblad solution (Thm. 1, App. A).

L = 6 XXX chain, sigma^- and Z on every site at 0.1, |0..0>, dt = 0.1, T = 5,
chi_max = 16, 200 trajectories from Philox seed 0: <Z_i>(t) for all sites and
all 50 sampled times against the 64 x 64 density-matrix solution.

Criterion (multiplicity rule for 300 simultaneous comparisons): at least 99 %
of the points within 3 standard errors and none beyond 5.  The standard error
is floored at 1e-3, the size of the method's own deterministic time-step error
at dt = 0.1 (Strang splitting and TDVP are second order, Sec. "Error
measures"): at the earliest times almost no trajectory has jumped, the sample
spread is ~1e-16 and only that deterministic error is left.
"""
import numpy as np

from oracle import dense as O2
from oracle import mps_tjm as O1
from paper_2501_17913_gb300 import inputs as I

from _pool import oracle_pool
from oracle_jobs import run_traj


def test_tjm_ensemble_matches_lindblad_within_standard_errors():
    wl = I.config_small_fp64()
    with oracle_pool() as pool:
        res = pool.map(run_traj, [('config_small_fp64', {}, t, {}) for t in range(wl.n_traj)])
    vals = np.array([r[0] for r in res])
    mean, sem = O1.ensemble(vals)
    H = O2.mpo_to_dense(wl.W)
    psi = O2.product_state(wl.psi0)
    rhos = O2.lindblad_evolve(H, wl.jumps, wl.L, np.outer(psi, psi.conj()), wl.times)
    exact = np.array([[O2.expect(r, I.Z, l, wl.L) for l in range(wl.L)] for r in rhos])
    assert np.allclose(mean[0], exact[0], atol=1e-14)
    z = np.abs(mean - exact)[1:] / np.maximum(sem[1:], 1e-3)
    assert np.mean(z < 3) >= 0.99, np.mean(z < 3)
    assert z.max() < 5, z.max()
    assert sum(r[1]['jumps'] for r in res) > 100      # the noise is actually exercised
