"""Oracle pins for the first-order Trotter baseline of Fig. 4a (dotted lines).

* Exact mode (padded full bond dimension): the MPS-TJM with order=1 equals the
  dense first-order schedule (O2, order=1) trajectory by trajectory, one- and
  two-site observables included.
* On the 4-site TFIM at dt = 0.5 the first-order ensemble is biased away from
  the exact Lindblad value of <X> at Jt = 1 by more than its standard error,
  and by more than the second-order (Strang) ensemble on the same random
  numbers: the time-step error the paper's second-order splitting removes.
"""
import math

import numpy as np

from oracle import dense as O2
from oracle import mps_tjm as O1
from paper_2501_17913_gb300 import inputs as I


def test_first_order_exact_mode_equals_dense_per_trajectory():
    L, n = 4, 6
    W = I.xxx_mpo(L, 1.0, 0.5)
    jumps = I.noise(L, 0.3, 0.2)
    obs = I.z_observables(L) + I.xx_observables(L)
    prob = O1.Problem(W, jumps, 0.1, 16, 0.0, exact=True)
    ds = O2.DenseStrang(O2.mpo_to_dense(W), jumps, 0.1, L)
    psi = I.neel(L)
    for t in range(6):
        v1, _ = O1.run_trajectory(prob, O1.padded_product_mps(psi), t, 5, obs, n, list(range(n + 1)), order=1)
        v2, _ = ds.run(O2.product_state(psi), t, 5, obs, n, list(range(n + 1)), order=1)
        assert np.abs(v1 - v2).max() < 1e-10, t


def test_first_order_bias_exceeds_second_order_on_tfim():
    L, dt, N = 4, 0.5, 3000
    W = I.tfim_mpo(L, 1.0, 1.0)
    H = O2.mpo_to_dense(W)
    jumps = I.noise(L, 0.1, 0.1)
    site = 1
    rho0 = np.zeros((2 ** L, 2 ** L), complex)
    rho0[0, 0] = 1.0
    exact = O2.expect(O2.lindblad_evolve(H, jumps, L, rho0, [1.0])[0], I.X, site, L)
    ds = O2.DenseStrang(H, jumps, dt, L)
    psi0 = O2.product_state(I.all_zero(L))
    vals = {1: [], 2: []}
    for order in (1, 2):
        for t in range(N):
            v, _ = ds.run(psi0, t, 17, [(site, I.X)], 2, [2], order=order)
            vals[order].append(v[0, 0])
    err = {o: abs(np.mean(vals[o]) - exact) for o in (1, 2)}
    se = {o: np.std(vals[o], ddof=1) / math.sqrt(N) for o in (1, 2)}
    assert err[1] > 4 * se[1], (err, se)
    assert err[1] > 2 * err[2], (err, se)
