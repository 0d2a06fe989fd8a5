"""Two-site observables (Fig. 4b) and the first-order Trotter baseline (Fig. 4a) on the GPU.

* L = 6 XXX chain in FP64, 32 trajectories: <Z_i> and <X_i X_{i+1}> per
  trajectory equal the oracle's (same Philox streams) to 1e-10, for the
  Strang-split TJM and for the first-order baseline.
* The 10-site TFIM of Sec. "Benchmarking" (J = g = 1, sigma^- and Z at 0.1,
  |0..0>): <X_5> at Jt = 1.  The second-order TJM at
  dt = 0.1 agrees with the exact Lindblad value within its Monte Carlo error
  (the paper's point: the Strang splitting pushes the time-step error below the
  sampling error); the first-order baseline at dt = 0.5 is biased by many
  standard errors.  4096 trajectories per arm.
"""
import math

import numpy as np
import pytest

from oracle import dense as O2
from oracle import mps_tjm as O1
from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import tjm

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order", [2, 1])
def test_two_site_observables_per_trajectory_fp64(order):
    lib_ready()
    L, n, N, chi = 6, 20, 32, 8
    W = I.xxx_mpo(L, 1.0, 0.5)
    jumps = I.noise(L, 0.1, 0.1)
    obs = I.xx_observables(L)[:2] + I.z_observables(L) + I.xx_observables(L)[2:]
    steps = list(range(n + 1))
    ctx = tjm.Context(W, jumps, 0.1, chi, 1e-10, precision=tjm.PREC_FP64, trotter_order=order)
    rid = ctx.run(np.array(I.neel(L)), N, 4, obs, [0.1 * s for s in steps])
    _, _, pt = ctx.result(rid)
    m1, m2 = ctx.margins(rid)
    ctx.close()
    prob = O1.Problem(W, jumps, 0.1, chi, 1e-10)
    ok = 0
    for t in range(N):
        v, st = O1.run_trajectory(prob, O1.product_mps(I.neel(L)), t, 4, obs, n, steps, order=order)
        if min(st['min_margin1'], st['min_margin2']) < 1e-9:
            continue
        assert np.abs(pt[t] - v).max() < 1e-10, (t, np.abs(pt[t] - v).max())
        ok += 1
    assert ok >= N - 2


def _tfim_exact(L, site, t):
    W = I.tfim_mpo(L, 1.0, 1.0)
    rho0 = np.zeros((2 ** L, 2 ** L), complex)
    rho0[0, 0] = 1.0
    rho = O2.lindblad_evolve(O2.mpo_to_dense(W), I.noise(L, 0.1, 0.1), L, rho0, [t], rtol=1e-10, atol=1e-12)[0]
    return O2.expect(rho, I.X, site, L)


def test_tfim_convergence_second_vs_first_order():
    lib_ready()
    L, site, N = 10, 4, 4096           # <X^[5]> of the paper is the 5th site, index 4
    exact = _tfim_exact(L, site, 1.0)
    W = I.tfim_mpo(L, 1.0, 1.0)
    res = {}
    for order, dt in [(2, 0.1), (1, 0.5)]:
        n = int(round(1.0 / dt))
        ctx = tjm.Context(W, I.noise(L, 0.1, 0.1), dt, 32, 1e-10, precision=tjm.PREC_FP32_DF64, trotter_order=order)
        rid = ctx.run(np.array(I.all_zero(L)), N, 21, [(site, I.X)], [n * dt])
        _, _, pt = ctx.result(rid)
        ctx.close()
        v = pt[:, 0, 0]
        res[(order, dt)] = (abs(v.mean() - exact), v.std(ddof=1) / math.sqrt(N))
    err2, se2 = res[(2, 0.1)]
    err1, se1 = res[(1, 0.5)]
    assert err2 <= 4 * se2 + 1e-3, res
    assert err1 > 6 * se1, res
    # the Monte Carlo error of N trajectories, the paper's C / sqrt(N) with C ~ 0.1
    assert se2 * math.sqrt(N) < 0.5, res
