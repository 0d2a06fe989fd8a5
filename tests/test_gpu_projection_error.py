"""The 1TDVP projection error (paper Sec. "Error measures") computed by the kernel's diagnostic sweep,
against the oracle's dense definition ||(I - P) H psi|| on the same measured states.

* t = 0 of a Neel start: the closed form 2 |J| sqrt(L - 1).
* L = 6, chi_max = 4 (truncated, so the error is nonzero), FP64: every sampled
  state of 8 trajectories, per trajectory, within 1e-9 of the oracle.
* Full bond dimension (exact mode): zero to rounding.
"""
import math

import numpy as np
import pytest

from oracle import mps_tjm as O1
from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import tjm

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


def test_projection_error_matches_oracle_per_trajectory():
    lib_ready()
    L, n, N, chi = 6, 12, 8, 4
    W = I.xxx_mpo(L, 1.0, 0.5)
    jumps = I.noise(L, 0.1, 0.1)
    steps = list(range(0, n + 1, 2))
    ctx = tjm.Context(W, jumps, 0.1, chi, 1e-10, precision=tjm.PREC_FP64, projection_error=True)
    rid = ctx.run(np.array(I.neel(L)), N, 8, I.z_observables(L), [0.1 * s for s in steps])
    _, _, pt = ctx.result(rid)
    ctx.close()
    eps_gpu = pt[:, :, -1]
    assert np.abs(eps_gpu[:, 0] - 2 * math.sqrt(L - 1)).max() < 1e-10
    prob = O1.Problem(W, jumps, 0.1, chi, 1e-10)
    for t in range(N):
        got = {}
        v, st = O1.run_trajectory(prob, O1.product_mps(I.neel(L)), t, 8, I.z_observables(L), n, steps,
                                  on_sample=lambda j, s: got.__setitem__(j, O1.projection_error(s, W)))
        if min(st['min_margin1'], st['min_margin2']) < 1e-9:
            continue
        ref = np.array([got[s] for s in steps])
        assert np.abs(eps_gpu[t] - ref).max() < 1e-9, (t, eps_gpu[t], ref)
        assert np.abs(pt[t, :, :-1] - v).max() < 1e-10
    assert eps_gpu[:, 1:].max() > 1e-3          # truncated: the projection error is not zero


def test_projection_error_vanishes_at_full_bond_dimension():
    lib_ready()
    L, n = 6, 6
    W = I.xxx_mpo(L, 1.0, 0.5)
    ctx = tjm.Context(W, I.noise(L, 0.1, 0.1), 0.1, 16, 0.0, precision=tjm.PREC_FP64, exact=True,
                      projection_error=True)
    rid = ctx.run(np.array(I.neel(L)), 4, 2, I.z_observables(L), [0.1 * s for s in range(n + 1)])
    _, _, pt = ctx.result(rid)
    ctx.close()
    assert np.abs(pt[:, :, -1]).max() < 1e-5      # eps = sqrt(rounding of sums of O(L^2))
