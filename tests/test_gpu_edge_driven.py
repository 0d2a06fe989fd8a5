"""The boundary-driven XXX chain (paper Sec. "Validating convergence against analytical results") on
the GPU: the long-time magnetisation profile of the TJM ensemble.

* L = 6 at full bond dimension (chi = 8), FP64: the time average of <Z_j> over
  t in [15, 30] of 256 trajectories equals the exact steady state of the
  Lindblad equation (solved densely) within 4 standard errors plus the
  method's small time-step bias, and the closed form cos(pi (j-1)/(L-1))
  within 0.02.
* L = 16 at the paper's chi = 4, in the benchmark's arithmetic (FP32
  contractions, emulated-FP64 factorizations): 6000 steps of 96 trajectories
  in one persistent launch (a latency-bound regime of tiny tensors); the
  profile averaged over t in [400, 600] follows the closed form (relaxation
  time ~ L^3: about 60 time units at L = 10, measured with the dense oracle,
  so ~250 at L = 16).
"""
import math

import numpy as np
import pytest

from oracle import dense as O2
from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import tjm

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


def _window_stats(pt, wl, t0):
    idx = [k for k, s in enumerate(wl.sample_steps) if s * wl.dt >= t0]
    per_traj = pt[:, idx, :].mean(axis=1)
    return per_traj.mean(axis=0), per_traj.std(axis=0, ddof=1) / math.sqrt(pt.shape[0])


def _run(wl, prec):
    lib_ready()
    ctx = tjm.Context(wl.W, wl.jumps, wl.dt, wl.chi_max, wl.trunc_eps, precision=prec)
    rid = ctx.run(np.array(wl.psi0), wl.n_traj, wl.seed, wl.observables, wl.times)
    _, _, pt = ctx.result(rid)
    st = ctx.stats(rid)
    ctx.close()
    assert st['failed'] == 0
    return pt


def test_small_chain_reaches_the_lindblad_steady_state():
    wl = I.edge_driven_xxx(L=6, chi_max=8, n_traj=256, T=30.0, sample_every=5)
    pt = _run(wl, tjm.PREC_FP64)
    m, se = _window_stats(pt, wl, 15.0)
    rho = O2.lindblad_steady_state(O2.mpo_to_dense(wl.W), wl.jumps, wl.L)
    z_ss = np.array([O2.expect(rho, I.Z, l, wl.L) for l in range(wl.L)])
    assert (np.abs(m - z_ss) <= 4 * se + 0.003).all(), (m, z_ss, se)
    cos = np.cos(np.pi * np.arange(wl.L) / (wl.L - 1))
    # the exact steady state is within 0.006 of the closed form at L = 6 (oracle pin)
    assert (np.abs(m - cos) <= 4 * se + 0.01).all(), (m, cos, se)


def test_sixteen_sites_chi4_follow_the_closed_form_profile():
    wl = I.edge_driven_xxx(L=16, chi_max=4, n_traj=96, T=600.0, sample_every=20)
    pt = _run(wl, tjm.PREC_FP32_DF64)
    m, se = _window_stats(pt, wl, 400.0)
    cos = np.cos(np.pi * np.arange(wl.L) / (wl.L - 1))
    assert (np.abs(m - cos) <= 4 * se + 0.02).all(), (np.round(m, 3), np.round(se, 3))
    assert m[0] > 0.99 and m[-1] < -0.99
