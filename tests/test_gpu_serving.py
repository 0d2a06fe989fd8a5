"""Serving loop: requests admitted while others run must give the same result as alone."""
import time

import numpy as np
import pytest

from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import tjm
from paper_2501_17913_gb300.serve import Server, state_bytes

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


def _requests():
    specs = [(8, 4, 6, 5, 0.3, 0.0), (12, 8, 10, 6, 0.1, 0.0), (16, 8, 6, 4, 0.5, 0.05), (10, 4, 8, 3, 0.05, 0.1),
             (14, 8, 5, 6, 0.2, 0.15)]
    out = []
    for k, (L, chi, N, n, g, t_arr) in enumerate(specs):
        wl = I.Workload('req%d' % k, I.xxx_mpo(L, 1.0, 0.3 + 0.1 * k), I.noise(L, g, g), 0.1, n, chi, 1e-10, N,
                        100 + k, I.neel(L), I.z_observables(L), list(range(n + 1)))
        out.append((t_arr, wl))
    return out


@pytest.mark.parametrize("budget", [None, "tight"])
def test_results_in_the_mix_equal_results_alone(budget):
    lib_ready()
    reqs = _requests()
    srv = Server(precision=tjm.PREC_FP32_DEC32, mem_budget=None, steps_per_tick=1, keep_per_traj=True)
    if budget == "tight":
        # the launch scratch for the largest request plus two requests' state: forces queueing for memory
        scratch = srv.anchor.scratch_bytes(max(wl.chi_max for _, wl in reqs), max(wl.L for _, wl in reqs))
        srv.budget = scratch + 2 * max(state_bytes(wl, tjm.PREC_FP32_DEC32) for _, wl in reqs)
    t0 = time.perf_counter()
    for t_arr, wl in reqs:
        srv.submit(wl, t0 + t_arr)
    done = srv.drain()
    rep = srv.report(t0, time.perf_counter())
    assert rep['requests'] == len(reqs)
    assert rep['p99_latency_s'] >= rep['p50_latency_s'] > 0
    # continuous batching: some request was admitted while another was still running
    assert any(a.admitted < b.done and a.admitted > b.admitted for a in done for b in done if a is not b)
    for r in done:
        wl = r.wl
        ctx = tjm.Context(wl.W, wl.jumps, wl.dt, wl.chi_max, wl.trunc_eps, precision=tjm.PREC_FP32_DEC32)
        rid = ctx.run(np.array(wl.psi0), wl.n_traj, wl.seed, wl.observables, wl.times)
        alone = ctx.result(rid)[2]
        assert np.array_equal(alone, r.per_traj), r.rid
        ctx.close()
    srv.close()
