"""Helpers shared by the GPU tests: running a workload through the C ABI."""
import numpy as np

from paper_2501_17913_gb300 import tjm
from paper_2501_17913_gb300 import build as _build


def lib_ready():
    _build.build()
    return tjm.load()


def run_gpu(wl, precision, n_traj=None, exact=False, first_traj=0, n_steps=None, krylov_tol=0.0, krylov_max=30,
            psi=None, **opts):
    """Run a Workload on the GPU; returns (per_traj [N][T][O], mean, sem, stats, margins, ctx)."""
    lib_ready()
    n = wl.n_traj if n_traj is None else n_traj
    steps = wl.sample_steps if n_steps is None else [s for s in wl.sample_steps if s <= n_steps]
    times = [s * wl.dt for s in steps]
    ctx = tjm.Context(wl.W, wl.jumps, wl.dt, wl.chi_max, wl.trunc_eps, precision=precision, exact=exact,
                      krylov_tol=krylov_tol, krylov_max=krylov_max, **opts)
    if psi is None:
        psi = np.array(wl.psi0_per_traj[first_traj:first_traj + n]) if wl.psi0_per_traj is not None else np.array(wl.psi0)
    rid = ctx.run(psi, n, wl.seed, wl.observables, times, first_traj=first_traj)
    mean, sem, pt = ctx.result(rid)
    st = ctx.stats(rid)
    m1, m2 = ctx.margins(rid)
    return pt, mean, sem, st, (m1, m2), ctx
