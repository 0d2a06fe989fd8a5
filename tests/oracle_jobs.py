"""Picklable oracle jobs for the process pool (test helper)."""
import numpy as np

from oracle import mps_tjm as O1
from paper_2501_17913_gb300 import inputs as I


def workload(name, **kw):
    return getattr(I, name)(**kw)


def run_traj(args):
    """(workload factory name, kwargs, traj index, options) -> (values, stats summary)."""
    name, kw, traj, opts = args
    wl = workload(name, **kw)
    prob = O1.Problem(wl.W, wl.jumps, wl.dt, wl.chi_max, wl.trunc_eps,
                      krylov_tol=opts.get('krylov_tol', 1e-12), krylov_max=opts.get('krylov_max', 30),
                      exact=opts.get('exact', False))
    psi = wl.psi0_per_traj[traj] if wl.psi0_per_traj is not None else wl.psi0
    if 'mps' in wl.meta:
        mps = [np.array(x, dtype=np.complex128) for x in wl.meta['mps'][1]]
    else:
        mps = O1.padded_product_mps(psi) if opts.get('exact', False) else O1.product_mps(psi)
    gid = opts.get('traj_offset', 0) + traj
    n_steps = opts.get('n_steps', wl.n_steps)
    samples = [s for s in wl.sample_steps if s <= n_steps]
    v, st = O1.run_trajectory(prob, mps, gid, wl.seed, wl.observables, n_steps, samples)
    # smallest decision margin among the decisions taken up to each sampled step
    upto = []
    for s in samples:
        m = [min(r['margin1'], r['margin2']) for r in st['records'] if r['step'] <= s]
        upto.append(min(m) if m else np.inf)
    return v, {'jumps': st['jumps'], 'min_margin1': st['min_margin1'], 'min_margin2': st['min_margin2'],
               'margin_upto': np.array(upto),
               'matvecs': st['matvecs'], 'updates': st['updates'], 'final_bonds': st['final_bonds'],
               'trunc_margin': st['trunc_margin'], 'cut_gap': st['cut_gap']}
