"""Write the stored oracle outputs used by the GPU parity tests at full size.

Calls only the CPU oracle (oracle/) and the input generator; nothing here
comes from the CUDA path.  Usage:

    python tests/golden/make_golden.py l30      # L=30, chi=32: 32 sampled trajectories, all 100 steps
    python tests/golden/make_golden.py l1000    # L=1000, chi=64 from Neel: 8 sampled trajectories, 3 steps
    python tests/golden/make_golden.py bench    # the benchmark workload (random chi=64 MPS): 4 trajectories, 1 step
    python tests/golden/make_golden.py tfim     # exact <X_5>(t=1) of the L=10 TFIM with relaxation + dephasing
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

from _pool import oracle_pool  # noqa: E402
from oracle_jobs import run_traj  # noqa: E402

SETS = {
    # name: (workload factory, kwargs, sampled global trajectory ids, options)
    "l30": ("config_l30", {}, sorted([0, 137, 274, 411, 548, 685, 822, 959] + list(range(20, 1024, 43))), {}),
    "l1000": ("config_l1000", {}, [0, 33, 67, 101, 150, 201, 230, 255], {"n_steps": 3}),
    "bench": ("config_bench", {}, [0, 64, 128, 192], {"n_steps": 1}),
}


def make(name):
    fac, kw, trajs, opts = SETS[name]
    with oracle_pool(min(os.cpu_count() or 1, 16, len(trajs))) as pool:
        res = pool.map(run_traj, [(fac, kw, t, opts) for t in trajs])
    vals = np.array([r[0] for r in res])
    m1 = np.array([r[1]["min_margin1"] for r in res])
    m2 = np.array([r[1]["min_margin2"] for r in res])
    tm = np.array([r[1]["trunc_margin"] for r in res])
    upto = np.array([r[1]["margin_upto"] for r in res])
    out = os.path.join(HERE, "oracle_%s.npz" % name)
    np.savez_compressed(out, traj=np.array(trajs), values=vals, margin_jump=m1, margin_pick=m2, trunc_margin=tm,
                        margin_upto=upto, n_steps=opts.get("n_steps", -1))
    print(out, vals.shape)


def make_tfim():
    """<X> on site index 4 at t = 1 of the L = 10 transverse-field Ising chain (J = g = 1) with sigma^- and Z
    at rate 0.1 on every site, from |0...0>: the dense Lindblad density matrix (O3) integrated to 1e-10."""
    import json
    from oracle import dense as O2
    from paper_2501_17913_gb300 import inputs as I
    L, site, t = 10, 4, 1.0
    H = O2.mpo_to_dense(I.tfim_mpo(L, 1.0, 1.0))
    rho0 = np.zeros((2 ** L, 2 ** L), complex)
    rho0[0, 0] = 1.0
    rho = O2.lindblad_evolve(H, I.noise(L, 0.1, 0.1), L, rho0, [t], rtol=1e-10, atol=1e-12)[0]
    out = os.path.join(HERE, "tfim_l10_x5_t1.json")
    with open(out, "w") as f:
        json.dump({"L": L, "site": site, "t": t, "J": 1.0, "g": 1.0, "gamma_relax": 0.1, "gamma_dephase": 0.1,
                   "x": float(O2.expect(rho, I.X, site, L)), "rtol": 1e-10, "atol": 1e-12}, f, indent=1)
    print(out)


if __name__ == "__main__":
    for n in sys.argv[1:]:
        make_tfim() if n == "tfim" else make(n)
